// pcg.cu -- the space-charge Poisson solve M Phi = f (App. B, eq. poisson_mat)
// as one persistent cooperative kernel per solve: Jacobi-preconditioned
// conjugate gradients, warm-started from the previous potential.
//
// The matrix is stored as sliced ELLPACK with slices of 32 rows (one warp
// per slice, one thread per row, columns of a slice interleaved so each load
// of the warp is coalesced).  Each warp owns the same slices in every phase,
// so a thread only ever reads its own rows' x, r, z, p; neighbours' z and p
// are gathered after a grid barrier through L2 (ld.global.cg).
//
// One CG iteration needs two grid-wide reductions.  The search direction is
// not materialised in a separate phase: the SpMV forms p = z + beta p_old on
// the fly from the gathered z and p_old (double-buffered p), so two grid
// barriers per iteration suffice.  Dot products: butterfly within the warp,
// in warp order within the block, then every block sums the per-block
// partials in block order -- a fixed order, so all blocks obtain identical
// scalars and the result is reproducible run to run.
//
// FP32_IR: the inner CG runs in FP32 (matrix values, vectors, SpMV) with
// FP64 dot products; the outer loop recomputes the residual f - M x in FP64
// and applies the correction in FP64 (iterative refinement).
//
// The grid barrier waits with an iteration limit: a block that waits too
// long records PIC_ERR_TIMEOUT and the whole kernel returns.
#include "common.cuh"

namespace pf {

constexpr int PCG_BLOCK = 256;
constexpr int PCG_WARPS = PCG_BLOCK / 32;
constexpr long long SPIN_LIMIT = 1LL << 25;
#define FULL_MASK 0xffffffffu

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile_i32(const int *p)
{
    return *(const volatile int *)p;
}

// Grid-wide barrier over co-resident blocks (cooperative launch).  Returns
// false when the wait ran out or another block already failed.
__device__ bool grid_sync(DevState *st)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned g = ld_acquire_u32(&st->bar_gen);
        __threadfence();
        unsigned arrived = atomicAdd(&st->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&st->bar_count, 0u);
            __threadfence();
            atomicAdd(&st->bar_gen, 1u);
        } else {
            long long spins = 0;
            while (ld_acquire_u32(&st->bar_gen) == g) {
                if (++spins > SPIN_LIMIT) {
                    atomicCAS(&st->err, 0, PIC_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                if (spins > 32)
                    __nanosleep(40);
            }
        }
        __threadfence();
        if (ld_volatile_i32(&st->err) == PIC_ERR_TIMEOUT)
            ok = 0;
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

// Sum NV per-thread values over the whole grid; out[] identical in every
// block.  `set` alternates between calls so a fast block never overwrites
// partials a slow block has not read yet.
template <int NV>
__device__ bool grid_sum(const double (&v)[NV], double *partials, int set, DevState *st,
                         double (&out)[NV])
{
    __shared__ double red[PCG_WARPS][NV];
    __shared__ double res[NV];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s = warp_sum(v[k]);
        if (lane == 0)
            red[wid][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < PCG_WARPS; ++w)
            s += red[w][threadIdx.x];
        partials[((size_t)set * gridDim.x + blockIdx.x) * 4 + threadIdx.x] = s;
    }
    if (!grid_sync(st))
        return false;
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int b = lane; b < (int)gridDim.x; b += 32)
                s += __ldcg(partials + ((size_t)set * gridDim.x + b) * 4 + k);
            s = warp_sum(s);
            if (lane == 0)
                res[k] = s;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k)
        out[k] = res[k];
    return true;
}

// f_i = (q w_sp / eps0) W_i 2^-S + f_Neumann,i (eq. poisson_rhs), written
// without contraction so it equals the plain evaluation bit for bit
__device__ __forceinline__ double rhs_entry(const PcgArgs &a, int row)
{
    if (row >= a.n)
        return 0.0;
    double w = (double)(long long)a.W[a.dof_node[row]];
    return __dadd_rn(__dmul_rn(a.coef, __dmul_rn(w, a.wscale)), a.fN[row]);
}

__device__ __forceinline__ void finish(const PcgArgs &a, int it, double relres, int status,
                                       int outer = 0)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (status)
            atomicCAS(&a.st->err, 0, status);
        if (a.stats) {
            a.stats->pcg_iters = it;
            a.stats->pcg_relres = relres;
            a.stats->pcg_outer = outer;
            if (a.alive)
                a.stats->alive = (int64_t)*a.alive;
        }
    }
}

__device__ __forceinline__ void scatter_phi(const PcgArgs &a, int gw, int NW, int lane)
{
    for (int s = gw; s < a.n_slices; s += NW) {
        int row = s * 32 + lane;
        if (row < a.n)
            a.phi[a.dof_node[row]] = a.x[row];
    }
}

// ---------------------------------------------------------------------------
// FP64 Jacobi-PCG
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(PCG_BLOCK) k_pcg64(PcgArgs a)
{
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * PCG_WARPS + (threadIdx.x >> 5);
    const int NW = gridDim.x * PCG_WARPS;
    int set = 0;

    // r = f - M x, z = D^-1 r, p_old = 0
    double acc[3] = {0.0, 0.0, 0.0}, tot[3];
    for (int s = gw; s < a.n_slices; s += NW) {
        int row = s * 32 + lane;
        int b = a.slice_ptr[s], width = (a.slice_ptr[s + 1] - b) >> 5;
        double ax = 0.0;
        for (int c = 0; c < width; ++c) {
            int k = b + c * 32 + lane;
            ax += a.val64[k] * a.x[a.col[k]];
        }
        double f = rhs_entry(a, row);
        double r = f - ax;
        double z = a.dinv64[row] * r;
        a.r[row] = r;
        a.z[row] = z;
        a.p0[row] = 0.0;
        acc[0] += r * z;
        acc[1] += r * r;
        acc[2] += f * f;
    }
    if (!grid_sum<3>(acc, a.partials, set, a.st, tot))
        return;
    set ^= 1;
    double rz = tot[0], rr = tot[1], ff = tot[2];
    if (ff == 0.0) {
        for (int s = gw; s < a.n_slices; s += NW)
            a.x[s * 32 + lane] = 0.0;
        scatter_phi(a, gw, NW, lane);
        finish(a, 0, 0.0, 0);
        return;
    }
    const double tol = a.rtol * sqrt(ff);
    int it = 0;
    double beta = 0.0;
    double *pold = a.p0, *pnew = a.p1;
    int status = 0;
    while (sqrt(rr) > tol) {
        if (it >= a.max_iter) {
            status = PIC_ERR_NOT_CONVERGED;
            break;
        }
        // phase A: p = z + beta p_old (on the fly), Ap = M p, p.Ap
        double pap[1] = {0.0}, pt[1];
        for (int s = gw; s < a.n_slices; s += NW) {
            int row = s * 32 + lane;
            int b = a.slice_ptr[s], width = (a.slice_ptr[s + 1] - b) >> 5;
            double ap = 0.0;
            for (int c = 0; c < width; ++c) {
                int k = b + c * 32 + lane;
                int j = a.col[k];
                ap += a.val64[k] * (__ldcg(a.z + j) + beta * __ldcg(pold + j));
            }
            double p = a.z[row] + beta * pold[row];
            pnew[row] = p;
            a.ap[row] = ap;
            pap[0] += p * ap;
        }
        if (!grid_sum<1>(pap, a.partials, set, a.st, pt))
            return;
        set ^= 1;
        double alpha = rz / pt[0];
        // phase B: x += alpha p, r -= alpha Ap, z = D^-1 r
        double acc2[2] = {0.0, 0.0}, t2[2];
        for (int s = gw; s < a.n_slices; s += NW) {
            int row = s * 32 + lane;
            double p = pnew[row];
            a.x[row] = a.x[row] + alpha * p;
            double r = a.r[row] - alpha * a.ap[row];
            double z = a.dinv64[row] * r;
            a.r[row] = r;
            a.z[row] = z;
            acc2[0] += r * z;
            acc2[1] += r * r;
        }
        if (!grid_sum<2>(acc2, a.partials, set, a.st, t2))
            return;
        set ^= 1;
        beta = t2[0] / rz;
        rz = t2[0];
        rr = t2[1];
        ++it;
        double *tmp = pold;
        pold = pnew;
        pnew = tmp;
    }
    scatter_phi(a, gw, NW, lane);
    finish(a, it, sqrt(rr) / sqrt(ff), status);
}

// ---------------------------------------------------------------------------
// FP32 PCG inside FP64 iterative refinement
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(PCG_BLOCK) k_pcg32ir(PcgArgs a)
{
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * PCG_WARPS + (threadIdx.x >> 5);
    const int NW = gridDim.x * PCG_WARPS;
    int set = 0;

    for (int s = gw; s < a.n_slices; s += NW) {
        int row = s * 32 + lane;
        a.f[row] = rhs_entry(a, row);
    }
    // own rows only: no barrier needed before the first residual
    int it = 0, status = 0, outer = 0;
    double ff = -1.0, rr64 = 0.0;
    for (;;) {
        // FP64 residual r = f - M x (x of neighbours complete after the
        // barrier that ended the previous refinement)
        double acc[2] = {0.0, 0.0}, tot[2];
        for (int s = gw; s < a.n_slices; s += NW) {
            int row = s * 32 + lane;
            int b = a.slice_ptr[s], width = (a.slice_ptr[s + 1] - b) >> 5;
            double ax = 0.0;
            for (int c = 0; c < width; ++c) {
                int k = b + c * 32 + lane;
                ax += a.val64[k] * __ldcg(a.x + a.col[k]);
            }
            double f = a.f[row];
            double r = f - ax;
            a.r[row] = r;
            acc[0] += r * r;
            acc[1] += f * f;
        }
        if (!grid_sum<2>(acc, a.partials, set, a.st, tot))
            return;
        set ^= 1;
        rr64 = tot[0];
        if (ff < 0.0)
            ff = tot[1];
        if (ff == 0.0) {
            for (int s = gw; s < a.n_slices; s += NW)
                a.x[s * 32 + lane] = 0.0;
            scatter_phi(a, gw, NW, lane);
            finish(a, 0, 0.0, 0);
            return;
        }
        if (sqrt(rr64) <= a.rtol * sqrt(ff))
            break;
        if (it >= a.max_iter) {
            status = PIC_ERR_NOT_CONVERGED;
            break;
        }
        // inner FP32 PCG on M d = r, d = 0
        double acc2[2] = {0.0, 0.0}, t2[2];
        for (int s = gw; s < a.n_slices; s += NW) {
            int row = s * 32 + lane;
            float r = (float)a.r[row];
            float z = a.dinv32[row] * r;
            a.r32[row] = r;
            a.z32[row] = z;
            a.p32_0[row] = 0.f;
            a.dx32[row] = 0.f;
            acc2[0] += (double)r * (double)z;
            acc2[1] += (double)r * (double)r;
        }
        if (!grid_sum<2>(acc2, a.partials, set, a.st, t2))
            return;
        set ^= 1;
        double rz = t2[0], rr = t2[1];
        const double itol2 = a.inner_rtol * a.inner_rtol * rr;
        double beta = 0.0;
        float *pold = a.p32_0, *pnew = a.p32_1;
        while (rr > itol2 && it < a.max_iter) {
            float b32 = (float)beta;
            double pap[1] = {0.0}, pt[1];
            for (int s = gw; s < a.n_slices; s += NW) {
                int row = s * 32 + lane;
                int b = a.slice_ptr[s], width = (a.slice_ptr[s + 1] - b) >> 5;
                float ap = 0.f;
                for (int c = 0; c < width; ++c) {
                    int k = b + c * 32 + lane;
                    int j = a.col[k];
                    ap += a.val32[k] * (__ldcg(a.z32 + j) + b32 * __ldcg(pold + j));
                }
                float p = a.z32[row] + b32 * pold[row];
                pnew[row] = p;
                a.ap32[row] = ap;
                pap[0] += (double)p * (double)ap;
            }
            if (!grid_sum<1>(pap, a.partials, set, a.st, pt))
                return;
            set ^= 1;
            float alpha = (float)(rz / pt[0]);
            double acc3[2] = {0.0, 0.0}, t3[2];
            for (int s = gw; s < a.n_slices; s += NW) {
                int row = s * 32 + lane;
                float p = pnew[row];
                a.dx32[row] = a.dx32[row] + alpha * p;
                float r = a.r32[row] - alpha * a.ap32[row];
                float z = a.dinv32[row] * r;
                a.r32[row] = r;
                a.z32[row] = z;
                acc3[0] += (double)r * (double)z;
                acc3[1] += (double)r * (double)r;
            }
            if (!grid_sum<2>(acc3, a.partials, set, a.st, t3))
                return;
            set ^= 1;
            beta = t3[0] / rz;
            rz = t3[0];
            rr = t3[1];
            ++it;
            float *tmp = pold;
            pold = pnew;
            pnew = tmp;
        }
        // refinement update in FP64
        for (int s = gw; s < a.n_slices; s += NW) {
            int row = s * 32 + lane;
            a.x[row] = a.x[row] + (double)a.dx32[row];
        }
        if (!grid_sync(a.st))
            return;
        ++outer;
    }
    scatter_phi(a, gw, NW, lane);
    finish(a, it, sqrt(rr64) / sqrt(ff), status, outer);
}

cudaError_t pcg_plan(int n_slices, int num_sms, int precision, PcgLaunch *plan)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, precision == PIC_PREC_FP64 ? (const void *)k_pcg64 : (const void *)k_pcg32ir,
        PCG_BLOCK, 0);
    if (e != cudaSuccess)
        return e;
    if (per_sm < 1)
        return cudaErrorInvalidConfiguration;
    int max_blocks = per_sm * num_sms;
    int want = (n_slices + PCG_WARPS - 1) / PCG_WARPS;  // one slice per warp
    int cap = 2 * num_sms;                              // barrier cost grows with blocks
    plan->grid = want < cap ? (want < 1 ? 1 : want) : cap;
    if (plan->grid > max_blocks)
        plan->grid = max_blocks;
    plan->block = PCG_BLOCK;
    return cudaSuccess;
}

cudaError_t launch_pcg(cudaStream_t s, const PcgLaunch &plan, const PcgArgs &a)
{
    void *args[] = {(void *)&a};
    const void *fn = a.precision == PIC_PREC_FP64 ? (const void *)k_pcg64 : (const void *)k_pcg32ir;
    return cudaLaunchCooperativeKernel(fn, dim3(plan.grid), dim3(plan.block), args, 0, s);
}

}  // namespace pf
