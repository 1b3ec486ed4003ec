// noalloc.cu -- pic_pcg_solve_static: a Jacobi-preconditioned CG solve of a
// caller-supplied sparse SPD system that allocates no device memory.
//
// Who needs it: callers that cannot call cudaMalloc at all -- for example a
// host application that hands this library a fixed device arena it manages
// itself, code running where the allocator is locked or budgeted by someone
// else, or a solver step that must not grow the process's device footprint
// between checkpoints.  Such callers own every input and output buffer; the
// work vectors of the solve live in one file-scope device array below.
//
// The array is a fixed STATIC_MAX_ROWS rows; each GPU that loads the library
// keeps it (about 10 MiB) until the process exits.  Every call on a device
// uses the same array, so calls whose kernels overlap on the GPU (different
// streams, or different host threads) race and must be serialised by the
// caller.  Its contents are whatever the last call left; this entry point
// clears what must start at zero (the grid-barrier counter and the error
// word) at the start of each call.
#include <cstdio>
#include <mutex>

#include "common.cuh"

namespace {

constexpr int STATIC_MAX_ROWS = 1 << 18;  // 262,144 rows
constexpr int NA_BLOCK = 256;
constexpr int NA_WARPS = NA_BLOCK / 32;
constexpr int NA_MAX_BLOCKS = 4096;
constexpr long long NA_SPIN_LIMIT = 1LL << 25;
#define NA_FULL 0xffffffffu

// Layout of the scratch array (in doubles):
//   [0, 5 R)        r, z, p0, p1, ap          (R = STATIC_MAX_ROWS)
//   [5 R, 5 R + 8 B) partials of the grid reductions, 2 sets x B blocks x 4
//   then the control words: barrier count, barrier generation, error word,
//   iterations, relative residual.
constexpr size_t NA_VEC = (size_t)STATIC_MAX_ROWS;
constexpr size_t NA_PART = 2 * (size_t)NA_MAX_BLOCKS * 4;
constexpr size_t NA_CTRL = 8;
constexpr size_t NA_DOUBLES = 5 * NA_VEC + NA_PART + NA_CTRL;

static __device__ __align__(256) double g_static_scratch[NA_DOUBLES];

struct Ctrl {
    unsigned bar_count, bar_gen;
    int err, iters;
    double relres;
};
static_assert(sizeof(Ctrl) <= NA_CTRL * sizeof(double), "control words");

struct NaArgs {
    int n;
    const int *rowptr, *col;
    const double *val, *b;
    double *x;
    double rtol;
    int max_iter;
    double *r, *z, *p0, *p1, *ap, *partials;
    Ctrl *ctrl;
};

__device__ __forceinline__ unsigned na_ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// grid barrier with an iteration limit (cooperative launch keeps all blocks
// resident); false when the wait ran out or another block failed
__device__ bool na_grid_sync(Ctrl *c)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned g = na_ld_acquire(&c->bar_gen);
        __threadfence();
        unsigned arrived = atomicAdd(&c->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&c->bar_count, 0u);
            __threadfence();
            atomicAdd(&c->bar_gen, 1u);
        } else {
            long long spins = 0;
            while (na_ld_acquire(&c->bar_gen) == g) {
                if (++spins > NA_SPIN_LIMIT) {
                    atomicCAS(&c->err, 0, PIC_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        // any error recorded before the barrier (a timed-out wait, or an
        // input check of the first pass) ends the solve in every block
        if (*(volatile int *)&c->err != 0)
            ok = 0;
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

__device__ __forceinline__ double na_warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(NA_FULL, v, o);
    return v;
}

template <int NV>
__device__ bool na_grid_sum(const double (&v)[NV], const NaArgs &a, int set, double (&out)[NV])
{
    __shared__ double red[NA_WARPS][NV];
    __shared__ double res[NV];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s = na_warp_sum(v[k]);
        if (lane == 0)
            red[wid][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < NA_WARPS; ++w)
            s += red[w][threadIdx.x];
        a.partials[((size_t)set * gridDim.x + blockIdx.x) * 4 + threadIdx.x] = s;
    }
    if (!na_grid_sync(a.ctrl))
        return false;
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int b = lane; b < (int)gridDim.x; b += 32)
                s += __ldcg(a.partials + ((size_t)set * gridDim.x + b) * 4 + k);
            s = na_warp_sum(s);
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

// Row i of A times v for the first pass, which also checks the caller's
// pattern: a row whose end precedes its start, or a column outside [0, n),
// records PIC_ERR_ARG and is skipped (nothing outside v is read).  The
// grid barrier after the first pass ends the solve in every block when
// an error was recorded, so the later passes only see checked rows.
__device__ __forceinline__ double na_row_dot_checked(const NaArgs &a, int i, const double *v)
{
    const int k0 = a.rowptr[i], k1 = a.rowptr[i + 1];
    if (k1 < k0 || k0 < 0) {
        atomicCAS(&a.ctrl->err, 0, PIC_ERR_ARG);
        return 0.0;
    }
    double s = 0.0;
    for (int k = k0; k < k1; ++k) {
        const int j = a.col[k];
        if (j < 0 || j >= a.n) {
            atomicCAS(&a.ctrl->err, 0, PIC_ERR_ARG);
            continue;
        }
        s += a.val[k] * v[j];
    }
    return s;
}

__device__ __forceinline__ double na_diag(const NaArgs &a, int i)
{
    for (int k = a.rowptr[i]; k < a.rowptr[i + 1]; ++k)
        if (a.col[k] == i)
            return a.val[k];
    return 0.0;
}

__device__ __forceinline__ bool rowptr_ok(const NaArgs &a, int i)
{
    return a.rowptr[i] >= 0 && a.rowptr[i + 1] >= a.rowptr[i];
}

// Jacobi-PCG on a CSR matrix, thread per row, two grid barriers per
// iteration (the search direction is formed inside the SpMV from z and the
// previous direction, double-buffered).  Same algorithm and stopping rule
// as the solve of poisson_solve: ||b - A x||_2 <= rtol ||b||_2 on the
// recursively updated residual.
__global__ void __launch_bounds__(NA_BLOCK) k_pcg_static(NaArgs a)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nt = gridDim.x * blockDim.x;
    int set = 0;
    double acc[3] = {0.0, 0.0, 0.0}, tot[3];
    for (int i = tid; i < a.n; i += nt) {
        double r = a.b[i] - na_row_dot_checked(a, i, a.x);
        double d = rowptr_ok(a, i) ? na_diag(a, i) : 0.0;
        double z = d != 0.0 ? r / d : 0.0;
        a.r[i] = r;
        a.z[i] = z;
        a.p0[i] = 0.0;
        acc[0] += r * z;
        acc[1] += r * r;
        acc[2] += a.b[i] * a.b[i];
    }
    if (!na_grid_sum<3>(acc, a, set, tot))
        return;
    set ^= 1;
    double rz = tot[0], rr = tot[1], bb = tot[2];
    int it = 0, status = 0;
    // every block holds the same totals, so every block takes the same
    // branch: a non-finite value in b, x or A reaches these sums
    if (!isfinite(bb) || !isfinite(rr) || !isfinite(rz)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            atomicCAS(&a.ctrl->err, 0, PIC_ERR_ARG);
            a.ctrl->iters = 0;
            a.ctrl->relres = rr / bb;
        }
        return;
    }
    if (bb == 0.0) {
        for (int i = tid; i < a.n; i += nt)
            a.x[i] = 0.0;
        rr = 0.0;
        bb = 1.0;
    }
    const double tol = a.rtol * sqrt(bb);
    double beta = 0.0;
    double *pold = a.p0, *pnew = a.p1;
    while (sqrt(rr) > tol) {
        if (it >= a.max_iter) {
            status = PIC_ERR_NOT_CONVERGED;
            break;
        }
        double pap[1] = {0.0}, pt[1];
        for (int i = tid; i < a.n; i += nt) {
            double s = 0.0;
            for (int k = a.rowptr[i]; k < a.rowptr[i + 1]; ++k) {
                int j = a.col[k];
                s += a.val[k] * (__ldcg(a.z + j) + beta * __ldcg(pold + j));
            }
            double p = a.z[i] + beta * pold[i];
            pnew[i] = p;
            a.ap[i] = s;
            pap[0] += p * s;
        }
        if (!na_grid_sum<1>(pap, a, set, pt))
            return;
        set ^= 1;
        // breakdown: A not positive definite along p, or a non-finite value
        // (the same in every block)
        if (!(pt[0] > 0.0) || !isfinite(pt[0])) {
            status = PIC_ERR_NOT_CONVERGED;
            break;
        }
        double alpha = rz / pt[0];
        double acc2[2] = {0.0, 0.0}, t2[2];
        for (int i = tid; i < a.n; i += nt) {
            double p = pnew[i];
            a.x[i] = a.x[i] + alpha * p;
            double r = a.r[i] - alpha * a.ap[i];
            double d = na_diag(a, i);
            double z = d != 0.0 ? r / d : 0.0;
            a.r[i] = r;
            a.z[i] = z;
            acc2[0] += r * z;
            acc2[1] += r * r;
        }
        if (!na_grid_sum<2>(acc2, a, set, t2))
            return;
        set ^= 1;
        if (!isfinite(t2[0]) || !isfinite(t2[1])) {
            status = PIC_ERR_NOT_CONVERGED;
            ++it;
            rr = t2[1];
            break;
        }
        beta = t2[0] / rz;
        rz = t2[0];
        rr = t2[1];
        ++it;
        double *tmp = pold;
        pold = pnew;
        pnew = tmp;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (status)
            atomicCAS(&a.ctrl->err, 0, status);
        a.ctrl->iters = it;
        a.ctrl->relres = sqrt(rr) / sqrt(bb);
    }
}

// Per-device set-up: the device address of the scratch array and the grid
// that keeps every block resident.  Filled on the first call on a device,
// with that device current.
struct DevSetup {
    bool ready = false;
    double *base = nullptr;
    int grid = 0;
};
constexpr int NA_MAX_DEVICES = 64;
DevSetup g_setup[NA_MAX_DEVICES];
std::mutex g_setup_mu;
int na_fail(int code, const char *msg)
{
    char buf[256];
    snprintf(buf, sizeof buf, "pic_pcg_solve_static: %s", msg);
    pf::set_global_error(buf);
    return code;
}

int na_setup(int dev, DevSetup **out)
{
    std::lock_guard<std::mutex> lk(g_setup_mu);
    DevSetup &s = g_setup[dev];
    if (!s.ready) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess)
            return na_fail(PIC_ERR_CUDA, cudaGetErrorString(e));
        int sms = 0, per_sm = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_static, NA_BLOCK, 0);
        if (e != cudaSuccess)
            return na_fail(PIC_ERR_CUDA, cudaGetErrorString(e));
        int grid = sms * (per_sm < 2 ? per_sm : 2);
        if (grid < 1)
            return na_fail(PIC_ERR_CUDA, "kernel cannot be resident");
        s.base = (double *)p;
        s.grid = grid < NA_MAX_BLOCKS ? grid : NA_MAX_BLOCKS;
        s.ready = true;
    }
    *out = &s;
    return PIC_OK;
}

}  // namespace

extern "C" int pic_pcg_solve_static(int32_t n, const int32_t *rowptr, const int32_t *col,
                                    const double *val, const double *b, double *x, double rtol,
                                    int32_t max_iter, int32_t *iters, double *rel_res,
                                    void *stream)
{
    if (n < 1 || n > STATIC_MAX_ROWS)
        return na_fail(PIC_ERR_ARG, "n must be in [1, 262144] (the size of the static scratch)");
    if (!rowptr || !col || !val || !b || !x || !(rtol >= 0) || max_iter < 0)
        return na_fail(PIC_ERR_ARG, "null array or bad tolerance");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES)
        return na_fail(PIC_ERR_CUDA, "no current CUDA device");
    DevSetup *s = nullptr;
    int rc = na_setup(dev, &s);
    if (rc)
        return rc;
    cudaStream_t st = (cudaStream_t)stream;
    NaArgs a;
    a.n = n;
    a.rowptr = rowptr;
    a.col = col;
    a.val = val;
    a.b = b;
    a.x = x;
    a.rtol = rtol;
    a.max_iter = max_iter;
    a.r = s->base;
    a.z = s->base + NA_VEC;
    a.p0 = s->base + 2 * NA_VEC;
    a.p1 = s->base + 3 * NA_VEC;
    a.ap = s->base + 4 * NA_VEC;
    a.partials = s->base + 5 * NA_VEC;
    a.ctrl = (Ctrl *)(s->base + 5 * NA_VEC + NA_PART);
    // the barrier counter and the error word start at zero on every call
    e = cudaMemsetAsync(a.ctrl, 0, sizeof(Ctrl), st);
    if (e != cudaSuccess)
        return na_fail(PIC_ERR_CUDA, cudaGetErrorString(e));
    void *args[] = {(void *)&a};
    e = cudaLaunchCooperativeKernel((const void *)k_pcg_static, dim3(s->grid), dim3(NA_BLOCK),
                                    args, 0, st);
    if (e != cudaSuccess)
        return na_fail(PIC_ERR_CUDA, cudaGetErrorString(e));
    Ctrl h;
    e = cudaMemcpyAsync(&h, a.ctrl, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return na_fail(PIC_ERR_CUDA, cudaGetErrorString(e));
    if (iters)
        *iters = h.iters;
    if (rel_res)
        *rel_res = h.relres;
    if (h.err) {
        const char *why = h.err == PIC_ERR_NOT_CONVERGED
                              ? "not converged (max_iter reached, or CG broke down: p.Ap <= 0 "
                                "or a non-finite value)"
                          : h.err == PIC_ERR_ARG
                              ? "bad input (a column outside [0, n), a decreasing rowptr, or a "
                                "non-finite value in A, b or x)"
                              : "device-side wait timed out";
        return na_fail(h.err, why);
    }
    return PIC_OK;
}
