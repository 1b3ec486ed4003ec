// pcg.cu -- the space-charge Poisson solve M Phi = f (App. B, eq. poisson_mat)
// as one persistent cooperative kernel per solve: preconditioned conjugate
// gradients (Jacobi, a Chebyshev polynomial in D^-1 M with a two-level
// coarse correction, or an aggregation multigrid V-cycle), warm-started from
// the previous potential.
//
// The matrix is stored as sliced ELLPACK with slices of 32 rows (one warp
// per slice, one thread per row, columns of a slice interleaved so each load
// of the warp is coalesced).  Each warp owns the same slices in every phase,
// so a thread only ever reads its own rows' x, r, z, p; neighbours' values
// are gathered through L2.
//
// Two kernel families.  The resident kernels (one system that fits: one
// block per SM, the block's rows in registers, its matrix slices and vector
// segments in shared memory) exchange halo values either after a grid
// barrier or, for the Chebyshev steps of the FP32 solve, through tagged
// words that each block polls for the values it reads; the general kernels
// (batches of systems, systems too large for the resident blocks) keep the
// vectors in global memory and synchronise per group of blocks.  Both have a
// V-cycle of their own: the resident one keeps its two coarse levels in
// shared memory, block by block; the general one walks any number of levels
// whose vectors live in global memory, like the fine level's.
//
// A standard CG iteration takes two grid-wide reductions (p.Ap and r.z).
// Reductions: within the warp, in warp order within the block, then every
// block sums the per-block partials in block order -- a fixed order, so all
// blocks obtain identical scalars and the result is reproducible run to run.
//
// FP32_IR: the inner CG runs in FP32 (matrix values, vectors, SpMV) with
// double-float dot products; the outer loop recomputes the residual f - M x
// in FP64 and applies the correction in FP64 (iterative refinement).
//
// Every wait (grid barrier, tagged word) has an iteration limit: a block
// that waits too long records PIC_ERR_TIMEOUT and the whole kernel returns.
#include <algorithm>
#include <map>
#include <mutex>

#include "common.cuh"

namespace pf {

constexpr int PCG_BLOCK = 256;
constexpr int PCG_WARPS = PCG_BLOCK / 32;
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

// The blocks that solve one system: the whole grid, or (for a batch of
// independent systems) the group of blocks assigned to one of them.
struct Grp {
    unsigned *ctr;   // barrier counter of the group
    int nb, rank;    // blocks in the group, this block's rank in it
    int b0;          // first block of the group
};

__device__ __forceinline__ Grp grp_of(const PcgArgs &a)
{
    if (a.n_groups <= 0)
        return Grp{&a.st->bar_count, (int)gridDim.x, (int)blockIdx.x, 0};
    int g = a.blk_grp[blockIdx.x];
    int b0 = a.grp[4 * g + 2];
    return Grp{a.grp_bar + g, a.grp[4 * g + 3], (int)blockIdx.x - b0, b0};
}

__device__ __forceinline__ void red_release_add_u32(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Barriers this block has passed in the current launch; thread 0 alone reads
// and writes it, and grid_sync_init() clears it at the start of every kernel
// that calls grid_sync().
__device__ __noinline__ unsigned *bar_gen()
{
    __shared__ unsigned gen;
    return &gen;
}

__device__ __forceinline__ void grid_sync_init()
{
    if (threadIdx.x == 0)
        *bar_gen() = 0u;
}

// Barrier over the blocks of one group (all blocks are co-resident: the
// launch is cooperative).  The group's counter is zero at launch and every
// block adds 1 per barrier with a release reduction, so barrier number k
// (counted from 1) is complete once the counter has reached k * nb; thread 0
// spins on it with acquire loads and the block barrier hands the ordering to
// the other threads.  Two dependent trips to L2 per barrier (the reduction
// needs no reply), no fences.  The comparison is taken modulo 2^32, so the
// counter may wrap.  The wait has an iteration limit: a block that waits too
// long records PIC_ERR_TIMEOUT and the whole kernel returns; a block also
// gives up when it sees that error recorded by another block (read once
// before the wait, off the critical path, and every 1024 spins).
// A block sum that crosses a barrier on the way: thread 0 adds the n
// per-warp partials part[] (shared memory, in warp order) and publishes the
// sum to dst before arriving, so the sum needs no barrier of its own.
struct Ride {
    const double *part = nullptr;
    int n = 0;
    double *dst = nullptr;
};

__device__ bool grid_sync(const PcgArgs &a, Ride r1 = Ride(), Ride r2 = Ride(),
                          Ride r3 = Ride())
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        const Ride *rides[3] = {&r1, &r2, &r3};
        for (int k = 0; k < 3; ++k) {
            if (!rides[k]->part)
                continue;
            double v = 0.0;
            for (int i = 0; i < rides[k]->n; ++i)
                v += rides[k]->part[i];
            *rides[k]->dst = v;
        }
        const Grp g = grp_of(a);
        const int err0 = ld_volatile_i32(&a.st->err);
        const unsigned gen = *bar_gen() + 1u;
        *bar_gen() = gen;
        const unsigned target = gen * (unsigned)g.nb;
        red_release_add_u32(g.ctr, 1u);
        int ok = err0 != PIC_ERR_TIMEOUT;
        long long spins = 0;
        while ((int)(ld_acquire_u32(g.ctr) - target) < 0) {
            ++spins;
            if (spins > a.spin_limit ||
                ((spins & 1023) == 0 && ld_volatile_i32(&a.st->err) == PIC_ERR_TIMEOUT)) {
                atomicCAS(&a.st->err, 0, PIC_ERR_TIMEOUT);
                ok = 0;
                break;
            }
        }
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

// one static buffer per kernel for every reduction: 3 x 512 values + 4 results
__device__ __noinline__ double *reduction_buffer()
{
    __shared__ double buf[3 * 512 + 4];
    return buf;
}

struct NoFinish {
    __device__ void operator()(double *) const {}
};

// Sum NV per-thread FP64 values over the whole grid in a fixed order, so that
// every block obtains identical totals.  In the block the values go through
// shared memory and one warp adds them (each lane a strided run, then a
// butterfly): far fewer FP64 operations than a butterfly in every warp, which
// matters on a part whose FP64 rate is low.  The block partials cross the
// grid barrier in global memory (`set` alternates between calls so a fast
// block never overwrites partials a slow block has not read yet).  `fin` runs
// once per block on the totals and may append derived scalars (e.g. the CG
// step lengths) after them, so that divisions are not repeated by every
// thread.  out[0..NV) = totals, out[NV..NO) = what fin wrote.
template <int NV, int NO, int BLOCK, typename F>
__device__ bool grid_sum_f(const double (&v)[NV], int set, const PcgArgs &a, double (&out)[NO],
                           F fin)
{
    static_assert(NV <= 3 && NO <= 4 && BLOCK <= 512, "reduction buffer size");
    double *vals = reduction_buffer();
    double *res = vals + 3 * 512;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        vals[k * BLOCK + threadIdx.x] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int i = lane; i < BLOCK; i += 32)
                s += vals[k * BLOCK + i];
            s = warp_sum(s);
            if (lane == 0)
                a.partials[((size_t)set * gridDim.x + blockIdx.x) * 4 + k] = s;
        }
    }
    if (!grid_sync(a))
        return false;
    if (wid == 0) {
        const Grp g = grp_of(a);
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int b = lane; b < g.nb; b += 32)
                s += __ldcg(a.partials + ((size_t)set * gridDim.x + g.b0 + b) * 4 + k);
            s = warp_sum(s);
            if (lane == 0)
                res[k] = s;
        }
        if (lane == 0)
            fin(res);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NO; ++k)
        out[k] = res[k];
    return true;
}

template <int NV, int BLOCK = PCG_BLOCK>
__device__ bool grid_sum(const double (&v)[NV], int set, const PcgArgs &a, double (&out)[NV])
{
    return grid_sum_f<NV, NV, BLOCK>(v, set, a, out, NoFinish());
}

// Double-float accumulation: the unevaluated sum hi + lo of two floats
// (about 48 significant bits).  A product enters exactly (the fused
// multiply-add gives the rounding error of the float product) and a sum
// through Knuth's two-sum, so the FP32 solver's dot products take no FP64
// instruction per row: on this part the FP64 rate is a small fraction of the
// FP32 rate, and the per-row FP64 products and conversions were a visible
// share of an iteration.  The intrinsics keep the compiler from contracting
// or reordering the error terms.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ void df_add(DF &s, float x)
{
    const float t = __fadd_rn(s.hi, x);
    const float bp = __fsub_rn(t, s.hi);
    const float e = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    s.hi = t;
    s.lo = __fadd_rn(s.lo, e);
}

__device__ __forceinline__ void df_add_prod(DF &s, float a, float b)
{
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);
    df_add(s, p);
    s.lo = __fadd_rn(s.lo, pe);
}

__device__ __forceinline__ void df_add_df(DF &s, const DF &o)
{
    df_add(s, o.hi);
    s.lo = __fadd_rn(s.lo, o.lo);
}

__device__ __forceinline__ double df_value(const DF &s)
{
    return (double)s.hi + (double)s.lo;
}

// butterfly over the warp in double-float; the FP64 value of lane 0's sum
__device__ __forceinline__ double df_warp_sum(DF x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        DF y;
        y.hi = __shfl_xor_sync(FULL_MASK, x.hi, o);
        y.lo = __shfl_xor_sync(FULL_MASK, x.lo, o);
        df_add_df(x, y);
    }
    return df_value(x);
}

// The block reduction of grid_sum_f for double-float per-thread values: a
// butterfly in every warp (FP32 instructions), the warp sums to FP64 in
// shared memory, warp 0 adds them in warp order.  Then the same grid step.
template <int NV, int NO, int BLOCK, typename F>
__device__ bool grid_sum_df(const DF (&v)[NV], int set, const PcgArgs &a, double (&out)[NO],
                            F fin)
{
    constexpr int NWB = BLOCK / 32;
    static_assert(NV <= 3 && NO <= 4 && NWB <= 32, "reduction buffer size");
    double *vals = reduction_buffer();
    double *res = vals + 3 * 512;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const double x = df_warp_sum(v[k]);
        if (lane == 0)
            vals[k * NWB + wid] = x;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = lane < NWB ? vals[k * NWB + lane] : 0.0;
            s = warp_sum(s);
            if (lane == 0)
                a.partials[((size_t)set * gridDim.x + blockIdx.x) * 4 + k] = s;
        }
    }
    if (!grid_sync(a))
        return false;
    if (wid == 0) {
        const Grp g = grp_of(a);
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int b = lane; b < g.nb; b += 32)
                s += __ldcg(a.partials + ((size_t)set * gridDim.x + g.b0 + b) * 4 + k);
            s = warp_sum(s);
            if (lane == 0)
                res[k] = s;
        }
        if (lane == 0)
            fin(res);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NO; ++k)
        out[k] = res[k];
    return true;
}

// The FP32 inner solve of a refinement works on r / sc with sc the power of
// two nearest below ||r||_2: whatever the scale of the system (adjoint right
// sides included) its values and dot products stay far inside the FP32
// range, and since power-of-two scaling is exact and every step of the inner
// solve is homogeneous, the result is the unscaled one bit for bit wherever
// that did not overflow or underflow.  0 when ||r|| is not finite.
__device__ __forceinline__ double refinement_scale(double rr)
{
    const double nr = sqrt(rr);
    if (!(nr > 0.0) || !(nr < 1.0e300))
        return 0.0;
    return scalbn(1.0, ilogb(nr));
}

// f_i = ((q w_sp / eps0) W_i 2^-S + f_Neumann,i) + f_D,i (eq. poisson_rhs plus
// the load of the prescribed Dirichlet values), written without contraction
// so it equals the plain evaluation bit for bit; 0 on padding rows (no node)
__device__ __forceinline__ double rhs_entry(const PcgArgs &a, int row)
{
    if (a.rhs)
        return a.rhs[row];
    int node = a.dof_node[row];
    if (node < 0)
        return 0.0;
    double w = (double)(long long)a.W[node];
    return __dadd_rn(__dadd_rn(__dmul_rn(a.coef, __dmul_rn(w, a.wscale)), a.fN[row]), a.fD[row]);
}

// Statistics of the solve: the first block of each group reports; with
// several groups (a batch) the step reports the largest iteration count and
// residual among them.
__device__ __forceinline__ void finish(const PcgArgs &a, int it, double relres, int status,
                                       int outer = 0)
{
    if (threadIdx.x == 0 && grp_of(a).rank == 0) {
        if (status)
            atomicCAS(&a.st->err, 0, status);
        if (a.grp_iters && a.n_groups > 0)
            a.grp_iters[a.blk_grp[blockIdx.x]] = it;
        if (a.stats) {
            atomicMax(&a.stats->pcg_iters, it);
            atomicMax((unsigned long long *)&a.stats->pcg_relres,
                      (unsigned long long)__double_as_longlong(relres));
            atomicMax(&a.stats->pcg_outer, outer);
            if (a.alive)
                a.stats->alive = (int64_t)*a.alive;
        }
    }
}

// The slices a warp works on in the general kernels: the group's slice range
// strided by the group's warps (the whole matrix when there are no groups).
struct Span {
    int s0, s1, gw, nw;
    int g;   // the group (0 without groups)
};

__device__ __forceinline__ Span row_span(const PcgArgs &a)
{
    const int w = threadIdx.x >> 5;
    if (a.n_groups <= 0)
        return Span{0, a.n_slices, (int)blockIdx.x * PCG_WARPS + w, (int)gridDim.x * PCG_WARPS, 0};
    int g = a.blk_grp[blockIdx.x];
    const int *d = a.grp + 4 * g;
    return Span{d[0], d[1], ((int)blockIdx.x - d[2]) * PCG_WARPS + w, d[3] * PCG_WARPS, g};
}
#define FOR_SLICES(sp, s) for (int s = (sp).s0 + (sp).gw; s < (sp).s1; s += (sp).nw)

// Coarse correction of the general kernels: the group's slices in
// aggregates of AGG_SLICES consecutive slices (R0 sums an aggregate's rows),
// A0 = R0 M R0^T of the group inverted on the host.  Stage 1 (after the first
// barrier): each aggregate's residual from its slices' sums, in slice order;
// stage 2 (after the second): z0 = A0^-1 r0 for each aggregate; the slices add
// z0 after the third.  Each aggregate is owned by one warp of the group.
constexpr int AGG_SLICES = PCG_AGG_SLICES;

__device__ void coarse_stage(const PcgArgs &a, const Span &sp, int lane, int stage)
{
    const int base = a.agg_off[sp.g];
    const int n_agg = a.agg_off[sp.g + 1] - base;
    for (int ag = sp.gw; ag < n_agg; ag += sp.nw) {
        double v = 0.0;
        if (stage == 1) {
            const int s = sp.s0 + ag * AGG_SLICES + lane;
            if (lane < AGG_SLICES && s < sp.s1)
                v = __ldcg(a.slice_r + s);
        } else {
            const float *row = a.agg_inv + a.inv_off[sp.g] + (size_t)ag * n_agg;
            for (int b = lane; b < n_agg; b += 32)
                v += (double)row[b] * __ldcg(a.agg_r + base + b);
        }
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0)
            (stage == 1 ? a.agg_r : a.agg_z)[base + ag] = v;
    }
}

__device__ __forceinline__ void scatter_phi(const PcgArgs &a, const Span &sp, int lane)
{
    FOR_SLICES(sp, s)
    {
        int row = s * 32 + lane;
        int node = a.dof_node[row];
        if (node >= 0)
            a.phi[node] = a.x[row];
    }
}

// ---------------------------------------------------------------------------
// General kernels: any problem size, vectors in global memory, warps strided
// over their group's slices; used for a batch of replicas (one group each)
// and for systems too large for the resident kernels.
// ---------------------------------------------------------------------------

// Row `lane` of a 32-row slice times a vector: sum_c val[k_c] * X(col[k_c]),
// accumulated in column order.  Eight columns' loads are issued before their
// products so each warp keeps many loads in flight (the kernels are bound by
// memory latency).  When the matrix is much larger than L2 it is streamed once
// per product, and its loads are marked evict-first (__ldcs) so that the
// vectors, which the gathers re-read, stay in L2; a matrix that fits is read
// through the read-only path and stays in L2 across products.
template <bool STREAM, typename T>
__device__ __forceinline__ T ld_mat(const T *p)
{
    if constexpr (STREAM)
        return __ldcs(p);
    else
        return __ldg(p);
}

template <typename ACC, bool STREAM, typename V, typename LoadX>
__device__ __forceinline__ ACC sell_row_u(const V *__restrict__ val, const int *__restrict__ col,
                                          int b, int width, int lane, LoadX X)
{
    constexpr int U = 8;
    ACC sum = 0;
    int c = 0;
    for (; c + U <= width; c += U) {
        const int k = b + c * 32 + lane;
        V v[U];
        int j[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            v[u] = ld_mat<STREAM>(val + k + 32 * u);
            j[u] = ld_mat<STREAM>(col + k + 32 * u);
        }
        ACC x[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            x[u] = X(j[u]);
#pragma unroll
        for (int u = 0; u < U; ++u)
            sum += (ACC)v[u] * x[u];
    }
    for (; c < width; ++c) {
        const int k = b + c * 32 + lane;
        sum += (ACC)ld_mat<STREAM>(val + k) * X(ld_mat<STREAM>(col + k));
    }
    return sum;
}

template <typename ACC, typename V, typename LoadX>
__device__ __forceinline__ ACC sell_row(const PcgArgs &a, const V *__restrict__ val, int b,
                                        int width, int lane, LoadX X)
{
    return a.stream_matrix ? sell_row_u<ACC, true>(val, a.col, b, width, lane, X)
                           : sell_row_u<ACC, false>(val, a.col, b, width, lane, X);
}

// ---------------------------------------------------------------------------
// Multigrid V-cycle of the general kernels (z = B r, B symmetric positive
// definite).  Levels 0 (the fine matrix) .. L (coarsest) in GmgLevel records
// in device memory, every level's vectors in global memory; the warps of a
// system stride over that system's slices of each level exactly as over the
// fine slices, so a warp owns the same rows of a level throughout and reads
// other warps' values only after a barrier of the system.  On each level
// above the coarsest: Chebyshev smoothing of D^-1 A_l from zero (the
// residual rc kept by recurrence), the residual after it, restriction by
// sums over the aggregates; on the coarsest, x = A_L^-1 b per system (dense
// inverse); on the way up, x_l += P x_l+1 with the residual rc - A_l P x_l+1
// (the product gathers x_l+1 through the aggregate map, so the prolonged
// vector is never stored) and the same Chebyshev steps from there.  Pre- and
// post-smoothing use the same polynomial, so B is symmetric; P^T A P
// Galerkin coarse matrices and the exact coarsest solve keep it definite.
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ const T *gl_val(const GmgLevel &L);
template <> __device__ __forceinline__ const float *gl_val<float>(const GmgLevel &L) { return L.val32; }
template <> __device__ __forceinline__ const double *gl_val<double>(const GmgLevel &L) { return L.val64; }
template <typename T> __device__ __forceinline__ const T *gl_dinv(const GmgLevel &L);
template <> __device__ __forceinline__ const float *gl_dinv<float>(const GmgLevel &L) { return L.dinv32; }
template <> __device__ __forceinline__ const double *gl_dinv<double>(const GmgLevel &L) { return L.dinv64; }
template <typename T> __device__ __forceinline__ T gl_c1(const GmgLevel &L, int j);
template <> __device__ __forceinline__ float gl_c1<float>(const GmgLevel &L, int j) { return L.c1f[j]; }
template <> __device__ __forceinline__ double gl_c1<double>(const GmgLevel &L, int j) { return L.c1[j]; }
template <typename T> __device__ __forceinline__ T gl_c2(const GmgLevel &L, int j);
template <> __device__ __forceinline__ float gl_c2<float>(const GmgLevel &L, int j) { return L.c2f[j]; }
template <> __device__ __forceinline__ double gl_c2<double>(const GmgLevel &L, int j) { return L.c2[j]; }
template <typename T> __device__ __forceinline__ T gl_ith(const GmgLevel &L);
template <> __device__ __forceinline__ float gl_ith<float>(const GmgLevel &L) { return L.inv_thetaf; }
template <> __device__ __forceinline__ double gl_ith<double>(const GmgLevel &L) { return L.inv_theta; }

// this warp's slices of level L (its system's slices, strided by the system's warps)
#define FOR_LEVEL_SLICES(L, sp, s)                                                          \
    for (int s = (L).gsl[(sp).g] + (sp).gw, s##_end = (L).gsl[(sp).g + 1]; s < s##_end;      \
         s += (sp).nw)

// row `lane` of slice s of level L times the vector X
template <typename T, typename X>
__device__ __forceinline__ T gl_row(const GmgLevel &L, bool stream, int s, int lane, X x)
{
    const int b = L.sptr[s], width = (L.sptr[s + 1] - b) >> 5;
    return stream ? sell_row_u<T, true>(gl_val<T>(L), L.col, b, width, lane, x)
                  : sell_row_u<T, false>(gl_val<T>(L), L.col, b, width, lane, x);
}

// first Chebyshev step from zero: d_0 = D^-1 b / theta, x = d_0, rc = b
template <typename T, typename B>
__device__ __forceinline__ void gmg_start(const GmgLevel &L, const Span &sp, int lane, B bfun)
{
    const T *dinv = gl_dinv<T>(L);
    T *x = (T *)L.x, *rc = (T *)L.rc, *d1 = (T *)L.d[1];
    const T ith = gl_ith<T>(L);
    FOR_LEVEL_SLICES(L, sp, s)
    {
        const int row = 32 * s + lane;
        const T b = bfun(row);
        const T d = dinv[row] * b * ith;
        x[row] = d;
        rc[row] = b;
        d1[row] = d;
    }
}

// Chebyshev steps 1 .. deg-1 (d_j in d[(j+1)&1], each after a barrier that
// completes d_j-1); with final_res one more barrier and rc -= A d_deg-1, the
// residual of x
template <typename T>
__device__ bool gmg_steps(const PcgArgs &a, const GmgLevel &L, bool stream, int deg,
                          const Span &sp, int lane, bool final_res)
{
    const T *dinv = gl_dinv<T>(L);
    T *x = (T *)L.x, *rc = (T *)L.rc;
    for (int j = 1; j < deg; ++j) {
        const T *cur = (const T *)L.d[j & 1];
        T *nxt = (T *)L.d[(j + 1) & 1];
        const T c1 = gl_c1<T>(L, j - 1), c2 = gl_c2<T>(L, j - 1);
        if (!grid_sync(a))
            return false;
        FOR_LEVEL_SLICES(L, sp, s)
        {
            const int row = 32 * s + lane;
            const T ad = gl_row<T>(L, stream, s, lane, [cur](int c) { return __ldcg(cur + c); });
            const T r = rc[row] - ad;
            const T d = c1 * cur[row] + c2 * (dinv[row] * r);
            x[row] = x[row] + d;
            rc[row] = r;
            if (j + 1 < deg || final_res)
                nxt[row] = d;
        }
    }
    if (final_res) {
        const T *cur = (const T *)L.d[deg & 1];
        if (!grid_sync(a))
            return false;
        FOR_LEVEL_SLICES(L, sp, s)
        {
            const int row = 32 * s + lane;
            rc[row] = rc[row] - gl_row<T>(L, stream, s, lane, [cur](int c) { return __ldcg(cur + c); });
        }
    }
    return true;
}

template <typename T> __device__ __forceinline__ T warp_sum_t(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

// coarsest level C below F: b = R rc_F, then x = A_C^-1 b, one warp per row
// of the system's dense inverse
template <typename T>
__device__ bool gmg_coarsest(const PcgArgs &a, const GmgLevel &C, const GmgLevel &F,
                             const Span &sp, int lane)
{
    T *b = (T *)C.rc, *x = (T *)C.x;
    const T *rcf = (const T *)F.rc;
    if (!grid_sync(a))
        return false;
    FOR_LEVEL_SLICES(C, sp, s)
    {
        const int row = 32 * s + lane;
        T v = 0;
        for (int m = C.mptr[row]; m < C.mptr[row + 1]; ++m)
            v += __ldcg(rcf + C.midx[m]);
        b[row] = v;
    }
    if (!grid_sync(a))
        return false;
    const int n = a.gmg_cn[sp.g], r0 = 32 * C.gsl[sp.g];
    const float *inv = a.gmg_inv + a.gmg_ioff[sp.g];
    for (int q = sp.gw; q < n; q += sp.nw) {
        const float *row = inv + (size_t)q * n;
        T v = 0;
        for (int c = lane; c < n; c += 32)
            v += (T)__ldg(row + c) * __ldcg(b + r0 + c);
        v = warp_sum_t(v);
        if (lane == 0)
            x[r0 + q] = v;
    }
    return grid_sync(a);
}

// level L on the way up from the coarser level C: x += P x_C, rc -= A P x_C,
// then the smoothing steps from there; a barrier at the end when a finer
// level reads x next
template <typename T>
__device__ bool gmg_up(const PcgArgs &a, const GmgLevel &L, const GmgLevel &C, bool stream,
                       int deg, const Span &sp, int lane, bool barrier)
{
    const T *dinv = gl_dinv<T>(L);
    T *x = (T *)L.x, *rc = (T *)L.rc, *d1 = (T *)L.d[1];
    const T *xc = (const T *)C.x;
    const int *agg = C.agg;
    const T ith = gl_ith<T>(L);
    FOR_LEVEL_SLICES(L, sp, s)
    {
        const int row = 32 * s + lane;
        const T ae = gl_row<T>(L, stream, s, lane, [xc, agg](int c) {
            const int q = __ldg(agg + c);
            return q >= 0 ? __ldcg(xc + q) : T(0);
        });
        const int q = __ldg(agg + row);
        const T e = q >= 0 ? __ldcg(xc + q) : T(0);
        const T r = rc[row] - ae;
        const T d = dinv[row] * r * ith;
        x[row] = (x[row] + e) + d;
        rc[row] = r;
        d1[row] = d;
    }
    if (!gmg_steps<T>(a, L, stream, deg, sp, lane, false))
        return false;
    return barrier ? grid_sync(a) : true;
}

// z = B r: b0 = r on the fine rows, the result in the fine level's x; the
// caller reads z of other rows only after its next barrier
template <typename T>
__device__ bool gmg_vcycle(const PcgArgs &a, const Span &sp, int lane, const T *b0)
{
    const int nl = a.gmg_nlev;
    for (int l = 0; l < nl; ++l) {
        const GmgLevel &L = a.gmg[l];
        const int deg = l == 0 ? a.gmg_deg0 : a.gmg_deg1;
        if (l == 0) {
            gmg_start<T>(L, sp, lane, [b0](int row) { return b0[row]; });
        } else {
            if (!grid_sync(a))
                return false;
            const T *rcf = (const T *)a.gmg[l - 1].rc;
            const int *mp = L.mptr, *mi = L.midx;
            gmg_start<T>(L, sp, lane, [rcf, mp, mi](int row) {
                T v = 0;
                for (int m = mp[row]; m < mp[row + 1]; ++m)
                    v += __ldcg(rcf + mi[m]);
                return v;
            });
        }
        if (!gmg_steps<T>(a, L, l == 0 && a.stream_matrix, deg, sp, lane, true))
            return false;
    }
    if (!gmg_coarsest<T>(a, a.gmg[nl], a.gmg[nl - 1], sp, lane))
        return false;
    for (int l = nl - 1; l >= 0; --l)
        if (!gmg_up<T>(a, a.gmg[l], a.gmg[l + 1], l == 0 && a.stream_matrix,
                       l == 0 ? a.gmg_deg0 : a.gmg_deg1, sp, lane, l > 0))
            return false;
    return true;
}

// FP64 PCG (the plain FP64 form): Jacobi, or the multigrid V-cycle where the
// hierarchy is in use (z = B r after the update of r; the same reductions)
__global__ void __launch_bounds__(PCG_BLOCK, 4) k_pcg64(PcgArgs a)
{
    grid_sync_init();
    const int lane = threadIdx.x & 31;
    const Span sp = row_span(a);
    const bool mg = a.gmg_nlev > 0;
    int set = 0;

    // r = f - M x, z = B r, p_old = 0
    double acc[3] = {0.0, 0.0, 0.0}, tot[3];
    FOR_SLICES(sp, s)
    {
        int row = s * 32 + lane;
        int b = a.slice_ptr[s], width = (a.slice_ptr[s + 1] - b) >> 5;
        const double *xv = a.x;
        double ax = sell_row<double>(a, a.val64, b, width, lane,
                                     [xv](int j) { return __ldcg(xv + j); });
        double f = rhs_entry(a, row);
        double r = f - ax;
        a.r[row] = r;
        if (!mg) {
            double z = a.dinv64[row] * r;
            a.z[row] = z;
            acc[0] += r * z;
        }
        a.p0[row] = 0.0;
        acc[1] += r * r;
        acc[2] += f * f;
    }
    if (mg) {
        if (!gmg_vcycle<double>(a, sp, lane, a.r))
            return;
        FOR_SLICES(sp, s)
        {
            int row = s * 32 + lane;
            acc[0] += a.r[row] * a.z[row];
        }
    }
    if (!grid_sum<3>(acc, set, a, tot))
        return;
    set ^= 1;
    double rz = tot[0], rr = tot[1], ff = tot[2];
    if (ff == 0.0) {
        FOR_SLICES(sp, s) a.x[s * 32 + lane] = 0.0;
        scatter_phi(a, sp, lane);
        finish(a, 0, 0.0, 0);
        return;
    }
    const double tol2 = a.rtol * a.rtol * ff;
    int it = 0;
    double beta = 0.0;
    double *pold = a.p0, *pnew = a.p1;
    int status = 0;
    while (rr > tol2) {
        if (it >= a.max_iter) {
            status = PIC_ERR_NOT_CONVERGED;
            break;
        }
        // phase A: p = z + beta p_old (on the fly), Ap = M p, p.Ap
        double pap[1] = {0.0}, pt2[2];
        FOR_SLICES(sp, s)
        {
            int row = s * 32 + lane;
            int b = a.slice_ptr[s], width = (a.slice_ptr[s + 1] - b) >> 5;
            const double *zv = a.z, *pv = pold;
            double ap = sell_row<double>(a, a.val64, b, width, lane, [zv, pv, beta](int j) {
                return __ldcg(zv + j) + beta * __ldcg(pv + j);
            });
            double p = a.z[row] + beta * pold[row];
            pnew[row] = p;
            a.ap[row] = ap;
            pap[0] += p * ap;
        }
        if (!grid_sum_f<1, 2, PCG_BLOCK>(pap, set, a, pt2, [rz](double *q) { q[1] = rz / q[0]; }))
            return;
        set ^= 1;
        double alpha = pt2[1];
        // phase B: x += alpha p, r -= alpha Ap, z = B r
        double acc2[2] = {0.0, 0.0}, t3[3];
        FOR_SLICES(sp, s)
        {
            int row = s * 32 + lane;
            double p = pnew[row];
            a.x[row] = a.x[row] + alpha * p;
            double r = a.r[row] - alpha * a.ap[row];
            a.r[row] = r;
            if (!mg) {
                double z = a.dinv64[row] * r;
                a.z[row] = z;
                acc2[0] += r * z;
            }
            acc2[1] += r * r;
        }
        if (mg) {
            if (!gmg_vcycle<double>(a, sp, lane, a.r))
                return;
            FOR_SLICES(sp, s)
            {
                int row = s * 32 + lane;
                acc2[0] += a.r[row] * a.z[row];
            }
        }
        if (!grid_sum_f<2, 3, PCG_BLOCK>(acc2, set, a, t3, [rz](double *q) { q[2] = q[0] / rz; }))
            return;
        set ^= 1;
        beta = t3[2];
        rz = t3[0];
        rr = t3[1];
        ++it;
        double *tmp = pold;
        pold = pnew;
        pnew = tmp;
    }
    scatter_phi(a, sp, lane);
    finish(a, it, sqrt(rr / ff), status);
}

// z = M^-1 r on the rows of this warp, FP32, vectors in global memory:
// Jacobi, or the Chebyshev polynomial of degree k in D^-1 M (see
// apply_precond below); rc lives in ap32 and the step direction d in the
// double-buffered d32_0 / d32_1, which also serve as the halo copies.
__device__ bool precond_global(const PcgArgs &a, const Span &sp, int lane)
{
    if (a.cheb_degree < 2) {
        FOR_SLICES(sp, s)
        {
            int row = s * 32 + lane;
            a.z32[row] = a.dinv32[row] * a.r32[row];
        }
        return true;
    }
    const int kdeg = a.cheb_degree;
    // coarse correction over aggregates of AGG_SLICES slices of the group (see
    // coarse_stage); its three steps ride on the polynomial's first three grid
    // barriers, so it needs degree >= 4
    const bool coarse = a.agg_inv != nullptr && kdeg >= 4;
    FOR_SLICES(sp, s)
    {
        int row = s * 32 + lane;
        float rc = a.r32[row];
        float d = a.dinv32[row] * rc * a.cheb_inv_thetaf;
        a.z32[row] = d;
        a.ap32[row] = rc;
        a.d32_1[row] = d;
        if (coarse) {
            double v = a.dinv32[row] != 0.f ? (double)rc : 0.0;
            for (int o = 16; o > 0; o >>= 1)
                v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0)
                a.slice_r[s] = v;
        }
    }
    for (int j = 1; j < kdeg; ++j) {
        const float *cur = (j & 1) ? a.d32_1 : a.d32_0;
        float *nxt = (j & 1) ? a.d32_0 : a.d32_1;
        const float c1 = a.cheb_c1f[j - 1], c2 = a.cheb_c2f[j - 1];
        if (!grid_sync(a))
            return false;
        if (coarse && j <= 2)
            coarse_stage(a, sp, lane, j);
        FOR_SLICES(sp, s)
        {
            int row = s * 32 + lane;
            int b = a.slice_ptr[s], width = (a.slice_ptr[s + 1] - b) >> 5;
            float ad = sell_row<float>(a, a.val32, b, width, lane,
                                       [cur](int j) { return __ldcg(cur + j); });
            float rc = a.ap32[row] - ad;
            float d = c1 * cur[row] + c2 * (a.dinv32[row] * rc);
            a.z32[row] = a.z32[row] + d;
            a.ap32[row] = rc;
            if (j + 1 < kdeg)
                nxt[row] = d;
        }
    }
    if (coarse) {   // after the third barrier every aggregate's correction is ready
        const int base = a.agg_off[sp.g];
        FOR_SLICES(sp, s)
        {
            int row = s * 32 + lane;
            if (a.dinv32[row] != 0.f)
                a.z32[row] = a.z32[row] + (float)__ldcg(a.agg_z + base + (s - sp.s0) / AGG_SLICES);
        }
    }
    return true;
}

// the general FP32 solver's preconditioner: the V-cycle where the hierarchy
// is in use, else the polynomial (with its coarse correction) or Jacobi
__device__ __forceinline__ bool precond_general(const PcgArgs &a, const Span &sp, int lane)
{
    if (a.gmg_nlev > 0)
        return gmg_vcycle<float>(a, sp, lane, a.r32);
    return precond_global(a, sp, lane);
}

// FP32 PCG inside FP64 iterative refinement (see the resident form below)
__global__ void __launch_bounds__(PCG_BLOCK, 4) k_pcg32ir(PcgArgs a)
{
    grid_sync_init();
    const int lane = threadIdx.x & 31;
    const Span sp = row_span(a);
    int set = 0;

    FOR_SLICES(sp, s)
    {
        int row = s * 32 + lane;
        a.f[row] = rhs_entry(a, row);
    }
    int it = 0, status = 0, outer = 0;
    double ff = -1.0, rr64 = 0.0;
    for (;;) {
        // FP64 residual r = f - M x (x of the other blocks complete after the
        // barrier that ended the previous refinement)
        double acc[2] = {0.0, 0.0}, tot[2];
        FOR_SLICES(sp, s)
        {
            int row = s * 32 + lane;
            int b = a.slice_ptr[s], width = (a.slice_ptr[s + 1] - b) >> 5;
            const double *xv = a.x;
            double ax = sell_row<double>(a, a.val64, b, width, lane,
                                         [xv](int j) { return __ldcg(xv + j); });
            double f = a.f[row];
            double r = f - ax;
            a.r[row] = r;
            acc[0] += r * r;
            acc[1] += f * f;
        }
        if (!grid_sum<2>(acc, set, a, tot))
            return;
        set ^= 1;
        rr64 = tot[0];
        if (ff < 0.0)
            ff = tot[1];
        if (ff == 0.0) {
            FOR_SLICES(sp, s) a.x[s * 32 + lane] = 0.0;
            rr64 = 0.0;
            ff = 1.0;
            break;
        }
        if (rr64 <= a.rtol * a.rtol * ff)
            break;
        if (it >= a.max_iter) {
            status = PIC_ERR_NOT_CONVERGED;
            break;
        }
        double itol = 0.5 * a.rtol * sqrt(ff / rr64);
        if (itol < a.inner_rtol)
            itol = a.inner_rtol;
        const double sc = refinement_scale(rr64), inv_sc = 1.0 / sc;
        if (sc == 0.0) {
            status = PIC_ERR_NOT_CONVERGED;
            break;
        }
        // inner FP32 PCG on M d = r / sc, d = 0
        FOR_SLICES(sp, s)
        {
            int row = s * 32 + lane;
            a.r32[row] = (float)(a.r[row] * inv_sc);
            a.dx32[row] = 0.f;
            a.p32_0[row] = 0.f;
        }
        const int it0 = it;
        if (!precond_general(a, sp, lane))
            return;
        DF acc2[2] = {{0.f, 0.f}, {0.f, 0.f}};
        double t2[2];
        FOR_SLICES(sp, s)
        {
            int row = s * 32 + lane;
            float r = a.r32[row], z = a.z32[row];
            df_add_prod(acc2[0], r, z);
            df_add_prod(acc2[1], r, r);
            a.p32_1[row] = 0.f;
        }
        if (!grid_sum_df<2, 2, PCG_BLOCK>(acc2, set, a, t2, NoFinish()))
            return;
        set ^= 1;
        double rz = t2[0], rr = t2[1];
        const double itol2 = itol * itol * rr;
        // p and A p on own rows only: A p = A z + beta A p_old (the product
        // of z alone; p is never gathered).  A p lives in p32_1 (ap32 is the
        // preconditioner's scratch)
        double beta = 0.0;
        float *pv = a.p32_0, *apv = a.p32_1;
        for (int i = 0; rr > itol2 && rr > 0.0 && it < a.max_iter &&
                        !(a.inner_max > 0 && i >= a.inner_max);
             ++i) {
            float b32 = (float)beta;
            DF pap[1] = {{0.f, 0.f}};
            double pt2[2];
            FOR_SLICES(sp, s)
            {
                int row = s * 32 + lane;
                int b = a.slice_ptr[s], width = (a.slice_ptr[s + 1] - b) >> 5;
                const float *zv = a.z32;
                float az = sell_row<float>(a, a.val32, b, width, lane,
                                           [zv](int j) { return __ldcg(zv + j); });
                float p = a.z32[row] + b32 * pv[row];
                float ap = az + b32 * apv[row];
                pv[row] = p;
                apv[row] = ap;
                df_add_prod(pap[0], p, ap);
            }
            if (!grid_sum_df<1, 2, PCG_BLOCK>(pap, set, a, pt2,
                                              [rz](double *q) { q[1] = rz / q[0]; }))
                return;
            set ^= 1;
            float alpha = (float)pt2[1];
            FOR_SLICES(sp, s)
            {
                int row = s * 32 + lane;
                a.dx32[row] = a.dx32[row] + alpha * pv[row];
                a.r32[row] = a.r32[row] - alpha * apv[row];
            }
            if (!precond_general(a, sp, lane))
                return;
            DF acc3[2] = {{0.f, 0.f}, {0.f, 0.f}};
            double t3[3];
            FOR_SLICES(sp, s)
            {
                int row = s * 32 + lane;
                float r = a.r32[row], z = a.z32[row];
                df_add_prod(acc3[0], r, z);
                df_add_prod(acc3[1], r, r);
            }
            if (!grid_sum_df<2, 3, PCG_BLOCK>(acc3, set, a, t3,
                                              [rz](double *q) { q[2] = q[0] / rz; }))
                return;
            set ^= 1;
            beta = t3[2];
            rz = t3[0];
            rr = t3[1];
            ++it;
        }
        if (it == it0) {   // no inner iteration: no progress possible
            status = PIC_ERR_NOT_CONVERGED;
            break;
        }
        // refinement update in FP64
        FOR_SLICES(sp, s)
        {
            int row = s * 32 + lane;
            a.x[row] = a.x[row] + sc * (double)a.dx32[row];
        }
        if (!grid_sync(a))
            return;
        ++outer;
    }
    scatter_phi(a, sp, lane);
    finish(a, it, sqrt(rr64 / ff), status, outer);
}

// ===========================================================================
// Resident kernels.  Each block owns a contiguous range of slices (rows in
// Morton order: a compact piece of the mesh) and keeps its rows' vectors in
// registers for the whole solve.  The vectors the SpMV reads live in shared
// memory as [own rows | halo], where the halo is the sorted list of columns
// owned by other blocks that the block's rows reference; the block's stored
// column indices are rewritten to these local positions on the host.  Each
// SpMV phase first copies the halo values from global memory (independent
// loads, all in flight together) and then reads shared memory only.  When
// the block's matrix slices fit, they are copied into shared memory once per
// solve as well.
// ===========================================================================
constexpr int RB = 512;         // threads per resident block
constexpr int RW = RB / 32;     // warps per resident block

struct Seg {
    int s0, s1, row0, nrows;
    int e0;                     // first stored entry of the block's slices
    int h0, nh;                 // the block's halo in halo_idx
};

__device__ __forceinline__ Seg block_seg(const PcgArgs &a)
{
    long long G = gridDim.x, b = blockIdx.x;
    Seg g;
    g.s0 = (int)((b * a.n_slices) / G);
    g.s1 = (int)(((b + 1) * a.n_slices) / G);
    g.row0 = g.s0 * 32;
    g.nrows = (g.s1 - g.s0) * 32;
    g.e0 = a.slice_ptr[g.s0];
    g.h0 = a.halo_ptr[b];
    g.nh = a.halo_ptr[b + 1] - g.h0;
    return g;
}

// copy the block's stored entries [e0, e1) into shared memory
template <typename T>
__device__ __forceinline__ void stage_chunk(T *dst, const T *src, int e0, int e1)
{
    const int4 *s = reinterpret_cast<const int4 *>(src + e0);
    int4 *d = reinterpret_cast<int4 *>(dst);
    int n16 = (int)(((long long)(e1 - e0) * sizeof(T)) / 16);
    for (int i = threadIdx.x; i < n16; i += blockDim.x)
        d[i] = __ldg(s + i);
}

// halo values of a vector published in global memory by the other blocks
template <typename V>
__device__ __forceinline__ void stage_halo(V *s, const V *glob, const PcgArgs &a, const Seg &g)
{
    for (int i = threadIdx.x; i < g.nh; i += blockDim.x)
        s[g.nrows + i] = __ldcg(glob + a.halo_idx[g.h0 + i]);
}

// per-thread row slots; pub and epoch make the tags of the neighbour
// exchange (every thread of every block runs the same sequence of exchanges,
// so its own count is the block's and the grid's)
template <int RPT> struct Rows {
    int row[RPT], o[RPT], le[RPT], ge[RPT], wd[RPT];
    bool ok[RPT];
    mutable unsigned pub;   // tagged exchanges so far in this launch
    mutable unsigned pub1;  // tagged exchanges of the multigrid level 1 so far
    unsigned epoch;         // this launch's epoch, < 255
};

template <int RPT, bool SM>
__device__ __forceinline__ void init_rows(Rows<RPT> &t, const PcgArgs &a, const Seg &g)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    t.pub = 0u;
    t.pub1 = 0u;
    t.epoch = a.epoch ? (unsigned)ld_volatile_i32((const int *)a.epoch) : 0u;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        int s = g.s0 + w + k * RW;
        t.ok[k] = s < g.s1;
        t.row[k] = s * 32 + lane;
        t.o[k] = t.row[k] - g.row0;
        t.le[k] = t.ge[k] = t.wd[k] = 0;
        if (!t.ok[k])
            continue;
        int b0 = a.slice_ptr[s], b1 = a.slice_ptr[s + 1];
        t.wd[k] = (b1 - b0) >> 5;
        t.ge[k] = b0 + lane;
        t.le[k] = (SM ? b0 - g.e0 : b0) + lane;
    }
}

// sum_j A_ij v_j of row slot k from shared memory; LC = local columns
// (shared memory when SM, else global), VAL = matrix values
template <int RPT, typename MV, typename V, typename ACC>
__device__ __forceinline__ ACC spmv_local(const Rows<RPT> &t, int k, const int *LC, const MV *VAL,
                                          bool val_by_global, const V *sv)
{
    ACC sum = 0;
#pragma unroll 4
    for (int c = 0; c < t.wd[k]; ++c) {
        int lc = LC[t.le[k] + c * 32];
        MV v = val_by_global ? __ldg(VAL + t.ge[k] + c * 32) : VAL[t.le[k] + c * 32];
        sum += (ACC)v * (ACC)sv[lc];
    }
    return sum;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Neighbour exchange of a Chebyshev step direction without a grid barrier.
// The block writes its own values to its shared segment and, with the step's
// tag, to the tagged buffer (one 64-bit store per row: value and tag arrive
// together); then it reads each halo value from the owner's word until the
// tag is the current one.  Two buffers alternate: when a block overwrites
// its word of step n - 2 with step n, every block that reads it has already
// published step n - 1, which it does only after it has read step n - 2 (the
// halo relation of a symmetric matrix is symmetric; the host checks it).
// Tags: epoch << 24 | step count; stale words hold another step count or
// another epoch.  Each wait has an iteration limit and gives up when another
// block has recorded PIC_ERR_TIMEOUT.
template <int RPT>
__device__ bool tagged_exchange(const Rows<RPT> &t, const PcgArgs &a, const Seg &g, float *s_d,
                                const float (&d)[RPT])
{
    const unsigned tag = (t.epoch << 24) | (t.pub & 0xFFFFFFu);
    unsigned long long *buf = a.dtag[t.pub & 1u];
    ++t.pub;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        if (!t.ok[k])
            continue;
        s_d[t.o[k]] = d[k];
        st_relaxed_u64(buf + t.row[k],
                       (unsigned long long)__float_as_uint(d[k]) | ((unsigned long long)tag << 32));
    }
    int bad = 0;
    for (int i = threadIdx.x; i < g.nh && !bad; i += blockDim.x) {
        const unsigned long long *src = buf + a.halo_idx[g.h0 + i];
        unsigned long long v = ld_relaxed_u64(src);
        long long spins = 0;
        while ((unsigned)(v >> 32) != tag) {
            ++spins;
            if (spins > a.spin_limit ||
                ((spins & 1023) == 0 && ld_volatile_i32(&a.st->err) == PIC_ERR_TIMEOUT)) {
                bad = 1;
                break;
            }
            v = ld_relaxed_u64(src);
        }
        s_d[g.nrows + i] = __uint_as_float((unsigned)v);
    }
    if (bad)
        atomicCAS(&a.st->err, 0, PIC_ERR_TIMEOUT);
    return __syncthreads_or(bad) == 0;
}

template <int RPT, typename T>
__device__ __forceinline__ bool tagged_exchange_t(const Rows<RPT> &t, const PcgArgs &a,
                                                  const Seg &g, T *s_d, const T (&d)[RPT])
{
    if constexpr (sizeof(T) == 4)
        return tagged_exchange<RPT>(t, a, g, s_d, d);
    return false;
}

// z = M^-1 r for the preconditioner.  Jacobi: z = D^-1 r.  Chebyshev of
// degree k: z = p_k(D^-1 M) D^-1 r, computed as k steps of the Chebyshev
// iteration for M y = r from y = 0 on the interval [a, b] (Saad, Iterative
// Methods for Sparse Linear Systems, Alg. 12.1).  This is a fixed symmetric
// positive definite operator as long as b bounds the spectrum of D^-1 M
// (Gershgorin), so CG stays CG.  Each step after the first needs one SpMV of
// the step direction: published to the block's shared segment and to a
// double-buffered global halo copy, one plain grid barrier, no reduction.
template <typename T> __device__ __forceinline__ T cheb_coef(double d, float f);
template <> __device__ __forceinline__ double cheb_coef<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float cheb_coef<float>(double, float f) { return f; }

// One Chebyshev step after the direction d_j has been staged in s_d (own
// rows and halo): rc -= M d_j, d_{j+1} = c1 d_j + c2 D^-1 rc.
template <int RPT, typename T>
__device__ __forceinline__ void cheb_update(const Rows<RPT> &t, const PcgArgs &a, const int *LC,
                                            const T *VAL, const T (&dinv)[RPT], const T *s_d,
                                            int j, T (&rc)[RPT], T (&d)[RPT])
{
    const T c1 = cheb_coef<T>(a.cheb_c1[j - 1], a.cheb_c1f[j - 1]);
    const T c2 = cheb_coef<T>(a.cheb_c2[j - 1], a.cheb_c2f[j - 1]);
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        if (!t.ok[k])
            continue;
        T ad = 0;
#pragma unroll 4
        for (int c = 0; c < t.wd[k]; ++c) {
            int lc = LC[t.le[k] + c * 32];
            ad += VAL[t.le[k] + c * 32] * s_d[lc];
        }
        rc[k] = rc[k] - ad;
        d[k] = c1 * d[k] + c2 * (dinv[k] * rc[k]);
    }
}

template <int RPT, typename T>
__device__ bool coarse_correction(const Rows<RPT> &t, const PcgArgs &a, const T (&dinv)[RPT],
                                  const T (&r)[RPT], T (&z)[RPT]);
template <int RPT, typename T>
__device__ void coarse_publish(const Rows<RPT> &t, const PcgArgs &a, const T (&dinv)[RPT],
                               const T (&r)[RPT]);
__device__ bool coarse_sync(const PcgArgs &a);
__device__ void coarse_apply(const PcgArgs &a);
__device__ double *coarse_z0();

// Per-warp partials of a sum that rides on the polynomial's first grid
// barrier, and ([RW]) its grid total.
__device__ __noinline__ double *ride_part()
{
    __shared__ double part[RW + 1];
    return part;
}

// After the barrier: warp 1 adds the blocks' partials of the ride in block
// order (the same order in every block) into ride_part()[RW].
__device__ __forceinline__ void ride_gather(const PcgArgs &a, int set)
{
    if ((threadIdx.x >> 5) != 1)
        return;
    const int lane = threadIdx.x & 31;
    const Grp g = grp_of(a);
    double v = 0.0;
    for (int b = lane; b < g.nb; b += 32)
        v += __ldcg(a.partials + ((size_t)set * gridDim.x + g.b0 + b) * 4);
    v = warp_sum(v);
    if (lane == 0)
        ride_part()[RW] = v;
}

// ---------------------------------------------------------------------------
// Multigrid V-cycle preconditioner (cheb_local == 4; hierarchy of mg.cu).
//
//   z  = S0 r                       Chebyshev smoothing of degree k0 from zero
//   r1 = P0^T (r - A z)             restriction: sums over the aggregates
//   e1 = V1 r1                      the same cycle on level 1 (degree k1),
//                                   with level 2 solved exactly: e2 = A2^-1 r2
//   z += P0 e1                      prolongation (piecewise constant)
//   z += S0 (r - A z)               smoothing of degree k0 from z
//
// S0 = p(D^-1 A) D^-1 is symmetric and the same on both sides, so the cycle is
// a fixed symmetric positive definite operator and CG stays CG.  Aggregates
// never cross blocks: restriction and prolongation are block-local; the
// smoothing steps exchange halo values as the Chebyshev preconditioner does
// (tagged words in FP32, grid barriers in FP64); the level-2 right-hand side
// crosses one grid barrier, after which every block applies its own rows of
// A2^-1.  Exchanges of the fine level: 2 k0; of level 1: 2 k1.
// ---------------------------------------------------------------------------
template <typename T> struct MgSm {
    T *v;          // [own | halo] level-1 vector of the current exchange
    T *r, *e, *rc, *d, *e2;
    int L0, own1, h0, nh, Q0, own2;
};

template <typename T> __device__ __forceinline__ const T *mg_a1_val(const PcgArgs &a);
template <> __device__ __forceinline__ const float *mg_a1_val<float>(const PcgArgs &a)
{
    return a.mg_a1_val32;
}
template <> __device__ __forceinline__ const double *mg_a1_val<double>(const PcgArgs &a)
{
    return a.mg_a1_val64;
}
template <typename T> __device__ __forceinline__ const T *mg_dinv1(const PcgArgs &a);
template <> __device__ __forceinline__ const float *mg_dinv1<float>(const PcgArgs &a)
{
    return a.mg_dinv1_32;
}
template <> __device__ __forceinline__ const double *mg_dinv1<double>(const PcgArgs &a)
{
    return a.mg_dinv1_64;
}

// Level-1 halo exchange of src (own rows) into m.v [own | halo].  FP32 with
// tagged words: the level's own count of exchanges and buffers (the halo
// relation of the symmetric level-1 matrix is symmetric, checked on the
// host), so the double-buffer argument of the fine exchange holds per level;
// otherwise through a grid barrier and two alternating global buffers.
template <typename T>
__device__ bool mg_exchange1(const PcgArgs &a, const MgSm<T> &m, const T *src, unsigned &pub1,
                             unsigned epoch)
{
    __syncthreads();
    const unsigned par = pub1 & 1u;
    if constexpr (sizeof(T) == 4) {
        if (a.mg_dtag1) {
            const unsigned tag = (epoch << 24) | (pub1 & 0xFFFFFFu);
            unsigned long long *buf = a.mg_dtag1 + (size_t)par * a.mg_n1;
            ++pub1;
            for (int l = threadIdx.x; l < m.own1; l += blockDim.x) {
                const float v = (float)src[l];
                m.v[l] = v;
                st_relaxed_u64(buf + m.L0 + l, (unsigned long long)__float_as_uint(v) |
                                                    ((unsigned long long)tag << 32));
            }
            int bad = 0;
            for (int i = threadIdx.x; i < m.nh && !bad; i += blockDim.x) {
                const unsigned long long *q = buf + a.mg_h1_idx[m.h0 + i];
                unsigned long long v = ld_relaxed_u64(q);
                long long spins = 0;
                while ((unsigned)(v >> 32) != tag) {
                    ++spins;
                    if (spins > a.spin_limit ||
                        ((spins & 1023) == 0 && ld_volatile_i32(&a.st->err) == PIC_ERR_TIMEOUT)) {
                        bad = 1;
                        break;
                    }
                    v = ld_relaxed_u64(q);
                }
                m.v[m.own1 + i] = __uint_as_float((unsigned)v);
            }
            if (bad)
                atomicCAS(&a.st->err, 0, PIC_ERR_TIMEOUT);
            return __syncthreads_or(bad) == 0;
        }
    }
    ++pub1;
    T *gbuf;
    if constexpr (sizeof(T) == 4)
        gbuf = a.mg_g1f[par];
    else
        gbuf = a.mg_g1d[par];
    for (int l = threadIdx.x; l < m.own1; l += blockDim.x) {
        const T v = src[l];
        m.v[l] = v;
        gbuf[m.L0 + l] = v;
    }
    if (!grid_sync(a))
        return false;
    for (int i = threadIdx.x; i < m.nh; i += blockDim.x)
        m.v[m.own1 + i] = __ldcg(gbuf + a.mg_h1_idx[m.h0 + i]);
    __syncthreads();
    return true;
}

// (A1 m.v) of the block's level-1 row l
template <typename T>
__device__ __forceinline__ T mg_a1_row(const PcgArgs &a, const MgSm<T> &m, int l)
{
    const T *val = mg_a1_val<T>(a);
    const int k1 = __ldg(a.mg_a1_ptr + m.L0 + l + 1);
    T s = (T)0;
    for (int k = __ldg(a.mg_a1_ptr + m.L0 + l); k < k1; ++k)
        s += __ldg(val + k) * m.v[__ldg(a.mg_a1_col + k)];
    return s;
}

// Chebyshev smoothing on level 1 (degree mg_deg1), from zero (m.e = 0) or
// from the current m.e: m.e += p(D1^-1 A1) D1^-1 (m.r - A1 m.e)
template <typename T>
__device__ bool mg_smooth1(const PcgArgs &a, const MgSm<T> &m, bool from_zero, unsigned &pub1,
                           unsigned epoch)
{
    const T *dinv1 = mg_dinv1<T>(a);
    const T it1 = cheb_coef<T>(a.mg_inv_theta, a.mg_inv_thetaf);
    if (!from_zero && !mg_exchange1<T>(a, m, m.e, pub1, epoch))
        return false;
    for (int l = threadIdx.x; l < m.own1; l += blockDim.x) {
        const T rc = from_zero ? m.r[l] : m.r[l] - mg_a1_row<T>(a, m, l);
        const T d = __ldg(dinv1 + m.L0 + l) * rc * it1;
        m.rc[l] = rc;
        m.d[l] = d;
        m.e[l] = from_zero ? d : m.e[l] + d;
    }
    for (int j = 1; j < a.mg_deg1; ++j) {
        if (!mg_exchange1<T>(a, m, m.d, pub1, epoch))
            return false;
        const T c1 = cheb_coef<T>(a.mg_c1[j - 1], a.mg_c1f[j - 1]);
        const T c2 = cheb_coef<T>(a.mg_c2[j - 1], a.mg_c2f[j - 1]);
        for (int l = threadIdx.x; l < m.own1; l += blockDim.x) {
            const T rc = m.rc[l] - mg_a1_row<T>(a, m, l);
            const T d = c1 * m.d[l] + c2 * (__ldg(dinv1 + m.L0 + l) * rc);
            m.rc[l] = rc;
            m.d[l] = d;
            m.e[l] = m.e[l] + d;
        }
    }
    __syncthreads();
    return true;
}

// The level-1 cycle on m.r into m.e (level 2 exact)
template <typename T>
__device__ bool mg_level1(const PcgArgs &a, const MgSm<T> &m, unsigned &pub1, unsigned epoch)
{
    if (!mg_smooth1<T>(a, m, true, pub1, epoch))
        return false;
    // residual r - A1 e = rc - A1 d_last
    if (!mg_exchange1<T>(a, m, m.d, pub1, epoch))
        return false;
    for (int l = threadIdx.x; l < m.own1; l += blockDim.x)
        m.rc[l] = m.rc[l] - mg_a1_row<T>(a, m, l);
    __syncthreads();
    // restriction to the block's level-2 rows, published for every block
    T *r2;
    if constexpr (sizeof(T) == 4)
        r2 = a.mg_r2f;
    else
        r2 = a.mg_r2d;
    for (int q = threadIdx.x; q < m.own2; q += blockDim.x) {
        T s = (T)0;
        const int k1 = __ldg(a.mg_m1_ptr + m.Q0 + q + 1);
        for (int k = __ldg(a.mg_m1_ptr + m.Q0 + q); k < k1; ++k)
            s += m.rc[__ldg(a.mg_m1_idx + k)];
        r2[m.Q0 + q] = s;
    }
    if (!grid_sync(a))
        return false;
    // the block's rows of e2 = A2^-1 r2, one warp per row
    {
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
        const int n2 = a.mg_n2;
        for (int q = w; q < m.own2; q += nw) {
            const float *row = a.mg_a2inv + (size_t)(m.Q0 + q) * n2;
            T s = (T)0;
            for (int c = lane; c < n2; c += 32)
                s += (T)__ldg(row + c) * __ldcg(r2 + c);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                s += __shfl_xor_sync(FULL_MASK, s, o);
            if (lane == 0)
                m.e2[q] = s;
        }
    }
    __syncthreads();
    for (int l = threadIdx.x; l < m.own1; l += blockDim.x)
        m.e[l] = m.e[l] + m.e2[__ldg(a.mg_agg1 + m.L0 + l)];
    __syncthreads();
    return mg_smooth1<T>(a, m, false, pub1, epoch);
}

// fine-level halo exchange of d into s_d (tagged words in FP32 when
// available, otherwise own values to g_d, a grid barrier and the halo staged)
template <int RPT, typename T>
__device__ bool fine_exchange(const Rows<RPT> &t, const PcgArgs &a, const Seg &g, T *s_d, T *g_d,
                              const T (&d)[RPT])
{
    if (sizeof(T) == 4 && a.dtag[0])
        return tagged_exchange_t<RPT, T>(t, a, g, s_d, d);
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        if (!t.ok[k])
            continue;
        s_d[t.o[k]] = d[k];
        g_d[t.row[k]] = d[k];
    }
    if (!grid_sync(a))
        return false;
    stage_halo(s_d, (const T *)g_d, a, g);
    __syncthreads();
    return true;
}

template <int RPT, typename T>
__device__ __forceinline__ T fine_row(const Rows<RPT> &t, int k, const int *LC, const T *VAL,
                                      const T *s_v)
{
    T s = 0;
#pragma unroll 4
    for (int c = 0; c < t.wd[k]; ++c) {
        int lc = LC[t.le[k] + c * 32];
        s += VAL[t.le[k] + c * 32] * s_v[lc];
    }
    return s;
}

template <int RPT, typename T>
__device__ bool mg_vcycle(const Rows<RPT> &t, const PcgArgs &a, const Seg &g, const int *LC,
                          const T *VAL, const T (&dinv)[RPT], const T (&r)[RPT], T (&z)[RPT],
                          T *s_d0, T *s_d1, T *g_d0, T *g_d1)
{
    extern __shared__ __align__(16) unsigned char smem[];
    MgSm<T> m;
    {
        T *base = (T *)(smem + a.mg_smem_off);
        m.v = base;
        m.r = m.v + a.mg_max_l1_local;
        m.e = m.r + a.mg_max_l1_own;
        m.rc = m.e + a.mg_max_l1_own;
        m.d = m.rc + a.mg_max_l1_own;
        m.e2 = m.d + a.mg_max_l1_own;
        const int b = blockIdx.x;
        m.L0 = __ldg(a.mg_l1_off + b);
        m.own1 = __ldg(a.mg_l1_off + b + 1) - m.L0;
        m.h0 = __ldg(a.mg_h1_ptr + b);
        m.nh = __ldg(a.mg_h1_ptr + b + 1) - m.h0;
        m.Q0 = __ldg(a.mg_l2_off + b);
        m.own2 = __ldg(a.mg_l2_off + b + 1) - m.Q0;
    }
    const T it0 = cheb_coef<T>(a.cheb_inv_theta, a.cheb_inv_thetaf);
    T rc[RPT], d[RPT];
    int par = 0;
    // pre-smoothing from zero
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        rc[k] = r[k];
        d[k] = dinv[k] * rc[k] * it0;
        z[k] = d[k];
    }
    for (int j = 1; j < a.mg_deg0; ++j) {
        T *sd = par ? s_d1 : s_d0;
        T *gd = par ? g_d1 : g_d0;
        par ^= 1;
        if (!fine_exchange<RPT, T>(t, a, g, sd, gd, d))
            return false;
        cheb_update<RPT, T>(t, a, LC, VAL, dinv, sd, j, rc, d);
#pragma unroll
        for (int k = 0; k < RPT; ++k)
            z[k] = z[k] + d[k];
    }
    // the residual r - A z = rc - A d_last
    {
        T *sd = par ? s_d1 : s_d0;
        T *gd = par ? g_d1 : g_d0;
        par ^= 1;
        if (!fine_exchange<RPT, T>(t, a, g, sd, gd, d))
            return false;
#pragma unroll
        for (int k = 0; k < RPT; ++k)
            if (t.ok[k])
                rc[k] = rc[k] - fine_row<RPT, T>(t, k, LC, VAL, sd);
    }
    // restriction: the residual of the own rows in the other buffer, summed
    // over each aggregate in a fixed order
    T *st = par ? s_d1 : s_d0;
#pragma unroll
    for (int k = 0; k < RPT; ++k)
        if (t.ok[k])
            st[t.o[k]] = rc[k];
    __syncthreads();
    for (int l = threadIdx.x; l < m.own1; l += blockDim.x) {
        T s = (T)0;
        const int k1 = __ldg(a.mg_m0_ptr + m.L0 + l + 1);
        for (int k = __ldg(a.mg_m0_ptr + m.L0 + l); k < k1; ++k)
            s += st[__ldg(a.mg_m0_idx + k)];
        m.r[l] = s;
    }
    __syncthreads();
    if (!mg_level1<T>(a, m, t.pub1, t.epoch))
        return false;
    // prolongation
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        if (!t.ok[k])
            continue;
        const int l = __ldg(a.mg_agg0 + t.row[k]);
        if (l >= 0)
            z[k] = z[k] + m.e[l];
    }
    // post-smoothing from z
    {
        T *sd = par ? s_d1 : s_d0;
        T *gd = par ? g_d1 : g_d0;
        par ^= 1;
        if (!fine_exchange<RPT, T>(t, a, g, sd, gd, z))
            return false;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            if (!t.ok[k])
                continue;
            rc[k] = r[k] - fine_row<RPT, T>(t, k, LC, VAL, sd);
            d[k] = dinv[k] * rc[k] * it0;
            z[k] = z[k] + d[k];
        }
    }
    for (int j = 1; j < a.mg_deg0; ++j) {
        T *sd = par ? s_d1 : s_d0;
        T *gd = par ? g_d1 : g_d0;
        par ^= 1;
        if (!fine_exchange<RPT, T>(t, a, g, sd, gd, d))
            return false;
        cheb_update<RPT, T>(t, a, LC, VAL, dinv, sd, j, rc, d);
#pragma unroll
        for (int k = 0; k < RPT; ++k)
            z[k] = z[k] + d[k];
    }
    return true;
}

template <int RPT, typename T, bool MG = false>
__device__ bool apply_precond(const Rows<RPT> &t, const PcgArgs &a, const Seg &g, const int *LC,
                              const T *VAL, const T (&dinv)[RPT], const T (&r)[RPT],
                              T (&z)[RPT], T *s_d0, T *s_d1, T *g_d0, T *g_d1,
                              bool have_z0 = false, double z0_given = 0.0)
{
    if constexpr (MG && RPT <= 4) {
        if (a.cheb_local == 4 && a.mg_n1 > 0)
            return mg_vcycle<RPT, T>(t, a, g, LC, VAL, dinv, r, z, s_d0, s_d1, g_d0, g_d1);
    }
    if (a.cheb_degree < 2) {
#pragma unroll
        for (int k = 0; k < RPT; ++k)
            z[k] = dinv[k] * r[k];
        if (a.cheb_local >= 2 && a.coarse_inv)
            return coarse_correction<RPT, T>(t, a, dinv, r, z);
        return true;
    }
    // the whole-matrix polynomial with the coarse correction: the blocks'
    // residual sums cross the polynomial's first grid barrier (no barrier of
    // their own); the correction is added at the end
    // have_z0: the caller already formed this block's coarse correction
    // (A0^-1 R0 r)_b on an earlier barrier, so the polynomial's first step
    // needs no grid barrier either
    const bool fused_coarse = a.cheb_local == 3 && a.coarse_inv;
    const bool coarse_j1 = fused_coarse && !have_z0;
    T z0 = have_z0 ? (T)z0_given : (T)0;
    T rc[RPT], d[RPT];
    const T inv_theta = cheb_coef<T>(a.cheb_inv_theta, a.cheb_inv_thetaf);
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        rc[k] = r[k];
        d[k] = dinv[k] * rc[k] * inv_theta;
        z[k] = (T)0;
    }
    for (int j = 1;; ++j) {
#pragma unroll
        for (int k = 0; k < RPT; ++k)
            z[k] = z[k] + d[k];
        if (j >= a.cheb_degree)
            break;
        T *s_d = (j & 1) ? s_d1 : s_d0;
        T *g_d = (j & 1) ? g_d1 : g_d0;
        if (a.cheb_local == 1 || a.cheb_local == 2) {
            // block-local form: the polynomial in the block's own diagonal block
            // of D^-1 M (couplings to other blocks' rows dropped): still a fixed
            // symmetric positive definite operator, and no grid barrier
#pragma unroll
            for (int k = 0; k < RPT; ++k)
                if (t.ok[k])
                    s_d[t.o[k]] = d[k];
            for (int i = threadIdx.x; i < g.nh; i += blockDim.x)
                s_d[g.nrows + i] = (T)0;
            __syncthreads();
        } else if (sizeof(T) == 4 && a.dtag[0] && !(coarse_j1 && j == 1)) {
            if (!tagged_exchange_t<RPT, T>(t, a, g, s_d, d))
                return false;
        } else {
#pragma unroll
            for (int k = 0; k < RPT; ++k) {
                if (!t.ok[k])
                    continue;
                s_d[t.o[k]] = d[k];
                g_d[t.row[k]] = d[k];
            }
            if (coarse_j1 && j == 1) {
                coarse_publish<RPT, T>(t, a, dinv, r);
                if (!coarse_sync(a))
                    return false;
                coarse_apply(a);   // overlaps the halo staging; read after the block barrier
            } else if (!grid_sync(a)) {
                return false;
            }
            stage_halo(s_d, (const T *)g_d, a, g);
            __syncthreads();
            if (coarse_j1 && j == 1)
                z0 = (T)*coarse_z0();
        }
        cheb_update<RPT, T>(t, a, LC, VAL, dinv, s_d, j, rc, d);
    }
    if (fused_coarse) {
#pragma unroll
        for (int k = 0; k < RPT; ++k)
            if (t.ok[k] && dinv[k] != (T)0)
                z[k] = z[k] + z0;
        return true;
    }
    if (a.cheb_local == 2 && a.coarse_inv)
        return coarse_correction<RPT, T>(t, a, dinv, r, z);
    return true;
}

// Two-level form: z += R0^T A0^-1 R0 r with R0 summing the rows of each block
// (one constant coarse vector per block, A0 = R0 M R0^T factored on the host).
// The blocks' residual sums cross one grid barrier; each block then needs only
// its own row of A0^-1.
// The block's residual sum (R0 r)_b: each warp's share to coarse_part(); the
// grid barrier's arriving thread adds them up and publishes the sum
// (a Ride of grid_sync), so no block barrier of its own.
__device__ __noinline__ double *coarse_part()
{
    __shared__ double part[RW];
    return part;
}
__device__ __noinline__ double *coarse_z0()
{
    __shared__ double z0;
    return &z0;
}

template <int RPT, typename T>
__device__ void coarse_publish(const Rows<RPT> &t, const PcgArgs &a, const T (&dinv)[RPT],
                               const T (&r)[RPT])
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double s = 0.0;
    if constexpr (sizeof(T) == 4) {
        DF x = {0.f, 0.f};
#pragma unroll
        for (int k = 0; k < RPT; ++k)
            if (t.ok[k] && dinv[k] != (T)0)
                df_add(x, (float)r[k]);
        s = df_warp_sum(x);
    } else {
#pragma unroll
        for (int k = 0; k < RPT; ++k)
            if (t.ok[k] && dinv[k] != (T)0)
                s += (double)r[k];
        for (int o = 16; o > 0; o >>= 1)
            s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    if (lane == 0)
        coarse_part()[w] = s;
}

__device__ __forceinline__ bool coarse_sync(const PcgArgs &a)
{
    return grid_sync(a, Ride{coarse_part(), RW, a.coarse_r + blockIdx.x});
}

// After the barrier: warp 0 forms (A0^-1 R0 r)_b in shared memory; it is
// visible to the block after the next block barrier.
__device__ void coarse_apply(const PcgArgs &a)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w == 0) {
        const float *row = a.coarse_inv + (size_t)blockIdx.x * gridDim.x;
        double v = 0.0;
        for (int c = lane; c < (int)gridDim.x; c += 32)
            v += (double)row[c] * __ldcg(a.coarse_r + c);
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0)
            *coarse_z0() = v;
    }
}

template <int RPT, typename T>
__device__ bool coarse_correction(const Rows<RPT> &t, const PcgArgs &a, const T (&dinv)[RPT],
                                  const T (&r)[RPT], T (&z)[RPT])
{
    coarse_publish<RPT, T>(t, a, dinv, r);
    if (!coarse_sync(a))
        return false;
    coarse_apply(a);
    __syncthreads();
    const T z0 = (T)*coarse_z0();
#pragma unroll
    for (int k = 0; k < RPT; ++k)
        if (t.ok[k] && dinv[k] != (T)0)
            z[k] = z[k] + z0;
    return true;
}

// The merged form's coarse sums: the blocks' sums of r (coarse_part(),
// published to coarse_r[b]) and of A p (coarse_part2(), to coarse_r[G + b]);
// after the barrier warp 0 forms both (A0^-1 R0 .)_b.
__device__ __noinline__ double *coarse_part2()
{
    __shared__ double part[RW];
    return part;
}
__device__ __noinline__ double *coarse_z0_pair()
{
    __shared__ double z0[2];
    return z0;
}
__device__ void coarse_apply_pair(const PcgArgs &a)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w == 0) {
        const float *row = a.coarse_inv + (size_t)blockIdx.x * gridDim.x;
        double v = 0.0, u = 0.0;
        for (int c = lane; c < (int)gridDim.x; c += 32) {
            const double ic = (double)row[c];
            v += ic * __ldcg(a.coarse_r + c);
            u += ic * __ldcg(a.coarse_r + gridDim.x + c);
        }
        v = warp_sum(v);
        u = warp_sum(u);
        if (lane == 0) {
            coarse_z0_pair()[0] = v;
            coarse_z0_pair()[1] = u;
        }
    }
}

// ---------------------------------------------------------------------------
// FP64 Jacobi-PCG (the plain FP64 form), two grid barriers per iteration
// ---------------------------------------------------------------------------
template <int RPT, bool SM>
__global__ void __launch_bounds__(RB, 1) k_pcg64_res(PcgArgs a)
{
    grid_sync_init();
    extern __shared__ __align__(16) unsigned char smem[];
    const Seg g = block_seg(a);
    double *s_val = (double *)smem;
    int *s_lc = (int *)(smem + (SM ? a.max_chunk * 8 : 0));
    size_t off = SM ? (size_t)a.max_chunk * 12 : 0;
    off = (off + 15) & ~(size_t)15;
    double *s_z = (double *)(smem + off);
    double *s_p0 = s_z + a.max_local;
    double *s_p1 = s_p0 + a.max_local;
    double *s_d0 = s_p1 + a.max_local;
    double *s_d1 = s_d0 + a.max_local;
    if (SM) {
        int e1 = a.slice_ptr[g.s1];
        stage_chunk(s_val, a.val64, g.e0, e1);
        stage_chunk(s_lc, a.lcol, g.e0, e1);
    }
    const int *LC = SM ? s_lc : a.lcol;
    const double *VAL = SM ? s_val : a.val64;
    Rows<RPT> t;
    init_rows<RPT, SM>(t, a, g);
    double x[RPT], r[RPT], z[RPT], p[RPT], ap[RPT], dinv[RPT], f[RPT];
    // r = f - M x: x of the own rows into s_z, halo of x staged
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        x[k] = r[k] = z[k] = p[k] = ap[k] = dinv[k] = f[k] = 0.0;
        if (!t.ok[k])
            continue;
        x[k] = a.x[t.row[k]];
        dinv[k] = a.dinv64[t.row[k]];
        f[k] = rhs_entry(a, t.row[k]);
        s_z[t.o[k]] = x[k];
    }
    stage_halo(s_z, a.x, a, g);
    __syncthreads();
    double acc[3] = {0.0, 0.0, 0.0}, tot[3];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        if (!t.ok[k])
            continue;
        double axv = spmv_local<RPT, double, double, double>(t, k, LC, VAL, false, s_z);
        r[k] = f[k] - axv;
        acc[1] += r[k] * r[k];
        acc[2] += f[k] * f[k];
    }
    __syncthreads();
    if (!apply_precond<RPT, double, true>(t, a, g, LC, VAL, dinv, r, z, s_d0, s_d1, a.d0, a.d1))
        return;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        if (!t.ok[k])
            continue;
        acc[0] += r[k] * z[k];
        s_z[t.o[k]] = z[k];
        s_p0[t.o[k]] = 0.0;
        a.z[t.row[k]] = z[k];
        a.p0[t.row[k]] = 0.0;
    }
    int set = 0;
    if (!grid_sum<3, RB>(acc, set, a, tot))
        return;
    set ^= 1;
    double rz = tot[0], rr = tot[1], ff = tot[2];
    int it = 0, status = 0;
    if (ff == 0.0) {
#pragma unroll
        for (int k = 0; k < RPT; ++k)
            x[k] = 0.0;
        rr = 0.0;
        ff = 1.0;
    }
    const double tol2 = a.rtol * a.rtol * ff;
    double beta = 0.0;
    int cur = 0;
    while (rr > tol2) {
        if (it >= a.max_iter) {
            status = PIC_ERR_NOT_CONVERGED;
            break;
        }
        double *sp_old = cur ? s_p1 : s_p0;
        double *sp_new = cur ? s_p0 : s_p1;
        const double *gp_old = cur ? a.p1 : a.p0;
        double *gp_new = cur ? a.p0 : a.p1;
        stage_halo(s_z, a.z, a, g);
        stage_halo(sp_old, gp_old, a, g);
        __syncthreads();
        double pap[1] = {0.0};
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            if (!t.ok[k])
                continue;
            double sum = 0.0;
#pragma unroll 4
            for (int c = 0; c < t.wd[k]; ++c) {
                int lc = LC[t.le[k] + c * 32];
                sum += VAL[t.le[k] + c * 32] * (s_z[lc] + beta * sp_old[lc]);
            }
            p[k] = z[k] + beta * p[k];
            ap[k] = sum;
            sp_new[t.o[k]] = p[k];
            gp_new[t.row[k]] = p[k];
            pap[0] += p[k] * sum;
        }
        double pt2[2];
        if (!grid_sum_f<1, 2, RB>(pap, set, a, pt2,
                                  [rz](double *q) { q[1] = rz / q[0]; }))
            return;
        set ^= 1;
        double alpha = pt2[1];
        double acc2[2] = {0.0, 0.0};
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            if (!t.ok[k])
                continue;
            x[k] = x[k] + alpha * p[k];
            r[k] = r[k] - alpha * ap[k];
        }
        if (!apply_precond<RPT, double, true>(t, a, g, LC, VAL, dinv, r, z, s_d0, s_d1, a.d0, a.d1))
            return;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            if (!t.ok[k])
                continue;
            s_z[t.o[k]] = z[k];
            a.z[t.row[k]] = z[k];
            acc2[0] += r[k] * z[k];
            acc2[1] += r[k] * r[k];
        }
        double t3[3];
        if (!grid_sum_f<2, 3, RB>(acc2, set, a, t3,
                                  [rz](double *q) { q[2] = q[0] / rz; }))
            return;
        set ^= 1;
        beta = t3[2];
        rz = t3[0];
        rr = t3[1];
        ++it;
        cur ^= 1;
    }
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        if (!t.ok[k])
            continue;
        a.x[t.row[k]] = x[k];
        int node = a.dof_node[t.row[k]];
        if (node >= 0)
            a.phi[node] = x[k];
    }
    finish(a, it, sqrt(rr / ff), status);
}

// ---------------------------------------------------------------------------
// FP32 Jacobi-PCG inside FP64 iterative refinement.  The outer loop
// recomputes r = f - M x in FP64 (FP64 matrix values, FP64 x) and adds the
// FP32 correction d in FP64.  The inner solve of M d = r runs in FP32 with
// FP64 dot products, as standard PCG (two grid barriers per iteration) or as
// pipelined PCG (Ghysels & Vanroose, Parallel Computing 40, 2014), whose
// recurrences let one barrier per iteration publish m = D^-1 w for the SpMV
// n = A m and complete the reductions, at the price of a larger gap between
// the recursive and the true residual.
// ---------------------------------------------------------------------------
template <int RPT> struct In32 {
    const int *LC;
    const float *VAL;
    float dinv[RPT];
};

// The p.Ap reduction of the standard iteration carrying the coarse
// correction of the preconditioner application that follows it: with
// r' = r - alpha A p, R0 r' = R0 r - alpha R0 A p, so every block publishes
// its sums of r and of A p (rows with a nonzero diagonal) beside its p.Ap
// partial, and after the same barrier forms its rows of A0^-1 R0 r and
// A0^-1 R0 A p (warp 1) while warp 0 totals p.Ap (resident solver, one
// system).  out: [0] p.Ap, [1] alpha = rz / p.Ap, [2] (A0^-1 R0 r)_b,
// [3] (A0^-1 R0 A p)_b.
__device__ bool grid_sum_pap_coarse(const DF &pap, const DF &sr, const DF &sq, int set,
                                    const PcgArgs &a, double rz, double (&out)[4])
{
    double *vals = reduction_buffer();
    double *res = vals + 3 * 512;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const DF v[3] = {pap, sr, sq};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double x = df_warp_sum(v[k]);
        if (lane == 0)
            vals[k * RW + wid] = x;
    }
    __syncthreads();
    const size_t G = gridDim.x;
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double x = lane < RW ? vals[k * RW + lane] : 0.0;
            x = warp_sum(x);
            if (lane == 0)
                a.partials[((size_t)set * G + blockIdx.x) * 4 + k] = x;
        }
    }
    if (!grid_sync(a))
        return false;
    if (wid == 0) {
        double x = 0.0;
        for (size_t b = lane; b < G; b += 32)
            x += __ldcg(a.partials + ((size_t)set * G + b) * 4);
        x = warp_sum(x);
        if (lane == 0) {
            res[0] = x;
            res[1] = rz / x;
        }
    } else if (wid == 1) {
        const float *row = a.coarse_inv + (size_t)blockIdx.x * G;
        double v1 = 0.0, v2 = 0.0;
        for (size_t c = lane; c < G; c += 32) {
            const double ic = (double)row[c];
            v1 += ic * __ldcg(a.partials + ((size_t)set * G + c) * 4 + 1);
            v2 += ic * __ldcg(a.partials + ((size_t)set * G + c) * 4 + 2);
        }
        v1 = warp_sum(v1);
        v2 = warp_sum(v2);
        if (lane == 0) {
            res[2] = v1;
            res[3] = v2;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k)
        out[k] = res[k];
    return true;
}

template <int RPT>
__device__ bool inner_standard(const Rows<RPT> &t, const In32<RPT> &m, const PcgArgs &a,
                               const Seg &g, float (&rv)[RPT], float (&d)[RPT], float *s_z,
                               float *s_p0, float *s_p1, float *s_d0, float *s_d1,
                               double itol, int &set, int &it)
{
    float z[RPT], p[RPT], ap[RPT];
    DF acc[2] = {{0.f, 0.f}, {0.f, 0.f}};
    double tot[2];
    if (!apply_precond<RPT, float, true>(t, a, g, m.LC, m.VAL, m.dinv, rv, z, s_d0, s_d1, a.d32_0,
                                   a.d32_1))
        return false;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        p[k] = ap[k] = 0.f;
        if (!t.ok[k])
            continue;
        s_z[t.o[k]] = z[k];
        a.z32[t.row[k]] = z[k];
        df_add_prod(acc[0], rv[k], z[k]);
        df_add_prod(acc[1], rv[k], rv[k]);
    }
    if (!grid_sum_df<2, 2, RB>(acc, set, a, tot, NoFinish()))
        return false;
    set ^= 1;
    double rz = tot[0], rr = tot[1];
    const double itol2 = itol * itol * rr;
    // the coarse correction of the whole-matrix polynomial rides on the
    // p.Ap barrier (one grid barrier fewer per iteration)
    const bool coarse_ride = a.cheb_local == 3 && a.coarse_inv && a.cheb_degree >= 2;
    // p is needed on the block's own rows only: A p = A z + beta A p_old
    // takes the product of z alone (its halo was published before the r.z
    // barrier), and p itself is never exchanged.  The rounding of the
    // recurrence is damped by beta < 1 from one iteration to the next.
    double beta = 0.0;
    for (int i = 0; rr > itol2 && rr > 0.0 && it < a.max_iter &&
                    !(a.inner_max > 0 && i >= a.inner_max);
         ++i) {
        stage_halo(s_z, (const float *)a.z32, a, g);
        __syncthreads();
        float b32 = (float)beta;
        DF pap[1] = {{0.f, 0.f}}, sr = {0.f, 0.f}, sq = {0.f, 0.f};
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            if (!t.ok[k])
                continue;
            float az = 0.f;
#pragma unroll 4
            for (int c = 0; c < t.wd[k]; ++c) {
                int lc = m.LC[t.le[k] + c * 32];
                az += m.VAL[t.le[k] + c * 32] * s_z[lc];
            }
            p[k] = z[k] + b32 * p[k];
            ap[k] = az + b32 * ap[k];
            df_add_prod(pap[0], p[k], ap[k]);
            if (coarse_ride && m.dinv[k] != 0.f) {
                df_add(sr, rv[k]);
                df_add(sq, ap[k]);
            }
        }
        double pt2[2];
        double z0 = 0.0;
        if (coarse_ride) {
            double o4[4];
            if (!grid_sum_pap_coarse(pap[0], sr, sq, set, a, rz, o4))
                return false;
            pt2[1] = o4[1];
            z0 = o4[2] - o4[1] * o4[3];
        } else if (!grid_sum_df<1, 2, RB>(pap, set, a, pt2,
                                          [rz](double *q) { q[1] = rz / q[0]; })) {
            return false;
        }
        set ^= 1;
        float a32 = (float)pt2[1];
        DF acc2[2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            if (!t.ok[k])
                continue;
            d[k] = d[k] + a32 * p[k];
            rv[k] = rv[k] - a32 * ap[k];
        }
        if (!apply_precond<RPT, float, true>(t, a, g, m.LC, m.VAL, m.dinv, rv, z, s_d0, s_d1,
                                       a.d32_0, a.d32_1, coarse_ride, z0))
            return false;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            if (!t.ok[k])
                continue;
            s_z[t.o[k]] = z[k];
            a.z32[t.row[k]] = z[k];
            df_add_prod(acc2[0], rv[k], z[k]);
            df_add_prod(acc2[1], rv[k], rv[k]);
        }
        double t3[3];
        if (!grid_sum_df<2, 3, RB>(acc2, set, a, t3,
                                  [rz](double *q) { q[2] = q[0] / rz; }))
            return false;
        set ^= 1;
        beta = t3[2];
        rz = t3[0];
        rr = t3[1];
        ++it;
    }
    return true;
}

// The standard CG with one grid barrier fewer per iteration (a global
// Chebyshev polynomial of degree k >= 2: k barriers instead of k + 1).  The
// new preconditioned residual z' = M^-1 (r - alpha A p) is computed afresh
// as in the standard form; only the polynomial's first step, which is local,
// is split by linearity: each block publishes D^-1 r / theta and
// D^-1 A p / theta (and, with the coarse correction, its sums of r and of
// A p) before alpha is known, the block partials of p.Ap cross the same
// barrier, and after it every block forms alpha and combines the staged
// halves, d_1 = D^-1 r / theta - alpha D^-1 A p / theta, own rows and halo
// alike.  The polynomial then continues from d_1 with its remaining
// barriers.  Nothing is carried by recurrence beyond what the standard form
// carries (r and p), so the rounding is that of the standard form.
template <int RPT>
__device__ bool inner_merged(const Rows<RPT> &t, const In32<RPT> &m, const PcgArgs &a,
                             const Seg &g, float (&rv)[RPT], float (&d)[RPT], float *s_z,
                             float *s_p0, float *s_p1, float *s_d0, float *s_d1, double itol,
                             int &set, int &it)
{
    float z[RPT], p[RPT], ap[RPT];
    DF acc[2] = {{0.f, 0.f}, {0.f, 0.f}};
    double tot[2];
    if (!apply_precond<RPT, float>(t, a, g, m.LC, m.VAL, m.dinv, rv, z, s_d0, s_d1, a.d32_0,
                                   a.d32_1))
        return false;
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        p[k] = ap[k] = 0.f;
        if (!t.ok[k])
            continue;
        s_z[t.o[k]] = z[k];
        s_p0[t.o[k]] = 0.f;
        a.z32[t.row[k]] = z[k];
        a.p32_0[t.row[k]] = 0.f;
        df_add_prod(acc[0], rv[k], z[k]);
        df_add_prod(acc[1], rv[k], rv[k]);
    }
    if (!grid_sum_df<2, 2, RB>(acc, set, a, tot, NoFinish()))
        return false;
    set ^= 1;
    double rz = tot[0], rr = tot[1];
    const double itol2 = itol * itol * rr;
    const bool coarse = a.cheb_local == 3 && a.coarse_inv;
    const float inv_theta = a.cheb_inv_thetaf;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double beta = 0.0;
    int cur = 0;
    for (int i = 0; rr > itol2 && rr > 0.0 && it < a.max_iter &&
                    !(a.inner_max > 0 && i >= a.inner_max);
         ++i) {
        float *sp_old = cur ? s_p1 : s_p0;
        float *sp_new = cur ? s_p0 : s_p1;
        const float *gp_old = cur ? a.p32_1 : a.p32_0;
        float *gp_new = cur ? a.p32_0 : a.p32_1;
        stage_halo(s_z, (const float *)a.z32, a, g);
        stage_halo(sp_old, gp_old, a, g);
        __syncthreads();
        const float b32 = (float)beta;
        DF pap = {0.f, 0.f}, sr = {0.f, 0.f}, sq = {0.f, 0.f};
        float dr[RPT], dq[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            dr[k] = dq[k] = 0.f;
            if (!t.ok[k])
                continue;
            float sum = 0.f;
#pragma unroll 4
            for (int c = 0; c < t.wd[k]; ++c) {
                int lc = m.LC[t.le[k] + c * 32];
                sum += m.VAL[t.le[k] + c * 32] * (s_z[lc] + b32 * sp_old[lc]);
            }
            p[k] = z[k] + b32 * p[k];
            ap[k] = sum;
            sp_new[t.o[k]] = p[k];
            gp_new[t.row[k]] = p[k];
            df_add_prod(pap, p[k], sum);
            // the first polynomial step of r and of A p, side by side
            dr[k] = m.dinv[k] * rv[k] * inv_theta;
            dq[k] = m.dinv[k] * sum * inv_theta;
            a.d32_1[t.row[k]] = dr[k];
            a.ap32[t.row[k]] = dq[k];
            if (m.dinv[k] != 0.f) {
                df_add(sr, rv[k]);
                df_add(sq, sum);
            }
        }
        const double pap_w = df_warp_sum(pap);
        if (lane == 0)
            ride_part()[wid] = pap_w;
        Ride c_r, c_q;
        if (coarse) {
            const double sr_w = df_warp_sum(sr), sq_w = df_warp_sum(sq);
            if (lane == 0) {
                coarse_part()[wid] = sr_w;
                coarse_part2()[wid] = sq_w;
            }
            c_r = Ride{coarse_part(), RW, a.coarse_r + blockIdx.x};
            c_q = Ride{coarse_part2(), RW, a.coarse_r + gridDim.x + blockIdx.x};
        }
        if (!grid_sync(a, Ride{ride_part(), RW,
                               a.partials + ((size_t)set * gridDim.x + blockIdx.x) * 4},
                       c_r, c_q))
            return false;
        ride_gather(a, set);            // warp 1: p.Ap
        if (coarse)
            coarse_apply_pair(a);       // warp 0
        set ^= 1;
        stage_halo(s_d1, (const float *)a.d32_1, a, g);
        stage_halo(s_d0, (const float *)a.ap32, a, g);
        __syncthreads();
        const double alpha = rz / ride_part()[RW];
        const float a32 = (float)alpha;
        for (int h = threadIdx.x; h < g.nh; h += blockDim.x)
            s_d1[g.nrows + h] = s_d1[g.nrows + h] - a32 * s_d0[g.nrows + h];
        float rc[RPT], dc[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            rc[k] = dc[k] = z[k] = 0.f;
            if (!t.ok[k])
                continue;
            d[k] = d[k] + a32 * p[k];
            rv[k] = rv[k] - a32 * ap[k];
            rc[k] = rv[k];
            dc[k] = dr[k] - a32 * dq[k];
            s_d1[t.o[k]] = dc[k];
            z[k] = dc[k];
        }
        __syncthreads();
        for (int j = 1; j < a.cheb_degree; ++j) {
            float *s_dj = (j & 1) ? s_d1 : s_d0;
            float *g_dj = (j & 1) ? a.d32_1 : a.d32_0;
            if (j > 1 && a.dtag[0]) {
                if (!tagged_exchange<RPT>(t, a, g, s_dj, dc))
                    return false;
            } else if (j > 1) {
#pragma unroll
                for (int k = 0; k < RPT; ++k) {
                    if (!t.ok[k])
                        continue;
                    s_dj[t.o[k]] = dc[k];
                    g_dj[t.row[k]] = dc[k];
                }
                if (!grid_sync(a))
                    return false;
                stage_halo(s_dj, (const float *)g_dj, a, g);
                __syncthreads();
            }
            cheb_update<RPT, float>(t, a, m.LC, m.VAL, m.dinv, s_dj, j, rc, dc);
#pragma unroll
            for (int k = 0; k < RPT; ++k)
                z[k] = z[k] + dc[k];
        }
        if (coarse) {
            const float z0 = (float)(coarse_z0_pair()[0] - alpha * coarse_z0_pair()[1]);
#pragma unroll
            for (int k = 0; k < RPT; ++k)
                if (t.ok[k] && m.dinv[k] != 0.f)
                    z[k] = z[k] + z0;
        }
        DF acc2[2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            if (!t.ok[k])
                continue;
            s_z[t.o[k]] = z[k];
            a.z32[t.row[k]] = z[k];
            df_add_prod(acc2[0], rv[k], z[k]);
            df_add_prod(acc2[1], rv[k], rv[k]);
        }
        double t3[3];
        if (!grid_sum_df<2, 3, RB>(acc2, set, a, t3,
                                  [rz](double *q3) { q3[2] = q3[0] / rz; }))
            return false;
        set ^= 1;
        beta = t3[2];
        rz = t3[0];
        rr = t3[1];
        ++it;
        cur ^= 1;
    }
    return true;
}

// The one reduction of an iteration of the one-reduction CG (resident
// solver, one system): block values gamma = r.u, delta = (A u).u, rr = r.r
// and, with the coarse correction, the block sums of r, w = A u and the
// previous s (rows with a nonzero diagonal), in a.part8.  After the barrier
// warp 0 totals the three dot products and lane 0 forms alpha and beta
// (Chronopoulos & Gear; i == 0: beta = 0, alpha = gamma / delta), while warp
// 1 forms this block's rows of A0^-1 applied to the three coarse vectors.
// out: gamma, delta, rr, (A0^-1 R0 r)_b, (A0^-1 R0 w)_b, (A0^-1 R0 s)_b,
// alpha, beta.
__device__ bool grid_sum_single(const DF (&v)[3], const DF (&cs)[3], bool coarse, int set,
                                const PcgArgs &a, int i, double gamma_old, double alpha_old,
                                double (&out)[8])
{
    double *vals = reduction_buffer();
    double *res = vals + 3 * 512 - 4;   // 8 results after 6 x RW block values
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nv = coarse ? 6 : 3;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        if (k >= nv)
            break;
        const double x = df_warp_sum(k < 3 ? v[k] : cs[k - 3]);
        if (lane == 0)
            vals[k * RW + wid] = x;
    }
    __syncthreads();
    const size_t G = gridDim.x;
    if (wid == 0) {
        for (int k = 0; k < nv; ++k) {
            double x = lane < RW ? vals[k * RW + lane] : 0.0;
            x = warp_sum(x);
            if (lane == 0)
                a.part8[((size_t)set * G + blockIdx.x) * 8 + k] = x;
        }
    }
    if (!grid_sync(a))
        return false;
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double x = 0.0;
            for (size_t b = lane; b < G; b += 32)
                x += __ldcg(a.part8 + ((size_t)set * G + b) * 8 + k);
            x = warp_sum(x);
            if (lane == 0)
                res[k] = x;
        }
        if (lane == 0) {
            const double gamma = res[0], delta = res[1];
            double alpha, beta;
            if (i == 0) {
                beta = 0.0;
                alpha = gamma / delta;
            } else {
                beta = gamma / gamma_old;
                alpha = gamma / (delta - beta * gamma / alpha_old);
            }
            res[6] = alpha;
            res[7] = beta;
        }
    } else if (wid == 1 && coarse) {
        const float *row = a.coarse_inv + (size_t)blockIdx.x * G;
        double v0 = 0.0, v1 = 0.0, v2 = 0.0;
        for (size_t c = lane; c < G; c += 32) {
            const double ic = (double)row[c];
            const double *pc = a.part8 + ((size_t)set * G + c) * 8;
            v0 += ic * __ldcg(pc + 3);
            v1 += ic * __ldcg(pc + 4);
            v2 += ic * __ldcg(pc + 5);
        }
        v0 = warp_sum(v0);
        v1 = warp_sum(v1);
        v2 = warp_sum(v2);
        if (lane == 0) {
            res[3] = v0;
            res[4] = v1;
            res[5] = v2;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 8; ++k)
        out[k] = (k >= 3 && k < 6 && !coarse) ? 0.0 : res[k];
    return true;
}

// Chronopoulos & Gear's CG (one reduction per iteration; Comput. Appl.
// Math. 25, 1989), preconditioned: with u = M^-1 r and w = A u,
// gamma = r.u, delta = w.u, beta = gamma / gamma_old,
// alpha = gamma / (delta - beta gamma / alpha_old), p = u + beta p,
// s = w + beta s (= A p), x += alpha p, r -= alpha s.  The coarse correction
// of the next preconditioner application rides on the same reduction
// (R0 r' = R0 r - alpha (R0 w + beta R0 s_old)), so the polynomial and the
// product A u exchange their halos through tagged words only: one grid
// barrier per iteration.  Same arithmetic in exact arithmetic as the
// standard form; s carries rounding like the A p recurrence of the standard
// form (damped by beta < 1).
template <int RPT>
__device__ bool inner_single(const Rows<RPT> &t, const In32<RPT> &m, const PcgArgs &a,
                             const Seg &g, float (&rv)[RPT], float (&d)[RPT], float *s_z,
                             float *s_d0, float *s_d1, double itol, int &set, int &it)
{
    const bool coarse = a.cheb_local == 3 && a.coarse_inv;
    float u[RPT], p[RPT], sv[RPT];
    if (!apply_precond<RPT, float>(t, a, g, m.LC, m.VAL, m.dinv, rv, u, s_d0, s_d1, a.d32_0,
                                   a.d32_1))
        return false;
#pragma unroll
    for (int k = 0; k < RPT; ++k)
        p[k] = sv[k] = 0.f;
    double gamma_old = 0.0, alpha_old = 0.0, itol2 = 0.0;
    for (int i = 0;; ++i) {
        if (!tagged_exchange<RPT>(t, a, g, s_z, u))
            return false;
        DF acc[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        DF cs[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        float w[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            w[k] = 0.f;
            if (!t.ok[k])
                continue;
            float sum = 0.f;
#pragma unroll 4
            for (int c = 0; c < t.wd[k]; ++c) {
                int lc = m.LC[t.le[k] + c * 32];
                sum += m.VAL[t.le[k] + c * 32] * s_z[lc];
            }
            w[k] = sum;
            df_add_prod(acc[0], rv[k], u[k]);
            df_add_prod(acc[1], sum, u[k]);
            df_add_prod(acc[2], rv[k], rv[k]);
            if (coarse && m.dinv[k] != 0.f) {
                df_add(cs[0], rv[k]);
                df_add(cs[1], sum);
                df_add(cs[2], sv[k]);
            }
        }
        double o[8];
        if (!grid_sum_single(acc, cs, coarse, set, a, i, gamma_old, alpha_old, o))
            return false;
        set ^= 1;
        const double rr = o[2];
        if (i == 0)
            itol2 = itol * itol * rr;
        if (!(rr > itol2 && rr > 0.0 && it < a.max_iter && !(a.inner_max > 0 && i >= a.inner_max)))
            break;
        const double alpha = o[6], beta = o[7];
        const float a32 = (float)alpha, b32 = (float)beta;
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            if (!t.ok[k])
                continue;
            p[k] = u[k] + b32 * p[k];
            sv[k] = w[k] + b32 * sv[k];
            d[k] = d[k] + a32 * p[k];
            rv[k] = rv[k] - a32 * sv[k];
        }
        const double z0 = coarse ? o[3] - alpha * (o[4] + beta * o[5]) : 0.0;
        if (!apply_precond<RPT, float>(t, a, g, m.LC, m.VAL, m.dinv, rv, u, s_d0, s_d1,
                                       a.d32_0, a.d32_1, coarse, z0))
            return false;
        gamma_old = o[0];
        alpha_old = alpha;
        ++it;
    }
    return true;
}

template <int RPT>
__device__ bool inner_pipelined(const Rows<RPT> &t, const In32<RPT> &m, const PcgArgs &a,
                                const Seg &g, float (&rv)[RPT], float (&d)[RPT], float *s_m0,
                                float *s_m1, int &set, int &it)
{
    float u[RPT], wv[RPT], zz[RPT], q[RPT], sv[RPT], p[RPT], mm[RPT];
    float *gm[2] = {a.z32, a.p32_0};
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        u[k] = m.dinv[k] * rv[k];
        wv[k] = zz[k] = q[k] = sv[k] = p[k] = mm[k] = 0.f;
        if (!t.ok[k])
            continue;
        s_m0[t.o[k]] = u[k];
        gm[0][t.row[k]] = u[k];
    }
    if (!grid_sync(a))
        return false;
    stage_halo(s_m0, (const float *)gm[0], a, g);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < RPT; ++k)
        if (t.ok[k])
            wv[k] = spmv_local<RPT, float, float, float>(t, k, m.LC, m.VAL, false, s_m0);
    double gamma_old = 1.0, alpha_old = 1.0, rr0 = -1.0;
    int cur = 0;
    for (int i = 0;; ++i) {
        cur ^= 1;
        float *s_m = cur ? s_m1 : s_m0;
        float *g_m = gm[cur];
        double dots[3] = {0.0, 0.0, 0.0}, dt3[3];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            if (!t.ok[k])
                continue;
            mm[k] = m.dinv[k] * wv[k];
            s_m[t.o[k]] = mm[k];
            g_m[t.row[k]] = mm[k];
            dots[0] += (double)rv[k] * (double)u[k];
            dots[1] += (double)wv[k] * (double)u[k];
            dots[2] += (double)rv[k] * (double)rv[k];
        }
        if (!grid_sum<3, RB>(dots, set, a, dt3))
            return false;
        set ^= 1;
        double gamma = dt3[0], delta = dt3[1], rr = dt3[2];
        if (rr0 < 0.0)
            rr0 = rr;
        if (rr <= a.inner_rtol * a.inner_rtol * rr0 || it >= a.max_iter || rr == 0.0 ||
            (a.inner_max > 0 && i >= a.inner_max))
            return true;
        double beta = i == 0 ? 0.0 : gamma / gamma_old;
        double alpha = i == 0 ? gamma / delta : gamma / (delta - beta * gamma / alpha_old);
        float b32 = (float)beta, a32 = (float)alpha;
        stage_halo(s_m, (const float *)g_m, a, g);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            if (!t.ok[k])
                continue;
            float n = spmv_local<RPT, float, float, float>(t, k, m.LC, m.VAL, false, s_m);
            zz[k] = n + b32 * zz[k];
            q[k] = mm[k] + b32 * q[k];
            sv[k] = wv[k] + b32 * sv[k];
            p[k] = u[k] + b32 * p[k];
            d[k] = d[k] + a32 * p[k];
            rv[k] = rv[k] - a32 * sv[k];
            u[k] = u[k] - a32 * q[k];
            wv[k] = wv[k] - a32 * zz[k];
        }
        gamma_old = gamma;
        alpha_old = alpha;
        ++it;
    }
}

template <int RPT, bool SM, bool PIPE>
__device__ __forceinline__ void pcg32ir_res(const PcgArgs &a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Seg g = block_seg(a);
    float *s_val = (float *)smem;
    int *s_lc = (int *)(smem + (SM ? a.max_chunk * 4 : 0));
    size_t off = SM ? (size_t)a.max_chunk * 8 : 0;
    off = (off + 15) & ~(size_t)15;
    double *s_x = (double *)(smem + off);
    float *s_a = (float *)(s_x + a.max_local);
    float *s_b = s_a + a.max_local;
    float *s_c = s_b + a.max_local;
    float *s_d0 = s_c + a.max_local;
    float *s_d1 = s_d0 + a.max_local;
    if (SM) {
        int e1 = a.slice_ptr[g.s1];
        stage_chunk(s_val, a.val32, g.e0, e1);
        stage_chunk(s_lc, a.lcol, g.e0, e1);
    }
    In32<RPT> m;
    m.LC = SM ? s_lc : a.lcol;
    m.VAL = SM ? s_val : a.val32;
    Rows<RPT> t;
    init_rows<RPT, SM>(t, a, g);
    double x[RPT], f[RPT], r64[RPT];
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        x[k] = f[k] = r64[k] = 0.0;
        m.dinv[k] = 0.f;
        if (!t.ok[k])
            continue;
        x[k] = a.x[t.row[k]];
        f[k] = rhs_entry(a, t.row[k]);
        m.dinv[k] = a.dinv32[t.row[k]];
        s_x[t.o[k]] = x[k];
    }
    int set = 0, it = 0, outer = 0, status = 0;
    double ff = -1.0, rr64 = 0.0;
    // the merged form needs a grid barrier inside the preconditioner
    const bool merged = a.variant == PIC_PCG_MERGED && a.cheb_degree >= 2 &&
                        (a.cheb_local == 0 || a.cheb_local == 3);
    // the one-reduction form needs the tagged exchange (its products take no
    // grid barrier of their own)
    const bool single = a.variant == PIC_PCG_SINGLE && a.cheb_degree >= 2 &&
                        (a.cheb_local == 0 || a.cheb_local == 3) && a.dtag[0];
    for (;;) {
        // FP64 residual r = f - M x (own x in s_x; halo of x staged)
        stage_halo(s_x, (const double *)a.x, a, g);
        __syncthreads();
        double acc[2] = {0.0, 0.0}, tot[2];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            if (!t.ok[k])
                continue;
            double axv = spmv_local<RPT, double, double, double>(t, k, m.LC, a.val64, true, s_x);
            r64[k] = f[k] - axv;
            acc[0] += r64[k] * r64[k];
            acc[1] += f[k] * f[k];
        }
        if (!grid_sum<2, RB>(acc, set, a, tot))
            return;
        set ^= 1;
        rr64 = tot[0];
        if (ff < 0.0)
            ff = tot[1];
        if (ff == 0.0) {
#pragma unroll
            for (int k = 0; k < RPT; ++k)
                x[k] = 0.0;
            rr64 = 0.0;
            ff = 1.0;
            break;
        }
        if (sqrt(rr64) <= a.rtol * sqrt(ff))
            break;
        if (it >= a.max_iter) {
            status = PIC_ERR_NOT_CONVERGED;
            break;
        }
        const double sc = refinement_scale(rr64), inv_sc = 1.0 / sc;
        if (sc == 0.0) {
            status = PIC_ERR_NOT_CONVERGED;
            break;
        }
        float rv[RPT], d[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            rv[k] = (float)(r64[k] * inv_sc);
            d[k] = 0.f;
        }
        // ask the FP32 solve for what the FP64 target still needs (with a
        // margin), but never for more than ir_inner_rtol in one refinement
        double itol = 0.5 * a.rtol * sqrt(ff) / sqrt(rr64);
        if (itol < a.inner_rtol)
            itol = a.inner_rtol;
        const int it0 = it;
        bool good;
        if constexpr (PIPE)
            good = inner_pipelined<RPT>(t, m, a, g, rv, d, s_a, s_b, set, it);
        else
            good = single ? inner_single<RPT>(t, m, a, g, rv, d, s_a, s_d0, s_d1, itol, set, it)
                   : merged ? inner_merged<RPT>(t, m, a, g, rv, d, s_a, s_b, s_c, s_d0, s_d1,
                                                itol, set, it)
                            : inner_standard<RPT>(t, m, a, g, rv, d, s_a, s_b, s_c, s_d0, s_d1,
                                                  itol, set, it);
        if (!good)
            return;
        if (it == it0) {   // no inner iteration: no progress possible
            status = PIC_ERR_NOT_CONVERGED;
            break;
        }
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            if (!t.ok[k])
                continue;
            x[k] = x[k] + sc * (double)d[k];
            s_x[t.o[k]] = x[k];
            a.x[t.row[k]] = x[k];
        }
        if (!grid_sync(a))
            return;
        ++outer;
    }
#pragma unroll
    for (int k = 0; k < RPT; ++k) {
        if (!t.ok[k])
            continue;
        a.x[t.row[k]] = x[k];
        int node = a.dof_node[t.row[k]];
        if (node >= 0)
            a.phi[node] = x[k];
    }
    finish(a, it, sqrt(rr64) / sqrt(ff), status, outer);
}

template <int RPT, bool SM, bool PIPE>
__global__ void __launch_bounds__(RB, 1) k_pcg32ir_res(PcgArgs a)
{
    grid_sync_init();
    pcg32ir_res<RPT, SM, PIPE>(a);
    // the next launch's tags take a new epoch, whichever way this one ended
    // (every block has read the epoch before its first grid barrier)
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.epoch)
        atomicInc(a.epoch, 254u);   // 0, 1, ..., 254, 0, ...: consecutive epochs differ
}

template <int RPT, bool SM> const void *res_kernel(int precision, int variant)
{
    if (precision == PIC_PREC_FP64)
        return (const void *)k_pcg64_res<RPT, SM>;
    return variant == PIC_PCG_PIPELINED ? (const void *)k_pcg32ir_res<RPT, SM, true>
                                        : (const void *)k_pcg32ir_res<RPT, SM, false>;
}

const void *pick_resident(int precision, int variant, int rpt, bool sm)
{
    switch (rpt) {
    case 1: return sm ? res_kernel<1, true>(precision, variant) : res_kernel<1, false>(precision, variant);
    case 2: return sm ? res_kernel<2, true>(precision, variant) : res_kernel<2, false>(precision, variant);
    case 4: return sm ? res_kernel<4, true>(precision, variant) : res_kernel<4, false>(precision, variant);
    default: return sm ? res_kernel<8, true>(precision, variant) : res_kernel<8, false>(precision, variant);
    }
}

constexpr size_t SMEM_LIMIT = 200 * 1024;   // + static reduction buffers

// The dynamic shared memory a kernel may take is a property of the function,
// shared by every context: only ever raise it, so that a plan made for a
// smaller system never breaks the launch of a larger one.
static cudaError_t raise_smem_attr(const void *fn, size_t bytes)
{
    static std::mutex mu;
    static std::map<const void *, size_t> set;
    std::lock_guard<std::mutex> lk(mu);
    size_t &cur = set[fn];
    if (bytes <= cur)
        return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e == cudaSuccess)
        cur = bytes;
    return e;
}

// Row ownership, local column indices and halos of the resident kernels.
static void build_halo(const int *slice_ptr, const int *col, int n_slices, int G, PcgHalo *h,
                       int *max_local, long long *max_chunk, int *symmetric)
{
    // reads[b * G + o]: block b reads rows of block o
    std::vector<char> reads((size_t)G * G, 0);
    auto owner = [&](int j) {
        const long long sl = j / 32;
        long long b = (sl * G) / n_slices;   // first guess, then adjust to the split
        while (b > 0 && (b * n_slices) / G > sl)
            --b;
        while (b + 1 < G && ((b + 1) * n_slices) / G <= sl)
            ++b;
        return (int)b;
    };
    h->lcol.assign((size_t)slice_ptr[n_slices], 0);
    h->halo_ptr.assign((size_t)G + 1, 0);
    h->halo_idx.clear();
    *max_local = 0;
    *max_chunk = 0;
    std::vector<int> ext;
    for (long long b = 0; b < G; ++b) {
        int s0 = (int)((b * n_slices) / G), s1 = (int)(((b + 1) * n_slices) / G);
        int row0 = 32 * s0, nrows = 32 * (s1 - s0);
        int e0 = slice_ptr[s0], e1 = slice_ptr[s1];
        ext.clear();
        for (int e = e0; e < e1; ++e) {
            int j = col[e];
            if (j < row0 || j >= row0 + nrows)
                ext.push_back(j);
        }
        std::sort(ext.begin(), ext.end());
        ext.erase(std::unique(ext.begin(), ext.end()), ext.end());
        for (int e = e0; e < e1; ++e) {
            int j = col[e];
            h->lcol[e] = (j >= row0 && j < row0 + nrows)
                             ? j - row0
                             : nrows + (int)(std::lower_bound(ext.begin(), ext.end(), j) - ext.begin());
        }
        for (int j : ext)
            reads[(size_t)b * G + owner(j)] = 1;
        h->halo_idx.insert(h->halo_idx.end(), ext.begin(), ext.end());
        h->halo_ptr[b + 1] = (int)h->halo_idx.size();
        *max_local = std::max(*max_local, nrows + (int)ext.size());
        *max_chunk = std::max(*max_chunk, (long long)(e1 - e0));
    }
    *symmetric = 1;
    for (int b = 0; b < G && *symmetric; ++b)
        for (int o = 0; o < G; ++o)
            if (reads[(size_t)b * G + o] != reads[(size_t)o * G + b]) {
                *symmetric = 0;
                break;
            }
}

int pcg_max_group_blocks(int precision, int num_sms)
{
    const void *fn = precision == PIC_PREC_FP64 ? (const void *)k_pcg64 : (const void *)k_pcg32ir;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PCG_BLOCK, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * num_sms;
}

cudaError_t pcg_plan(const int *slice_ptr, const int *col, int n_slices, int num_sms,
                     int precision, int variant, int n_sys, const int *grp_slices,
                     const double *grp_work, int blocks_per_sm, PcgLaunch *plan, PcgHalo *halo)
{
    *plan = PcgLaunch{};
    if (n_sys > 1) {
        // a batch: the general kernels, each system on its own group of
        // blocks.  A group's time is its iterations x its slices / its
        // blocks, so blocks in proportion to slices x iterations (grp_work,
        // from the previous solve) make the groups finish together; without
        // that information, in proportion to the slices.
        const void *fn = precision == PIC_PREC_FP64 ? (const void *)k_pcg64 : (const void *)k_pcg32ir;
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PCG_BLOCK, 0);
        if (e != cudaSuccess)
            return e;
        if (blocks_per_sm > 0 && blocks_per_sm < per_sm)
            per_sm = blocks_per_sm;
        int max_blocks = per_sm * num_sms;
        if (per_sm < 1 || n_sys > max_blocks)
            return cudaErrorInvalidConfiguration;
        std::vector<int> nb((size_t)n_sys, 1);
        int spare = max_blocks - n_sys;
        auto work = [&](int g) {
            double sl = (double)(grp_slices[g + 1] - grp_slices[g]);
            return grp_work ? grp_work[g] : sl;
        };
        double tot = 0.0;
        for (int g = 0; g < n_sys; ++g)
            tot += work(g);
        int used = 0;
        for (int g = 0; g < n_sys; ++g) {
            long long sl = grp_slices[g + 1] - grp_slices[g];
            int want = (int)((double)spare * work(g) / (tot > 0.0 ? tot : 1.0));
            int cap = (int)((sl + PCG_WARPS - 1) / PCG_WARPS);  // at most a slice per warp
            want = std::min(want, std::max(0, cap - 1));
            nb[g] += want;
            used += want;
        }
        (void)used;
        halo->grp.assign(4 * (size_t)n_sys, 0);
        halo->blk_grp.clear();
        int b = 0;
        for (int g = 0; g < n_sys; ++g) {
            halo->grp[4 * g + 0] = grp_slices[g];
            halo->grp[4 * g + 1] = grp_slices[g + 1];
            halo->grp[4 * g + 2] = b;
            halo->grp[4 * g + 3] = nb[g];
            for (int k = 0; k < nb[g]; ++k)
                halo->blk_grp.push_back(g);
            b += nb[g];
        }
        plan->grid = b;
        plan->block = PCG_BLOCK;
        plan->n_groups = n_sys;
        return cudaSuccess;
    }
    // resident: one block per SM (fewer for small problems), rows in registers
    int G = (n_slices + RW - 1) / RW;
    if (G > num_sms)
        G = num_sms;
    if (G < 1)
        G = 1;
    int max_sl = (n_slices + G - 1) / G;
    int need = (max_sl + RW - 1) / RW;
    int rpt = need <= 1 ? 1 : need <= 2 ? 2 : need <= 4 ? 4 : need <= 8 ? 8 : 0;
    if (rpt) {
        int max_local = 0;
        long long chunk = 0;
        int symmetric = 0;
        build_halo(slice_ptr, col, n_slices, G, halo, &max_local, &chunk, &symmetric);
        bool fp64 = precision == PIC_PREC_FP64;
        size_t vec = fp64 ? (size_t)max_local * 8 * 5 : (size_t)max_local * (8 + 4 * 5);
        size_t mat = (size_t)chunk * (fp64 ? 12 : 8);
        mat = (mat + 15) & ~(size_t)15;
        bool sm = mat + vec <= SMEM_LIMIT;
        size_t bytes = (sm ? mat : 0) + vec;
        if (bytes <= SMEM_LIMIT) {
            const void *fn = pick_resident(precision, variant, rpt, sm);
            cudaError_t e = raise_smem_attr(fn, bytes);
            int per_sm = 0;
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, RB, bytes);
            if (e != cudaSuccess)
                return e;
            if (per_sm >= 1) {
                plan->grid = G;
                plan->block = RB;
                plan->resident = 1;
                plan->rpt = rpt;
                plan->smem_matrix = sm ? 1 : 0;
                plan->smem_bytes = bytes;
                plan->max_rows = 32 * max_sl;
                plan->max_chunk = chunk;
                plan->max_local = max_local;
                plan->halo_symmetric = symmetric;
                return cudaSuccess;
            }
        }
        *halo = PcgHalo{};
    }
    // general path: vectors in global memory, any size
    plan->grid = pcg_general_grid(precision, n_slices, num_sms, blocks_per_sm);
    if (plan->grid < 1)
        return cudaErrorInvalidConfiguration;
    plan->block = PCG_BLOCK;
    return cudaSuccess;
}

int pcg_general_grid(int precision, int n_slices, int num_sms, int blocks_per_sm)
{
    const int max_blocks = pcg_max_group_blocks(precision, num_sms);
    if (max_blocks < 1)
        return 0;
    // as many blocks as fit by default: the products are bound by memory
    // latency, and every resident warp adds loads in flight (on the 7.9M-tet
    // tip 4 blocks per SM solve in 0.67x the time of 2, barriers included)
    const int want = (n_slices + PCG_WARPS - 1) / PCG_WARPS;   // one slice per warp
    const int cap = blocks_per_sm > 0 ? blocks_per_sm * num_sms : max_blocks;
    int grid = want < cap ? (want < 1 ? 1 : want) : cap;
    return grid < max_blocks ? grid : max_blocks;
}

// dynamic shared memory a resident block may take with the multigrid arrays
// (the static reduction buffers come on top; 227 KB per block in all)
constexpr size_t SMEM_LIMIT_MG = 212 * 1024;

cudaError_t pcg_plan_mg(PcgLaunch *plan, int precision, int variant, size_t extra, bool *ok)
{
    *ok = false;
    if (!plan->resident || plan->rpt > 4)     // the V-cycle is compiled for up to 4 rows a thread
        return cudaSuccess;
    const size_t off = (plan->smem_bytes + 15) & ~(size_t)15;
    const size_t bytes = off + extra;
    if (bytes > SMEM_LIMIT_MG)
        return cudaSuccess;
    const void *fn = pick_resident(precision, variant, plan->rpt, plan->smem_matrix != 0);
    cudaError_t e = raise_smem_attr(fn, bytes);
    int per_sm = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, RB, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cudaSuccess;
    }
    if (per_sm < 1)
        return cudaSuccess;
    plan->mg_off = off;
    plan->smem_bytes = bytes;
    *ok = true;
    return cudaSuccess;
}

// Cooperative launch (all blocks co-resident, which the grid barrier needs)
// through the extensible launch API, which stream capture records as a
// cooperative kernel node.
cudaError_t launch_pcg(cudaStream_t s, const PcgLaunch &plan, const PcgArgs &a)
{
    void *args[] = {(void *)&a};
    const void *fn;
    size_t smem = 0;
    if (plan.resident) {
        fn = pick_resident(a.precision, a.variant, plan.rpt, plan.smem_matrix != 0);
        smem = plan.smem_bytes;
    } else {
        fn = a.precision == PIC_PREC_FP64 ? (const void *)k_pcg64 : (const void *)k_pcg32ir;
    }
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(plan.grid);
    cfg.blockDim = dim3(plan.block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace pf
