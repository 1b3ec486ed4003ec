// adjoint.cu -- mesh-side kernels of the reverse pass of pic_adjoint: the
// transpose of the field (E_t = -sum_i Phi_i grad N_i, Sec. II.B.2), the
// gather of the adjoint solve's right-hand side onto the solver rows, and the
// derivative of the Neumann load f_N = E0 A / 3 (eq. poisson_rhs) with
// respect to each replica's E0.  The per-SP part of the reverse pass lives in
// particles.cu next to the forward step it mirrors.
#include "common.cuh"

namespace pf {

// phibar[v_i] += -Ebar_t . grad N_i for the four nodes of tetrahedron t
__global__ void k_field_adjoint(int T, const TetRec64 *__restrict__ rec,
                                const int4 *__restrict__ tet, const double *__restrict__ Ebar,
                                double *phibar)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T)
        return;
    const double e[3] = {Ebar[3 * (size_t)t], Ebar[3 * (size_t)t + 1], Ebar[3 * (size_t)t + 2]};
    if (e[0] == 0.0 && e[1] == 0.0 && e[2] == 0.0)
        return;
    const TetRec64 &r = rec[t];
    double g[4][3];
    for (int c = 0; c < 3; ++c) {
        g[1][c] = r.j[c];
        g[2][c] = r.j[3 + c];
        g[3][c] = r.j[6 + c];
        g[0][c] = -((g[1][c] + g[2][c]) + g[3][c]);
    }
    const int4 v4 = tet[t];
    const int v[4] = {v4.x, v4.y, v4.z, v4.w};
    for (int i = 0; i < 4; ++i)
        atomicAdd(phibar + v[i], -((e[0] * g[i][0] + e[1] * g[i][1]) + e[2] * g[i][2]));
}

__global__ void k_gather_rows(int n_rows, const int *__restrict__ dof_node,
                              const double *__restrict__ node_v, double *rows)
{
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n_rows)
        return;
    const int node = dof_node[row];
    rows[row] = node >= 0 ? node_v[node] : 0.0;
}

// One warp per 32-row slice (a slice never mixes replicas): warp sum, one
// atomic per slice.
__global__ void k_dE0(int n_rows, const double *__restrict__ x, const double *__restrict__ fN,
                      const int *__restrict__ rep_slice, int n_rep,
                      const double *__restrict__ E0_rep, double *gE0)
{
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    const int slice = row >> 5;
    if (slice * 32 >= n_rows)
        return;
    int lo = 0, hi = n_rep;   // replica r owns slices [rep_slice[r], rep_slice[r+1])
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (rep_slice[mid] <= slice)
            lo = mid;
        else
            hi = mid;
    }
    const double e0 = E0_rep[lo];
    double v = (row < n_rows && e0 != 0.0) ? x[row] * (fN[row] / e0) : 0.0;
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0)
        atomicAdd(gE0 + lo, v);
}

static inline unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

cudaError_t launch_field_adjoint(cudaStream_t s, int T, const TetRec64 *rec, const int4 *tet,
                                 const double *Ebar, double *phibar)
{
    if (T <= 0)
        return cudaSuccess;
    k_field_adjoint<<<blocks_for(T, 256), 256, 0, s>>>(T, rec, tet, Ebar, phibar);
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(cudaStream_t s, int n_rows, const int *dof_node,
                               const double *node_v, double *rows)
{
    if (n_rows <= 0)
        return cudaSuccess;
    k_gather_rows<<<blocks_for(n_rows, 256), 256, 0, s>>>(n_rows, dof_node, node_v, rows);
    return cudaGetLastError();
}

cudaError_t launch_dE0(cudaStream_t s, int n_rows, const double *x, const double *fN,
                       const int *rep_slice, int n_rep, const double *E0_rep, double *gE0)
{
    if (n_rows <= 0)
        return cudaSuccess;
    k_dE0<<<blocks_for(n_rows, 256), 256, 0, s>>>(n_rows, x, fN, rep_slice, n_rep, E0_rep, gE0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// stable compaction of an ordered push: exclusive prefix sum of the survivor
// flags in blocks of 1024 (warp scans, then the warp totals), a single-block
// scan of the block totals, then the moves
// ---------------------------------------------------------------------------
constexpr int SCAN_B = 1024;

__global__ void __launch_bounds__(SCAN_B) k_scan_local(long long n, int *dest, int *blk_sum)
{
    __shared__ int wsum[32];
    const long long i = blockIdx.x * (long long)SCAN_B + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int d = i < n ? dest[i] : 0;
    const int flag = d == 1 ? 1 : 0;
    int incl = flag;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += y;
    }
    if (lane == 31)
        wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int t = wsum[lane];
        int x = t;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o)
                x += y;
        }
        wsum[lane] = x - t;   // exclusive offset of each warp
        if (lane == 31)
            blk_sum[blockIdx.x] = x;
    }
    __syncthreads();
    if (i < n && flag)
        dest[i] = wsum[w] + incl - 1;   // survivor's position within the block
}

__global__ void __launch_bounds__(SCAN_B) k_scan_blocks(int nb, const int *blk_sum, int *blk_off,
                                                        int *total)
{
    __shared__ int wsum[32];
    __shared__ int carry;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0)
        carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += SCAN_B) {
        const int b = base + threadIdx.x;
        const int v = b < nb ? blk_sum[b] : 0;
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o)
                incl += y;
        }
        if (lane == 31)
            wsum[w] = incl;
        __syncthreads();
        if (w == 0) {
            int t = wsum[lane], x = t;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o)
                    x += y;
            }
            wsum[lane] = x - t;
        }
        __syncthreads();
        if (b < nb)
            blk_off[b] = carry + wsum[w] + incl - v;
        __syncthreads();
        if (threadIdx.x == SCAN_B - 1)
            carry += wsum[w] + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0)
        *total = carry;
}

// exclusive scan of int values, out[n] = total (scratch: 2 ceil(n/1024) + 2 ints)
__global__ void __launch_bounds__(SCAN_B) k_escan_local(long long n, const int *in, int *out,
                                                        int *blk_sum)
{
    __shared__ int wsum[32];
    const long long i = blockIdx.x * (long long)SCAN_B + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int v = i < n ? in[i] : 0;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += y;
    }
    if (lane == 31)
        wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int t = wsum[lane], x = t;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o)
                x += y;
        }
        wsum[lane] = x - t;
        if (lane == 31)
            blk_sum[blockIdx.x] = x;
    }
    __syncthreads();
    if (i < n)
        out[i] = wsum[w] + incl - v;
}

__global__ void k_escan_add(long long n, int *out, const int *blk_off, const int *total)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n)
        out[i] += blk_off[i / SCAN_B];
    if (i == 0)
        out[n] = *total;
}

cudaError_t launch_exclusive_scan(cudaStream_t s, long long n, const int *in, int *out,
                                  int *scratch)
{
    const int nb = (int)((n + SCAN_B - 1) / SCAN_B);
    int *blk_sum = scratch, *blk_off = scratch + nb + 1, *total = scratch + 2 * nb + 1;
    if (nb == 0)
        return cudaMemsetAsync(out, 0, sizeof(int), s);
    k_escan_local<<<nb, SCAN_B, 0, s>>>(n, in, out, blk_sum);
    k_scan_blocks<<<1, SCAN_B, 0, s>>>(nb, blk_sum, blk_off, total);
    k_escan_add<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, out, blk_off, total);
    return cudaGetLastError();
}

template <typename R>
__global__ void k_compact(long long n, int *dest, const int *blk_off, const int *total,
                          Particles<R> B, Particles<R> A, DevState *st, int a)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i == 0) {
        st->cnt[a] = (unsigned long long)*total;
        st->n_fresh = 0;
    }
    if (i >= n)
        return;
    const int d = dest[i];
    if (d < 0)
        return;
    const long long o = (long long)blk_off[i / SCAN_B] + d;
    A.x[o] = B.x[i];
    A.y[o] = B.y[i];
    A.z[o] = B.z[i];
    A.vx[o] = B.vx[i];
    A.vy[o] = B.vy[i];
    A.vz[o] = B.vz[i];
    A.cell[o] = B.cell[i];
    A.id[o] = B.id[i];
    dest[i] = (int)o;
}

template <typename R>
cudaError_t launch_compact(cudaStream_t s, long long n, int *dest, Particles<R> B, Particles<R> A,
                           DevState *st, int a, int *scratch)
{
    const int nb = (int)((n + SCAN_B - 1) / SCAN_B);
    int *blk_sum = scratch, *blk_off = scratch + nb + 1, *total = scratch + 2 * nb + 1;
    if (nb > 0) {
        k_scan_local<<<nb, SCAN_B, 0, s>>>(n, dest, blk_sum);
        k_scan_blocks<<<1, SCAN_B, 0, s>>>(nb, blk_sum, blk_off, total);
    } else {
        cudaMemsetAsync(total, 0, sizeof(int), s);
    }
    k_compact<R><<<(unsigned)(n > 0 ? (n + 255) / 256 : 1), 256, 0, s>>>(n, dest, blk_off, total,
                                                                         B, A, st, a);
    return cudaGetLastError();
}
template cudaError_t launch_compact<double>(cudaStream_t, long long, int *, Particles<double>,
                                            Particles<double>, DevState *, int, int *);
template cudaError_t launch_compact<float>(cudaStream_t, long long, int *, Particles<float>,
                                           Particles<float>, DevState *, int, int *);

}  // namespace pf
