// collide.cu -- Monte Carlo binary collisions between the SPs of a cell
// (App. F of Veske et al., after Takizuka & Abe 1977): group the SPs by cell,
// pair them in a random order, collide each pair elastically with a Gaussian
// tan(theta/2) and a uniform azimuth.
//
// Grouping is a counting sort by cell (histogram, exclusive scan, fill with
// one atomic per SP); the order inside a cell is then fixed by sorting on a
// random key of (seed, step, SP id), so the pairs do not depend on the order
// in which the atomics ran or on the SPs' buffer order.  One thread per cell
// sorts and collides (a few SPs per cell; the few crowded cells near the apex
// are the long tail).
#include "common.cuh"
#include "rng.cuh"

namespace pf {

constexpr double PI = 3.14159265358979323846;

template <typename R>
__global__ void k_coll_count(CollArgs<R> g)
{
    const long long n = (long long)*g.n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        atomicAdd(g.cnt + g.P.cell[i], 1);
}

template <typename R>
__global__ void k_coll_fill(CollArgs<R> g)
{
    const long long n = (long long)*g.n;
    const long long step = *g.step;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int t = g.P.cell[i];
        const int slot = g.off[t] + atomicAdd(g.fill + t, 1);
        g.perm[slot] = (int)i;
        const uint64_t seed = g.seed + (uint64_t)g.tet_rep[t];
        g.key[i] = hash4(seed, (uint64_t)step, RNG_SHUF_DOMAIN, (uint64_t)g.P.id[i]);
    }
}

// One elastic collision (eqs. vel12, scat_vel, rot_mat, sin_theta): the
// relative velocity w = u_a - u_b turns, w' = w + M(theta, phi) w, and
// v_{a,b} = u_{a,b} +- M w / 2; delta = tan(theta/2) ~ N(0, C / |w|^3)
// (eq. variance with everything but the relative speed in C).
__device__ void collide_pair(double va[3], double vb[3], double C, double U1, double U2, double U3)
{
    const double w[3] = {va[0] - vb[0], va[1] - vb[1], va[2] - vb[2]};
    const double u = sqrt((w[0] * w[0] + w[1] * w[1]) + w[2] * w[2]);
    if (!(u > 0.0))
        return;
    const double var = C / ((u * u) * u);
    const double delta = sqrt(var) * (sqrt(-2.0 * log(1.0 - U1)) * cos((2.0 * PI) * U2));
    const double phi = (2.0 * PI) * U3;
    const double dd = delta * delta;
    const double s = (2.0 * delta) / (1.0 + dd);    // sin theta
    const double c1 = (2.0 * dd) / (1.0 + dd);      // 1 - cos theta
    const double sp = sin(phi), cp = cos(phi);
    const double wp = sqrt(w[0] * w[0] + w[1] * w[1]);
    double d[3];
    if (wp > 0.0) {
        const double a = (s * sp) * (u / wp);
        const double bx = (s * cp) * (w[0] / wp), by = (s * cp) * (w[1] / wp);
        d[0] = (-c1 * w[0] + a * w[1]) + bx * w[2];
        d[1] = (-a * w[0] - c1 * w[1]) + by * w[2];
        d[2] = (-bx * w[0] - by * w[1]) - c1 * w[2];
    } else {
        d[0] = (s * cp) * w[2];
        d[1] = (s * sp) * w[2];
        d[2] = -c1 * w[2];
    }
    for (int k = 0; k < 3; ++k) {
        va[k] = va[k] + 0.5 * d[k];
        vb[k] = vb[k] - 0.5 * d[k];
    }
}

template <typename R>
__device__ __forceinline__ void collide_slots(CollArgs<R> &g, int a, int b, double C, uint64_t seed,
                                              uint64_t step, uint64_t kq, uint64_t ci)
{
    double va[3] = {(double)g.P.vx[a], (double)g.P.vy[a], (double)g.P.vz[a]};
    double vb[3] = {(double)g.P.vx[b], (double)g.P.vy[b], (double)g.P.vz[b]};
    collide_pair(va, vb, C, uniform01(seed, step, kq, ci, 1), uniform01(seed, step, kq, ci, 2),
                 uniform01(seed, step, kq, ci, 3));
    g.P.vx[a] = (R)va[0];
    g.P.vy[a] = (R)va[1];
    g.P.vz[a] = (R)va[2];
    g.P.vx[b] = (R)vb[0];
    g.P.vy[b] = (R)vb[1];
    g.P.vz[b] = (R)vb[2];
}

// Per cell: order its SPs by (key, id), then an odd count collides the first
// three as (0,1), (1,2), (2,0) with half the variance, and the rest in pairs.
template <typename R>
__global__ void k_coll_cells(CollArgs<R> g)
{
    const uint64_t step = (uint64_t)*g.step;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < g.T; t += gridDim.x * blockDim.x) {
        const int m = g.cnt[t];
        if (m < 2)
            continue;
        int *p = g.perm + g.off[t];
        for (int i = 1; i < m; ++i) {   // insertion sort on (key, id)
            const int x = p[i];
            const unsigned long long kx = g.key[x];
            const long long ix = g.P.id[x];
            int j = i - 1;
            while (j >= 0) {
                const unsigned long long kj = g.key[p[j]];
                if (kj < kx || (kj == kx && g.P.id[p[j]] <= ix))
                    break;
                p[j + 1] = p[j];
                --j;
            }
            p[j + 1] = x;
        }
        const int rep = g.tet_rep[t];
        const uint64_t seed = g.seed + (uint64_t)rep;
        const uint64_t kq = RNG_COLL_DOMAIN | (uint64_t)(t - g.rep_tet_off[rep]);
        const double vol = g.det[t] / 6.0;
        const double nreal = (double)m * g.w_sp;
        const double q2 = g.q * g.q;
        const double num = ((q2 * q2) * nreal) * (g.coulomb_log * g.dt);
        const double den = ((2.0 * PI) * (g.eps0 * g.eps0)) * ((g.m * g.m) * vol);
        const double C = num / den;
        uint64_t ci = 0;
        int k0 = 0;
        if (m & 1) {
            collide_slots(g, p[0], p[1], 0.5 * C, seed, step, kq, ci++);
            collide_slots(g, p[1], p[2], 0.5 * C, seed, step, kq, ci++);
            collide_slots(g, p[2], p[0], 0.5 * C, seed, step, kq, ci++);
            k0 = 3;
        }
        for (int k = k0; k + 1 < m; k += 2)
            collide_slots(g, p[k], p[k + 1], C, seed, step, kq, ci++);
    }
}

template <typename R> cudaError_t launch_collide(cudaStream_t s, const CollArgs<R> &g)
{
    cudaError_t e = cudaMemsetAsync(g.cnt, 0, sizeof(int) * (size_t)g.T, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(g.fill, 0, sizeof(int) * (size_t)g.T, s);
    if (e != cudaSuccess)
        return e;
    k_coll_count<R><<<g.grid, 256, 0, s>>>(g);
    e = launch_exclusive_scan(s, g.T, g.cnt, g.off, g.scan);
    if (e != cudaSuccess)
        return e;
    k_coll_fill<R><<<g.grid, 256, 0, s>>>(g);
    k_coll_cells<R><<<(unsigned)((g.T + 127) / 128), 128, 0, s>>>(g);
    return cudaGetLastError();
}

template cudaError_t launch_collide<double>(cudaStream_t, const CollArgs<double> &);
template cudaError_t launch_collide<float>(cudaStream_t, const CollArgs<float> &);

// ---------------------------------------------------------------------------
// SPs ordered by cell (a counting sort): neighbouring SPs then walk through
// the same walk records, which the L1 keeps.  The order inside a cell is
// whatever the atomics gave; nothing computed depends on the SPs' order.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_sort_count(Particles<R> B, const unsigned long long *nB, int *cnt, int *rank)
{
    const long long n = (long long)*nB;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        rank[i] = atomicAdd(cnt + B.cell[i], 1);
}

template <typename R>
__global__ void k_sort_move(Particles<R> B, Particles<R> A, const unsigned long long *nB,
                            unsigned long long *nA, const int *off, const int *rank)
{
    const long long n = (long long)*nB;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        *nA = (unsigned long long)n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int t = B.cell[i];
        const long long o = (long long)off[t] + rank[i];
        A.x[o] = B.x[i];
        A.y[o] = B.y[i];
        A.z[o] = B.z[i];
        A.vx[o] = B.vx[i];
        A.vy[o] = B.vy[i];
        A.vz[o] = B.vz[i];
        A.cell[o] = t;
        A.id[o] = B.id[i];
    }
}

template <typename R>
cudaError_t launch_sort_by_cell(cudaStream_t s, int grid, int T, Particles<R> B, Particles<R> A,
                                const unsigned long long *nB, unsigned long long *nA, int *cnt,
                                int *off, int *rank, int *scan)
{
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)T, s);
    if (e != cudaSuccess)
        return e;
    k_sort_count<R><<<grid, 256, 0, s>>>(B, nB, cnt, rank);
    e = launch_exclusive_scan(s, T, cnt, off, scan);
    if (e != cudaSuccess)
        return e;
    k_sort_move<R><<<grid, 256, 0, s>>>(B, A, nB, nA, off, rank);
    return cudaGetLastError();
}
template cudaError_t launch_sort_by_cell<double>(cudaStream_t, int, int, Particles<double>,
                                                 Particles<double>, const unsigned long long *,
                                                 unsigned long long *, int *, int *, int *, int *);
template cudaError_t launch_sort_by_cell<float>(cudaStream_t, int, int, Particles<float>,
                                                Particles<float>, const unsigned long long *,
                                                unsigned long long *, int *, int *, int *, int *);

}  // namespace pf
