// particles.cu -- the particle side of one PIC step: field per tetrahedron,
// field-emission injection, leapfrog push, neighbour-walk relocation and
// fixed-point charge deposition (Sec. II.B of Veske et al., PRE 101, 053307).
//
// Compiled with --fmad=false so that the FP64 instantiation evaluates every
// expression exactly as written (no fused multiply-add): the FP64 path then
// reproduces a plain FP64 CPU implementation bit for bit.
//
// Layout: SPs are a structure of arrays (x, y, z, vx, vy, vz, cell, id), one
// thread per SP, grid-stride loops that keep each warp on consecutive SPs so
// loads and stores coalesce.  Each step of the walk is one 128-byte (FP64) or
// 64-byte (FP32) record fetch.  Survivors are appended to the other buffer
// with one atomic per warp; deposits are int64 atomics, so the node charge is
// independent of the order in which SPs arrive.
#include "common.cuh"
#include "rng.cuh"

namespace pf {

#define FULL_MASK 0xffffffffu

enum { FATE_ALIVE = 0, FATE_COLLECTED = 1, FATE_ABSORBED = 2, FATE_LIMIT = 3 };

__device__ __forceinline__ void set_err(int *err, int code) { atomicCAS(err, 0, code); }

// Fowler-Nordheim J [A/m^2] for a field F [V/m] and work function phi [eV]:
// J = a F^2 / (phi t^2) exp(-v b phi^1.5 / F) with F in V/nm, Forbes'
// v(f) = 1 - f + (f/6) ln f, t(f) = 1 + f/9 - (f/18) ln f, f = c_S^2 F / phi^2
// clamped to the barrier top f <= 1 (elementary model: v = t = 1).
__device__ double fn_current(double F, double phi, int model)
{
    const double a = 1.541434e-6, b = 6.830890, cS2 = 1.439964;
    if (!(F > 0.0))
        return 0.0;
    double Fn = F * 1e-9;
    double v = 1.0, t = 1.0;
    if (model == PIC_FN_MURPHY_GOOD) {
        double f = (cS2 * Fn) / (phi * phi);
        if (f > 1.0)
            f = 1.0;
        double lf = log(f);
        v = (1.0 - f) + (f / 6.0) * lf;
        t = (1.0 + f / 9.0) - (f / 18.0) * lf;
    }
    double pre = (a * Fn * Fn) / (phi * t * t);
    double expo = -((v * b) * (phi * sqrt(phi))) / Fn;
    return (pre * exp(expo)) * 1e18;
}

// ---------------------------------------------------------------------------
// walk records
// ---------------------------------------------------------------------------
// The walk issues one record fetch per face crossing, the lanes of a warp at
// different records, and is bound by the L1 data stage that hands the bytes
// to the lanes: the 64-byte FP32 record comes in two 32-byte loads (fused
// particle kernel 1.55 -> 1.48 ms on the 1M-tet tip against four 16-byte
// loads).  The FP64 record keeps 16-byte loads: the 32-byte form cost its
// persistent walk a register and a block per SM.
template <typename T>
__device__ __forceinline__ T load_rec(const T *p)
{
    static_assert(sizeof(T) % 16 == 0, "record size");
    T out;
    if constexpr (sizeof(T) == 64) {
        const char *s = reinterpret_cast<const char *>(p);
        unsigned *d = reinterpret_cast<unsigned *>(&out);
#pragma unroll
        for (int i = 0; i < 2; ++i)
            asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                : "=r"(d[8 * i + 0]), "=r"(d[8 * i + 1]), "=r"(d[8 * i + 2]), "=r"(d[8 * i + 3]),
                  "=r"(d[8 * i + 4]), "=r"(d[8 * i + 5]), "=r"(d[8 * i + 6]), "=r"(d[8 * i + 7])
                : "l"(s + 32 * i));
    } else {
        const int4 *s = reinterpret_cast<const int4 *>(p);
        int4 *d = reinterpret_cast<int4 *>(&out);
#pragma unroll
        for (int i = 0; i < (int)(sizeof(T) / 16); ++i)
            d[i] = __ldg(s + i);
    }
    return out;
}

// The part of an FP32 record a walk step always needs, J^-1 and x0 (the first
// 48 bytes: one 32-byte and one 16-byte load); the neighbour of the exit face
// is read on its own once the face is known, and not at all in the last
// tetrahedron -- the data stage then moves 52 bytes per crossing instead of 64
// (fused particle kernel 1.48 -> 1.26 ms on the 1M-tet tip).
__device__ __forceinline__ void load_rec_geometry(const TetRec32 *p, TetRec32 &rec)
{
    const char *base = reinterpret_cast<const char *>(p);
    unsigned *d = reinterpret_cast<unsigned *>(&rec);
    asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]),
          "=r"(d[7])
        : "l"(base));
    const int4 q = __ldg(reinterpret_cast<const int4 *>(base + 32));
    d[8] = (unsigned)q.x;
    d[9] = (unsigned)q.y;
    d[10] = (unsigned)q.z;
    d[11] = (unsigned)q.w;
}

// lambda_k = row_k(J^-1) . (r - x0), k = 1..3; lambda_0 = ((1 - l1) - l2) - l3
template <typename R, typename T>
__device__ __forceinline__ void barycentric(const T &rec, const R r[3], R lam[4])
{
    R d0 = r[0] - rec.x0[0], d1 = r[1] - rec.x0[1], d2 = r[2] - rec.x0[2];
    lam[1] = (rec.j[0] * d0 + rec.j[1] * d1) + rec.j[2] * d2;
    lam[2] = (rec.j[3] * d0 + rec.j[4] * d1) + rec.j[5] * d2;
    lam[3] = (rec.j[6] * d0 + rec.j[7] * d1) + rec.j[8] * d2;
    lam[0] = (((R)1 - lam[1]) - lam[2]) - lam[3];
}

// Relocation by walking neighbours (Sec. II.B.2): leave through the face
// opposite the most negative barycentric coordinate (lowest index on ties),
// never back through the face just entered; stop when every other coordinate
// is >= 0.  walk_step does one step: it returns WALK_CONTINUE after moving to
// the next tetrahedron (t, entered, r updated; r wrapped on Gamma_2) or the
// fate of the SP, with lam holding the barycentrics in its final tetrahedron.
constexpr int WALK_CONTINUE = -1;

template <typename R>
__device__ __forceinline__ int walk_step(const MeshView<R> &m, int walk_max, R r[3], int &t,
                                         int &entered, R lam[4], int &steps, int &wraps)
{
    using T = typename Rec<R>::type;
    T rec;
    if constexpr (sizeof(R) == 4)
        load_rec_geometry(m.rec + t, rec);      // rec.nb is not loaded
    else
        rec = load_rec(m.rec + t);
    barycentric<R>(rec, r, lam);
    int k = -1;
    R mn = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (i == entered)
            continue;
        if (k < 0 || lam[i] < mn) {
            k = i;
            mn = lam[i];
        }
    }
    if (mn >= (R)0)
        return FATE_ALIVE;
    if (steps >= walk_max)
        return FATE_LIMIT;
    ++steps;
    int p;
    if constexpr (sizeof(R) == 4)
        p = __ldg(&m.rec[t].nb[k]);
    else
        p = k == 0 ? rec.nb[0] : k == 1 ? rec.nb[1] : k == 2 ? rec.nb[2] : rec.nb[3];
    if (p >= 0) {
        t = p >> 2;
        entered = p & 3;
        return WALK_CONTINUE;
    }
    if (p == NB_TOP)
        return FATE_COLLECTED;
    if (p == NB_CATHODE)
        return FATE_ABSORBED;
    int v = NB_SIDE - p;
    int sc = (v >> 2) & 3;
    const double *L = m.rep_L + 2 * m.tet_rep[t];   // the replica's periodic box
    entered = v & 3;
    t = v >> 4;
    if (sc == 0)
        r[0] = r[0] + (R)L[0];
    else if (sc == 1)
        r[0] = r[0] + (R)(-L[0]);
    else if (sc == 2)
        r[1] = r[1] + (R)L[1];
    else
        r[1] = r[1] + (R)(-L[1]);
    ++wraps;
    return WALK_CONTINUE;
}

template <typename R>
__device__ int walk(const MeshView<R> &m, int walk_max, R r[3], int &t, R lam[4], int &steps,
                    int &wraps)
{
    int entered = -1;
    steps = 0;
    for (;;) {
        int f = walk_step<R>(m, walk_max, r, t, entered, lam, steps, wraps);
        if (f != WALK_CONTINUE)
            return f;
    }
}

template <typename R> __device__ __forceinline__ long long quantize(R x, double scale);
template <> __device__ __forceinline__ long long quantize<double>(double x, double scale)
{
    return __double2ll_rn(x * scale);
}
template <> __device__ __forceinline__ long long quantize<float>(float x, double scale)
{
    return __float2ll_rn(x * (float)scale);
}

// deposit (eq. poisson_rhs): w_i = rint(lambda_i 2^S), i = 0..2, w_3 the
// remainder, so that every SP adds exactly 2^S in total
template <typename R>
__device__ __forceinline__ void deposit_one(const int4 *tet, int t, const R lam[4], double scale,
                                            unsigned long long *W)
{
    long long one = (long long)scale;
    long long w0 = quantize<R>(lam[0], scale);
    long long w1 = quantize<R>(lam[1], scale);
    long long w2 = quantize<R>(lam[2], scale);
    long long w3 = ((one - w0) - w1) - w2;
    int4 v = __ldg(tet + t);
    atomicAdd(W + v.x, (unsigned long long)w0);
    atomicAdd(W + v.y, (unsigned long long)w1);
    atomicAdd(W + v.z, (unsigned long long)w2);
    atomicAdd(W + v.w, (unsigned long long)w3);
}

template <typename V> __device__ __forceinline__ void e3(const V &e, double o[3])
{
    o[0] = (double)e.x;
    o[1] = (double)e.y;
    o[2] = (double)e.z;
}

// Emission of SP j of quadrangle q (Sec. II.B.3 and App. E): a uniform point
// of the parallelogram V + R1 (m1 - V) + R2 (m2 - V) accepted when its
// triangle barycentric coordinate of V is the largest (i.e. it lies in the
// quadrangle V, m1, centroid, m2); v0 = (q/m) E dt (1/2 + R3); the point is
// displaced by v0 dt R3 (fractional push).  Returns false when 64 attempts
// were rejected.
template <typename R>
__device__ bool emit(const MeshView<R> &m, const RunConst &c, long long step, int q, long long j,
                     double r[3], double v[3], int &cell, long long &id)
{
    int f = q / 3, vtx = q - 3 * f;
    const int rep = m.face_rep[f];
    const uint64_t seed = c.seed + (uint64_t)rep;                    // replica's stream
    const uint64_t ql = (uint64_t)(q - 3 * m.rep_face_off[rep]);     // quadrangle in it
    const int *fn = m.face_nodes + 3 * f;
    int ia = fn[vtx], ib = fn[vtx == 2 ? 0 : vtx + 1], ic = fn[vtx == 0 ? 2 : vtx - 1];
    const double *V = m.xyz + 3 * (size_t)ia, *Vn = m.xyz + 3 * (size_t)ib;
    const double *Vp = m.xyz + 3 * (size_t)ic;
    double R1 = 0.0, R2 = 0.0;
    bool ok = false;
    for (int a = 0; a < MAX_ATTEMPTS && !ok; ++a) {
        R1 = uniform01(seed, (uint64_t)step, ql, (uint64_t)j, (uint64_t)(1 + 2 * a));
        R2 = uniform01(seed, (uint64_t)step, ql, (uint64_t)j, (uint64_t)(2 + 2 * a));
        double l_next = R1 * 0.5, l_prev = R2 * 0.5;
        double l_v = (1.0 - l_next) - l_prev;
        ok = l_v >= l_next && l_v >= l_prev;
    }
    if (!ok)
        return false;
    double R3 = uniform01(seed, (uint64_t)step, ql, (uint64_t)j, 255);
    int ft = m.face_tet[f];
    double E[3];
    e3(m.E[ft], E);
    double s = c.qmdt * (0.5 + R3);
    double tR = c.dt * R3;
    for (int i = 0; i < 3; ++i) {
        double m1 = (V[i] + Vn[i]) * 0.5;
        double m2 = (V[i] + Vp[i]) * 0.5;
        double pnt = (V[i] + R1 * (m1 - V[i])) + R2 * (m2 - V[i]);
        double v0 = s * E[i];
        v[i] = v0;
        r[i] = pnt + v0 * tR;
    }
    cell = ft;
    id = (step << ID_STEP_SHIFT) | ((long long)q << ID_QUAD_SHIFT) | j;
    return true;
}

// largest q with qoff[q] <= tn (qoff nondecreasing, qoff[nq] > tn)
__device__ __forceinline__ int find_quad(const long long *qoff, int nq, long long tn)
{
    int lo = 0, hi = nq - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(qoff + mid) <= tn)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// warp-level helpers: append survivors with one atomic per warp, and sum
// counters with one atomic per warp
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ long long append(bool alive, const R r[3], const R v[3], int cell,
                                            long long id, Particles<R> B, unsigned long long *cntB)
{
    unsigned mask = __ballot_sync(FULL_MASK, alive);
    if (!mask)
        return -1;
    int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == 0)
        base = atomicAdd(cntB, (unsigned long long)__popc(mask));
    base = __shfl_sync(FULL_MASK, base, 0);
    if (alive) {
        long long o = (long long)base + __popc(mask & ((1u << lane) - 1u));
        B.x[o] = r[0];
        B.y[o] = r[1];
        B.z[o] = r[2];
        B.vx[o] = v[0];
        B.vy[o] = v[1];
        B.vz[o] = v[2];
        B.cell[o] = cell;
        B.id[o] = id;
        return o;
    }
    return -1;
}

__device__ __forceinline__ void count_fates(int fate, int steps, int wraps, bool act,
                                            pic_step_stats *stats, bool warp_iters = true)
{
    if (!stats)
        return;
    unsigned col = __ballot_sync(FULL_MASK, act && fate == FATE_COLLECTED);
    unsigned abs_ = __ballot_sync(FULL_MASK, act && fate == FATE_ABSORBED);
    int sw = __reduce_add_sync(FULL_MASK, act ? (unsigned)steps : 0u);
    int sr = __reduce_add_sync(FULL_MASK, act ? (unsigned)wraps : 0u);
    int mx = (int)__reduce_max_sync(FULL_MASK, act ? (unsigned)steps : 0u);
    if ((threadIdx.x & 31) == 0) {
        if (col)
            atomicAdd((unsigned long long *)&stats->collected, (unsigned long long)__popc(col));
        if (abs_)
            atomicAdd((unsigned long long *)&stats->absorbed, (unsigned long long)__popc(abs_));
        if (sw)
            atomicAdd((unsigned long long *)&stats->crossings, (unsigned long long)sw);
        if (sr)
            atomicAdd((unsigned long long *)&stats->wrapped, (unsigned long long)sr);
        if (mx) {
            atomicMax(&stats->max_walk, mx);
            if (warp_iters)
                atomicAdd((unsigned long long *)&stats->walk_warp_iters, (unsigned long long)mx);
        }
    }
}

// ---------------------------------------------------------------------------
// field: E_t = -sum_i Phi_{v_i} grad N_i, constant per tetrahedron
// ---------------------------------------------------------------------------
// End of a step (see StepHdr): file the step's statistics and advance the
// step index.  Run by one thread of the step's last kernel.
__device__ __forceinline__ void end_step(DevState *st, pic_step_stats *slot)
{
    StepHdr &h = st->hdr;
    long long i = h.step - h.step0;
    if (i >= 0 && i < h.ring_cap)
        h.ring[i] = *slot;
    *slot = pic_step_stats{};
    h.step = h.step + 1;
}

__global__ void k_field64(int T, const TetRec64 *__restrict__ rec, const int4 *__restrict__ tet,
                          const double *__restrict__ phi, Vec4d *E, DevState *st,
                          pic_step_stats *slot)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (st && t == 0)
        end_step(st, slot);
    if (t >= T)
        return;
    TetRec64 r = load_rec(rec + t);
    int4 v = __ldg(tet + t);
    double p0 = phi[v.x], p1 = phi[v.y], p2 = phi[v.z], p3 = phi[v.w];
    double e[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        double g0 = -((r.j[0 + i] + r.j[3 + i]) + r.j[6 + i]);
        double s = ((p0 * g0 + p1 * r.j[0 + i]) + p2 * r.j[3 + i]) + p3 * r.j[6 + i];
        e[i] = -s;
    }
    E[t] = make_vec4d(e[0], e[1], e[2], 0.0);
}

// FP32 records: the same field written with potential differences
// E = -sum_{k=1..3} (Phi_k - Phi_0) grad N_k (identical since grad N_0 =
// -sum grad N_k), so that the FP32 gradients never multiply the large
// absolute potential.
__global__ void k_field32(int T, const TetRec32 *__restrict__ rec, const int4 *__restrict__ tet,
                          const double *__restrict__ phi, float4 *E, DevState *st,
                          pic_step_stats *slot)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (st && t == 0)
        end_step(st, slot);
    if (t >= T)
        return;
    TetRec32 r = load_rec(rec + t);
    int4 v = __ldg(tet + t);
    double p0 = phi[v.x];
    float d1 = (float)(phi[v.y] - p0), d2 = (float)(phi[v.z] - p0), d3 = (float)(phi[v.w] - p0);
    float e[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        e[i] = -((d1 * r.j[0 + i] + d2 * r.j[3 + i]) + d3 * r.j[6 + i]);
    E[t] = make_float4(e[0], e[1], e[2], 0.f);
}

// ---------------------------------------------------------------------------
// injection: count per quadrangle (eqs. nsp, rnd_nsp) and exclusive scan
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_inject_count(int nq, MeshView<R> m, RunConst c, const long long *stepp,
                               int *qcount, int *err)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq)
        return;
    const long long step = *stepp;
    int f = q / 3;
    double E[3];
    e3(m.E[m.face_tet[f]], E);
    const double *n = m.face_nhat + 3 * (size_t)f;
    double F = -((E[0] * n[0] + E[1] * n[1]) + E[2] * n[2]);
    if (!(F > 0.0))
        F = 0.0;
    double J = fn_current(F, m.wf[f], c.fn_model);
    double Aq = m.face_area[f] / 3.0;
    double nsp = ((J * Aq) * c.dt) / (c.e_charge * c.w_sp);
    const int rep = m.face_rep[f];
    double R0 = uniform01(c.seed + (uint64_t)rep, (uint64_t)step,
                          (uint64_t)(q - 3 * m.rep_face_off[rep]), 0, 0);
    double fl = floor(nsp);
    double frac = nsp - fl;
    long long cnt = (long long)fl + (R0 >= frac ? 0 : 1);
    if (!(nsp >= 0.0) || cnt >= MAX_PER_QUAD) {
        set_err(err, PIC_ERR_CAPACITY);
        cnt = 0;
    }
    qcount[q] = (int)cnt;
}

// single block: qoff[q] = sum_{p<q} qcount[p], qoff[nq] = total; capacity check
__global__ void __launch_bounds__(1024) k_inject_scan(int nq, const int *__restrict__ qcount,
                                                      long long *qoff, DevState *st, int buf,
                                                      long long capacity, int split,
                                                      pic_step_stats *stats)
{
    __shared__ long long warp_tot[32];
    __shared__ long long grand;
    int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int per = (nq + blockDim.x - 1) / blockDim.x;
    int lo = min(nq, tid * per), hi = min(nq, lo + per);
    long long local = 0;
    for (int i = lo; i < hi; ++i)
        local += qcount[i];
    long long incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= o)
            incl += y;
    }
    if (lane == 31)
        warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        long long w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
        long long wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(FULL_MASK, wi, o);
            if (lane >= o)
                wi += y;
        }
        warp_tot[lane] = wi - w;  // exclusive prefix of warp totals
        if (lane == 31)
            grand = wi;
    }
    __syncthreads();
    long long run = warp_tot[wid] + incl - local;
    for (int i = lo; i < hi; ++i) {
        qoff[i] = run;
        run += qcount[i];
    }
    if (tid == 0) {
        long long total = grand;
        qoff[nq] = total;
        long long n_alive = (long long)st->cnt[buf];
        if (n_alive + total > capacity) {
            atomicCAS(&st->err, 0, PIC_ERR_CAPACITY);
            total = 0;
        }
        st->n_new = total;
        if (split) {
            st->base = n_alive;
            st->n_fresh = total;
            st->cnt[buf] = (unsigned long long)(n_alive + total);
        }
        if (stats)
            stats->injected = total;
    }
}

// split API: write the fresh SPs at the end of buffer A
template <typename R>
__global__ void k_inject_emit(MeshView<R> m, RunConst c, const long long *stepp, int nq,
                              const long long *__restrict__ qoff, Particles<R> P, DevState *st)
{
    const long long step = *stepp;
    long long n_new = st->n_new, base = st->base;
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long tn = blockIdx.x * (long long)blockDim.x + threadIdx.x; tn < n_new; tn += stride) {
        int q = find_quad(qoff, nq, tn);
        long long j = tn - qoff[q];
        double r[3], v[3];
        int cell;
        long long id;
        if (!emit<R>(m, c, step, q, j, r, v, cell, id)) {
            set_err(&st->err, PIC_ERR_ARG);
            r[0] = r[1] = r[2] = 0.0;
            v[0] = v[1] = v[2] = 0.0;
            cell = m.face_tet[q / 3];
            id = -1;
        }
        long long o = base + tn;
        P.x[o] = (R)r[0];
        P.y[o] = (R)r[1];
        P.z[o] = (R)r[2];
        P.vx[o] = (R)v[0];
        P.vy[o] = (R)v[1];
        P.vz[o] = (R)v[2];
        P.cell[o] = cell;
        P.id[o] = id;
    }
}

// ---------------------------------------------------------------------------
// push + relocate (split API): kick non-fresh SPs by (q/m) dt E_cell, drift
// all by dt v, walk, append survivors to buffer B
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_push_relocate(MeshView<R> m, RunConst c, Particles<R> A, Particles<R> B, int a,
                                DevState *st, pic_step_stats *stats, int *dest)
{
    long long n = (long long)st->cnt[a];
    long long n_old = n - st->n_fresh;
    unsigned long long *cntB = &st->cnt[1 - a];
    const R qmdt = (R)c.qmdt, dt = (R)c.dt;
    long long wstride = ((long long)gridDim.x * blockDim.x) & ~31LL;
    long long wbase = (blockIdx.x * (long long)blockDim.x + threadIdx.x) & ~31LL;
    int lane = threadIdx.x & 31;
    for (long long base = wbase; base < n; base += wstride) {
        long long i = base + lane;
        bool act = i < n;
        R r[3] = {0, 0, 0}, v[3] = {0, 0, 0}, lam[4];
        int t = 0, fate = FATE_ABSORBED, steps = 0, wraps = 0;
        long long id = 0;
        if (act) {
            r[0] = A.x[i];
            r[1] = A.y[i];
            r[2] = A.z[i];
            v[0] = A.vx[i];
            v[1] = A.vy[i];
            v[2] = A.vz[i];
            t = A.cell[i];
            id = A.id[i];
            if (i < n_old) {
                typename Rec<R>::vec4 e = m.E[t];
                v[0] = v[0] + qmdt * (R)e.x;
                v[1] = v[1] + qmdt * (R)e.y;
                v[2] = v[2] + qmdt * (R)e.z;
            }
            r[0] = r[0] + dt * v[0];
            r[1] = r[1] + dt * v[1];
            r[2] = r[2] + dt * v[2];
            fate = walk<R>(m, c.walk_max, r, t, lam, steps, wraps);
            if (fate == FATE_LIMIT)
                set_err(&st->err, PIC_ERR_WALK_LIMIT);
        }
        bool alive = act && fate == FATE_ALIVE;
        if (dest) {
            // ordered form: a survivor keeps its index in B (the buffer is
            // compacted afterwards, in index order); dest flags the fate
            if (alive) {
                B.x[i] = r[0];
                B.y[i] = r[1];
                B.z[i] = r[2];
                B.vx[i] = v[0];
                B.vy[i] = v[1];
                B.vz[i] = v[2];
                B.cell[i] = t;
                B.id[i] = id;
            }
            if (act)
                dest[i] = alive ? 1 : fate == FATE_COLLECTED ? DEST_COLLECTED : DEST_ABSORBED;
        } else {
            append<R>(alive, r, v, t, id, B, cntB);
        }
        count_fates(fate, steps, wraps, act, stats);
    }
}

// deposit (split API): W += fixed-point weights of every SP in buffer A
template <typename R>
__global__ void k_deposit(MeshView<R> m, RunConst c, Particles<R> A, int a, DevState *st,
                          unsigned long long *W)
{
    using T = typename Rec<R>::type;
    long long n = (long long)st->cnt[a];
    long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        R r[3] = {A.x[i], A.y[i], A.z[i]};
        int t = A.cell[i];
        T rec = load_rec(m.rec + t);
        R lam[4];
        barycentric<R>(rec, r, lam);
        deposit_one<R>(m.tet, t, lam, c.scale, W);
    }
}

// ---------------------------------------------------------------------------
// one fused PIC step on the particle side: SPs [0, n_old) of buffer A are
// kicked, SPs [n_old, n_old + n_new) are emitted in place; all drift, walk,
// deposit, and survivors are appended to buffer B.
//
// Walk lengths differ by orders of magnitude between SPs (tens of crossings
// far from the tip, hundreds near the apex), so a warp that walks 32 SPs to
// completion idles lanes behind its slowest SP.  Two forms share the same
// per-SP arithmetic (start_sp, walk_step, deposit_one) as the split kernels:
// coherent warps, and persistent lanes that take the next SP from the warp's
// queue (refilled with CHUNK consecutive SPs from a global counter) as soon
// as theirs is done.
// ---------------------------------------------------------------------------
constexpr int CHUNK = 128;

template <typename R>
__device__ __forceinline__ void start_sp(const MeshView<R> &m, const RunConst &c, long long step,
                                         int nq, const long long *qoff, const Particles<R> &A,
                                         long long n_old, long long i, DevState *st, R r[3],
                                         R v[3], int &t, long long &id)
{
    const R qmdt = (R)c.qmdt, dt = (R)c.dt;
    if (i < n_old) {
        r[0] = A.x[i];
        r[1] = A.y[i];
        r[2] = A.z[i];
        v[0] = A.vx[i];
        v[1] = A.vy[i];
        v[2] = A.vz[i];
        t = A.cell[i];
        id = A.id[i];
        typename Rec<R>::vec4 e = m.E[t];
        v[0] = v[0] + qmdt * (R)e.x;
        v[1] = v[1] + qmdt * (R)e.y;
        v[2] = v[2] + qmdt * (R)e.z;
    } else {
        long long tn = i - n_old;
        int q = find_quad(qoff, nq, tn);
        double rd[3], vd[3];
        if (!emit<R>(m, c, step, q, tn - qoff[q], rd, vd, t, id)) {
            set_err(&st->err, PIC_ERR_ARG);
            rd[0] = rd[1] = rd[2] = 0.0;
            vd[0] = vd[1] = vd[2] = 0.0;
            t = m.face_tet[q / 3];
        }
        for (int k = 0; k < 3; ++k) {
            r[k] = (R)rd[k];
            v[k] = (R)vd[k];
        }
    }
    r[0] = r[0] + dt * v[0];
    r[1] = r[1] + dt * v[1];
    r[2] = r[2] + dt * v[2];
}

// Coherent form: each warp takes 32 consecutive SPs and walks them to the
// end together.  SPs that are neighbours in the buffer were injected or
// appended together and walk through the same records, so the warp's record
// fetches share L1 lines; on the FP32 path that locality is worth more than
// the lanes that idle behind the warp's longest walk.
// (FP32: at most 40 registers, six blocks of 256 threads per SM -- the 32-byte
// record loads would otherwise take it to 48 registers and five blocks; FP64,
// whose default is the persistent form: at most 64, no spills)
template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 6 : 4) k_step_fused(MeshView<R> m, RunConst c,
                                                    const long long *stepp, int nq,
                                                    const long long *__restrict__ qoff,
                                                    Particles<R> A, Particles<R> B, int a,
                                                    DevState *st, unsigned long long *W,
                                                    pic_step_stats *stats)
{
    const long long step = *stepp;
    const long long n_old = (long long)st->cnt[a];
    const long long n = n_old + st->n_new;
    unsigned long long *cntB = &st->cnt[1 - a];
    long long wstride = ((long long)gridDim.x * blockDim.x) & ~31LL;
    long long wbase = (blockIdx.x * (long long)blockDim.x + threadIdx.x) & ~31LL;
    int lane = threadIdx.x & 31;
    for (long long base = wbase; base < n; base += wstride) {
        long long i = base + lane;
        bool act = i < n;
        R r[3] = {0, 0, 0}, v[3] = {0, 0, 0}, lam[4];
        int t = 0, fate = FATE_ABSORBED, steps = 0, wraps = 0;
        long long id = 0;
        if (act) {
            start_sp<R>(m, c, step, nq, qoff, A, n_old, i, st, r, v, t, id);
            fate = walk<R>(m, c.walk_max, r, t, lam, steps, wraps);
            if (fate == FATE_LIMIT)
                set_err(&st->err, PIC_ERR_WALK_LIMIT);
            if (fate == FATE_ALIVE)
                deposit_one<R>(m.tet, t, lam, c.scale, W);
        }
        bool alive = act && fate == FATE_ALIVE;
        append<R>(alive, r, v, t, id, B, cntB);
        count_fates(fate, steps, wraps, act, stats);
    }
}

// Persistent form: lanes take the next SP as soon as theirs is done (see
// above); used where the walk is arithmetic-bound (FP64 on this part).
template <typename R>
__global__ void __launch_bounds__(256) k_step_fused_persistent(
    MeshView<R> m, RunConst c, const long long *stepp, int nq, const long long *__restrict__ qoff,
    Particles<R> A, Particles<R> B, int a, DevState *st, unsigned long long *W,
    pic_step_stats *stats)
{
    const long long step = *stepp;
    const long long n_old = (long long)st->cnt[a];
    const long long n = n_old + st->n_new;
    unsigned long long *cntB = &st->cnt[1 - a];
    const int lane = threadIdx.x & 31;
    const unsigned lower = (1u << lane) - 1u;
    long long q_next = 0, q_end = 0;  // the warp's queue (warp-uniform)
    bool exhausted = false;
    bool active = false;
    R r[3] = {0, 0, 0}, v[3] = {0, 0, 0}, lam[4] = {0, 0, 0, 0};
    int t = 0, entered = -1, steps = 0, wraps = 0;
    long long id = 0;
    unsigned long long n_cross = 0, n_iter = 0;
    unsigned n_col = 0, n_abs = 0, n_wrap = 0;
    int n_max = 0;
    for (;;) {
        // hand SPs to idle lanes
        unsigned idle = __ballot_sync(FULL_MASK, !active);
        while (idle) {
            if (q_next >= q_end) {
                if (exhausted)
                    break;
                long long b = 0;
                if (lane == 0)
                    b = (long long)atomicAdd(&st->work, (unsigned long long)CHUNK);
                b = __shfl_sync(FULL_MASK, b, 0);
                if (b >= n) {
                    exhausted = true;
                    break;
                }
                q_next = b;
                q_end = b + CHUNK < n ? b + CHUNK : n;
            }
            int nidle = __popc(idle);
            long long avail = q_end - q_next;
            int take = avail < nidle ? (int)avail : nidle;
            if (!active) {
                int rank = __popc(idle & lower);
                if (rank < take) {
                    start_sp<R>(m, c, step, nq, qoff, A, n_old, q_next + rank, st, r, v, t, id);
                    entered = -1;
                    steps = 0;
                    wraps = 0;
                    active = true;
                }
            }
            q_next += take;
            if (take == nidle)
                break;
            idle = __ballot_sync(FULL_MASK, !active);
        }
        if (!__any_sync(FULL_MASK, active))
            break;
        int fate = WALK_CONTINUE;
        ++n_iter;
        if (active)
            fate = walk_step<R>(m, c.walk_max, r, t, entered, lam, steps, wraps);
        bool finished = active && fate != WALK_CONTINUE;
        bool keep = finished && fate == FATE_ALIVE;
        if (finished) {
            if (keep)
                deposit_one<R>(m.tet, t, lam, c.scale, W);
            else if (fate == FATE_COLLECTED)
                ++n_col;
            else if (fate == FATE_ABSORBED)
                ++n_abs;
            else
                set_err(&st->err, PIC_ERR_WALK_LIMIT);
            n_cross += (unsigned long long)steps;
            n_wrap += (unsigned)wraps;
            n_max = steps > n_max ? steps : n_max;
            active = false;
        }
        append<R>(keep, r, v, t, id, B, cntB);
    }
    if (stats) {
        unsigned col = __reduce_add_sync(FULL_MASK, n_col);
        unsigned absb = __reduce_add_sync(FULL_MASK, n_abs);
        unsigned wr = __reduce_add_sync(FULL_MASK, n_wrap);
        int mx = (int)__reduce_max_sync(FULL_MASK, (unsigned)n_max);
        unsigned long long cr = n_cross;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            cr += __shfl_xor_sync(FULL_MASK, cr, o);
        if (lane == 0) {
            if (col)
                atomicAdd((unsigned long long *)&stats->collected, (unsigned long long)col);
            if (absb)
                atomicAdd((unsigned long long *)&stats->absorbed, (unsigned long long)absb);
            if (cr)
                atomicAdd((unsigned long long *)&stats->crossings, cr);
            if (wr)
                atomicAdd((unsigned long long *)&stats->wrapped, (unsigned long long)wr);
            if (mx)
                atomicMax(&stats->max_walk, mx);
            if (n_iter)
                atomicAdd((unsigned long long *)&stats->walk_warp_iters, n_iter);
        }
    }
}

// Rounds form: each warp owns a contiguous range of the buffer -- the SPs
// shared out evenly over the warps of the launch, in multiples of 32 -- and
// walks them in rounds of at most ROUND_STEPS face crossings; after every
// round the lanes whose SP has finished start the next SPs of the range, in
// order.  A lane then idles at most one round behind the warp's slowest walk
// instead of the whole walk, the per-crossing loop stays the tight loop of
// the coherent form (no warp vote per crossing), and the SPs in flight in a
// warp stay neighbours in the buffer (ordered by cell), so they keep sharing
// walk records in L1.
constexpr int ROUND_STEPS = 16;

template <typename R>
__global__ void __launch_bounds__(256) k_step_fused_rounds(
    MeshView<R> m, RunConst c, const long long *stepp, int nq, const long long *__restrict__ qoff,
    Particles<R> A, Particles<R> B, int a, DevState *st, unsigned long long *W,
    pic_step_stats *stats)
{
    const long long step = *stepp;
    const long long n_old = (long long)st->cnt[a];
    const long long n = n_old + st->n_new;
    unsigned long long *cntB = &st->cnt[1 - a];
    const int lane = threadIdx.x & 31;
    const unsigned lower = (1u << lane) - 1u;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long chunk = 32 * ((n + 32 * nwarps - 1) / (32 * nwarps));
    unsigned long long n_iter = 0;
    for (long long c0 = wid * chunk; c0 < n; c0 += nwarps * chunk) {
        const long long c1 = c0 + chunk < n ? c0 + chunk : n;
        long long next = c0;   // warp-uniform: the next SP of the range to start
        bool active = false;
        R r[3] = {0, 0, 0}, v[3] = {0, 0, 0}, lam[4] = {0, 0, 0, 0};
        int t = 0, entered = -1, steps = 0, wraps = 0;
        long long id = 0;
        for (;;) {
            const unsigned idle = __ballot_sync(FULL_MASK, !active);
            const long long avail = c1 - next;
            const int take = avail < (long long)__popc(idle) ? (int)avail : __popc(idle);
            if (!active) {
                const int rank = __popc(idle & lower);
                if (rank < take) {
                    start_sp<R>(m, c, step, nq, qoff, A, n_old, next + rank, st, r, v, t, id);
                    entered = -1;
                    steps = 0;
                    wraps = 0;
                    active = true;
                }
            }
            next += take;
            if (!__any_sync(FULL_MASK, active))
                break;
            int fate = WALK_CONTINUE;
            const int s0 = steps;
            if (active) {
                for (int k = 0; k < ROUND_STEPS; ++k) {
                    fate = walk_step<R>(m, c.walk_max, r, t, entered, lam, steps, wraps);
                    if (fate != WALK_CONTINUE)
                        break;
                }
            }
            n_iter += __reduce_max_sync(FULL_MASK, active ? (unsigned)(steps - s0) : 0u);
            const bool finished = active && fate != WALK_CONTINUE;
            if (finished && fate == FATE_LIMIT)
                set_err(&st->err, PIC_ERR_WALK_LIMIT);
            const bool keep = finished && fate == FATE_ALIVE;
            if (keep)
                deposit_one<R>(m.tet, t, lam, c.scale, W);
            append<R>(keep, r, v, t, id, B, cntB);
            count_fates(finished ? fate : FATE_ALIVE, steps, wraps, finished, stats, false);
            if (finished)
                active = false;
        }
    }
    if (stats && lane == 0 && n_iter)
        atomicAdd((unsigned long long *)&stats->walk_warp_iters, n_iter);
}

// ---------------------------------------------------------------------------
// state conversion between the SoA store and interleaved FP64 arrays
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_pack(long long n, Particles<R> A, double *r, double *v, int *cell, long long *id)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    if (r) {
        r[3 * i + 0] = (double)A.x[i];
        r[3 * i + 1] = (double)A.y[i];
        r[3 * i + 2] = (double)A.z[i];
    }
    if (v) {
        v[3 * i + 0] = (double)A.vx[i];
        v[3 * i + 1] = (double)A.vy[i];
        v[3 * i + 2] = (double)A.vz[i];
    }
    if (cell)
        cell[i] = A.cell[i];
    if (id)
        id[i] = A.id[i];
}

template <typename R>
__global__ void k_unpack(long long n, const double *r, const double *v, const int *cell,
                         const long long *id, Particles<R> A)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    A.x[i] = (R)r[3 * i + 0];
    A.y[i] = (R)r[3 * i + 1];
    A.z[i] = (R)r[3 * i + 2];
    A.vx[i] = (R)v[3 * i + 0];
    A.vy[i] = (R)v[3 * i + 1];
    A.vz[i] = (R)v[3 * i + 2];
    A.cell[i] = cell[i];
    A.id[i] = id[i];
}

template <typename V>
__global__ void k_field_unpack(int T, const V *E, double *out)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T)
        return;
    V e = E[t];
    out[3 * (size_t)t + 0] = (double)e.x;
    out[3 * (size_t)t + 1] = (double)e.y;
    out[3 * (size_t)t + 2] = (double)e.z;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

template <>
cudaError_t launch_field<double>(cudaStream_t s, int T, const TetRec64 *rec, const int4 *tet,
                                 const double *phi, Vec4d *E, DevState *st, pic_step_stats *slot)
{
    k_field64<<<blocks_for(T, 256), 256, 0, s>>>(T, rec, tet, phi, E, st, slot);
    return cudaGetLastError();
}
template <>
cudaError_t launch_field<float>(cudaStream_t s, int T, const TetRec32 *rec, const int4 *tet,
                                const double *phi, float4 *E, DevState *st, pic_step_stats *slot)
{
    k_field32<<<blocks_for(T, 256), 256, 0, s>>>(T, rec, tet, phi, E, st, slot);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_inject_count(cudaStream_t s, int nq, MeshView<R> m, RunConst c,
                                const long long *step, int *qcount, int *err)
{
    if (nq <= 0)
        return cudaSuccess;
    k_inject_count<R><<<blocks_for(nq, 256), 256, 0, s>>>(nq, m, c, step, qcount, err);
    return cudaGetLastError();
}

cudaError_t launch_inject_scan(cudaStream_t s, int nq, const int *qcount, long long *qoff,
                               DevState *st, int buf, long long capacity, int split_mode,
                               pic_step_stats *stats)
{
    k_inject_scan<<<1, 1024, 0, s>>>(nq, qcount, qoff, st, buf, capacity, split_mode, stats);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_inject_emit(cudaStream_t s, int grid, MeshView<R> m, RunConst c,
                               const long long *step, int nq, const long long *qoff,
                               Particles<R> P, DevState *st)
{
    k_inject_emit<R><<<grid, 256, 0, s>>>(m, c, step, nq, qoff, P, st);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_push_relocate(cudaStream_t s, int grid, MeshView<R> m, RunConst c,
                                 Particles<R> A, Particles<R> B, int a, DevState *st,
                                 pic_step_stats *stats, int *dest)
{
    k_push_relocate<R><<<grid, 256, 0, s>>>(m, c, A, B, a, st, stats, dest);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_deposit(cudaStream_t s, int grid, MeshView<R> m, RunConst c, Particles<R> A,
                           int a, DevState *st, unsigned long long *W)
{
    k_deposit<R><<<grid, 256, 0, s>>>(m, c, A, a, st, W);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_step_fused(cudaStream_t s, int grid, int walk_form, MeshView<R> m, RunConst c,
                              const long long *step, int nq, const long long *qoff, Particles<R> A,
                              Particles<R> B, int a, DevState *st, unsigned long long *W,
                              pic_step_stats *stats)
{
    const bool persistent = walk_form == WALK_FORM_AUTO ? sizeof(R) == 8
                                                         : walk_form == WALK_FORM_PERSISTENT;
    if (walk_form == WALK_FORM_ROUNDS)
        k_step_fused_rounds<R><<<grid, 256, 0, s>>>(m, c, step, nq, qoff, A, B, a, st, W, stats);
    else if (persistent)
        k_step_fused_persistent<R><<<grid, 256, 0, s>>>(m, c, step, nq, qoff, A, B, a, st, W, stats);
    else
        k_step_fused<R><<<grid, 256, 0, s>>>(m, c, step, nq, qoff, A, B, a, st, W, stats);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_pack(cudaStream_t s, long long n, Particles<R> A, double *r, double *v,
                        int *cell, long long *id)
{
    if (n <= 0)
        return cudaSuccess;
    k_pack<R><<<blocks_for(n, 256), 256, 0, s>>>(n, A, r, v, cell, id);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_unpack(cudaStream_t s, long long n, const double *r, const double *v,
                          const int *cell, const long long *id, Particles<R> A)
{
    if (n <= 0)
        return cudaSuccess;
    k_unpack<R><<<blocks_for(n, 256), 256, 0, s>>>(n, r, v, cell, id, A);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_field_unpack(cudaStream_t s, int T, const typename Rec<R>::vec4 *E, double *out)
{
    k_field_unpack<<<blocks_for(T, 256), 256, 0, s>>>(T, E, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// adjoint of one step for each SP (pic_adjoint)
// ---------------------------------------------------------------------------
// (d ln J/dF, d ln J/dphi) of fn_current: ln J = ln a + 2 ln Fn - ln phi
// - 2 ln t(f) - v(f) b phi^1.5 / Fn, Fn = F 1e-9, f = c_S^2 Fn / phi^2; where
// f is clamped to 1, v and t do not move with F or phi.
__device__ void fn_dlog(double F, double phi, int model, double &dF, double &dphi)
{
    const double b = 6.830890, cS2 = 1.439964;
    const double Fn = F * 1e-9;
    double v = 1.0, t = 1.0, vp = 0.0, tp = 0.0, fF = 0.0, fphi = 0.0;
    if (model == PIC_FN_MURPHY_GOOD) {
        const double fr = (cS2 * Fn) / (phi * phi);
        const double f = fr > 1.0 ? 1.0 : fr;
        const double lf = log(f);
        v = (1.0 - f) + (f / 6.0) * lf;
        t = (1.0 + f / 9.0) - (f / 18.0) * lf;
        if (fr <= 1.0) {
            vp = lf / 6.0 - 5.0 / 6.0;      // dv/df
            tp = 1.0 / 18.0 - lf / 18.0;    // dt/df
            fF = cS2 / (phi * phi);         // df/dFn
            fphi = -2.0 * fr / phi;         // df/dphi
        }
    }
    const double s15 = phi * sqrt(phi);
    const double dFn = 2.0 / Fn - 2.0 * (tp / t) * fF - b * s15 * (vp * fF / Fn - v / (Fn * Fn));
    dphi = -1.0 / phi - 2.0 * (tp / t) * fphi - b * (vp * fphi * s15 + 1.5 * v * sqrt(phi)) / Fn;
    dF = dFn * 1e-9;
}

// Reverse of one step for SP i of the step: collection (d Q / d omega =
// q w_sp), deposit (f = coef W 2^-S: omega_bar += coef sum_j fbar_j N_j,
// r_bar += coef sum_j fbar_j grad N_j in the final cell), drift r' = r + dt v'
// (the walk's cells and shifts are frozen), then the kick v' = v + (q/m) dt E
// of an old SP, or for a new one the emission v0 = (q/m) dt (1/2 + R3) E(t_f),
// r0 = point + v0 dt R3 and its weight J(F, phi_f) / J(theta0) with
// F = -E(t_f).n_f (eqs. sp_velocity, sp_displacement, nsp).
template <typename R>
__global__ void k_adjoint_sp(AdjStep<R> g)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= g.n)
        return;
    double rb[3] = {0.0, 0.0, 0.0}, vb[3] = {0.0, 0.0, 0.0}, wb = 0.0;
    const int d = g.dest[i];
    if (d >= 0) {
        rb[0] = g.in.rx[d];
        rb[1] = g.in.ry[d];
        rb[2] = g.in.rz[d];
        vb[0] = g.in.vx[d];
        vb[1] = g.in.vy[d];
        vb[2] = g.in.vz[d];
        wb = g.in.w[d];
        const int t = g.post.cell[d];
        const double r[3] = {(double)g.post.x[d], (double)g.post.y[d], (double)g.post.z[d]};
        const TetRec64 rec = load_rec(g.rec64 + t);
        double lam[4];
        barycentric<double>(rec, r, lam);
        const int4 nd = __ldg(g.tet + t);
        const double fb[4] = {g.fbar[nd.x], g.fbar[nd.y], g.fbar[nd.z], g.fbar[nd.w]};
        wb += g.coef * (((fb[0] * lam[0] + fb[1] * lam[1]) + fb[2] * lam[2]) + fb[3] * lam[3]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double g0 = -((rec.j[c] + rec.j[3 + c]) + rec.j[6 + c]);
            rb[c] += g.coef * (((fb[0] * g0 + fb[1] * rec.j[c]) + fb[2] * rec.j[3 + c]) +
                               fb[3] * rec.j[6 + c]);
        }
    } else if (d == DEST_COLLECTED) {
        wb = g.qw;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
        vb[c] += g.dt * rb[c];
    if (i < g.n_old) {
        const size_t t = (size_t)g.pre.cell[i];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            atomicAdd(g.Ebar + 3 * t + c, g.qmdt * vb[c]);
        g.out.rx[i] = rb[0];
        g.out.ry[i] = rb[1];
        g.out.rz[i] = rb[2];
        g.out.vx[i] = vb[0];
        g.out.vy[i] = vb[1];
        g.out.vz[i] = vb[2];
        g.out.w[i] = wb;
        return;
    }
    const long long id = g.pre.id[i];
    const long long step = id >> 42;
    const int q = (int)((id >> 18) & ((1LL << 24) - 1));
    const long long j = id & ((1LL << 18) - 1);
    const int f = q / 3;
    const int rep = g.face_rep[f];
    const double R3 = uniform01(g.seed + (uint64_t)rep, (uint64_t)step,
                                (uint64_t)(q - 3 * g.rep_face_off[rep]), (uint64_t)j, 255);
    const size_t ft = (size_t)g.face_tet[f];
    const double s = g.qmdt * (0.5 + R3);
#pragma unroll
    for (int c = 0; c < 3; ++c)
        atomicAdd(g.Ebar + 3 * ft + c, s * (vb[c] + (g.dt * R3) * rb[c]));
    const Vec4d e = g.E[ft];
    const double *n = g.fnhat + 3 * (size_t)f;
    const double F = -((e.x * n[0] + e.y * n[1]) + e.z * n[2]);
    if (!(F > 0.0) || wb == 0.0)
        return;
    double dF, dphi;
    fn_dlog(F, g.wf[f], g.fn_model, dF, dphi);
    atomicAdd(g.gwf + f, wb * dphi);
    const double Fb = wb * dF;
#pragma unroll
    for (int c = 0; c < 3; ++c)
        atomicAdd(g.Ebar + 3 * ft + c, -Fb * n[c]);
}

template <typename R> cudaError_t launch_adjoint_sp(cudaStream_t s, const AdjStep<R> &g)
{
    if (g.n <= 0)
        return cudaSuccess;
    k_adjoint_sp<R><<<(unsigned)((g.n + 255) / 256), 256, 0, s>>>(g);
    return cudaGetLastError();
}

#define PF_INSTANTIATE(R)                                                                      \
    template cudaError_t launch_inject_count<R>(cudaStream_t, int, MeshView<R>, RunConst,      \
                                                const long long *, int *, int *);              \
    template cudaError_t launch_inject_emit<R>(cudaStream_t, int, MeshView<R>, RunConst,       \
                                               const long long *, int, const long long *,      \
                                               Particles<R>, DevState *);                      \
    template cudaError_t launch_push_relocate<R>(cudaStream_t, int, MeshView<R>, RunConst,     \
                                                 Particles<R>, Particles<R>, int, DevState *,  \
                                                 pic_step_stats *, int *);                     \
    template cudaError_t launch_deposit<R>(cudaStream_t, int, MeshView<R>, RunConst,           \
                                           Particles<R>, int, DevState *,                      \
                                           unsigned long long *);                              \
    template cudaError_t launch_step_fused<R>(cudaStream_t, int, int, MeshView<R>, RunConst,   \
                                              const long long *, int, const long long *,       \
                                              Particles<R>,                                    \
                                              Particles<R>, int, DevState *,                   \
                                              unsigned long long *, pic_step_stats *);         \
    template cudaError_t launch_pack<R>(cudaStream_t, long long, Particles<R>, double *,       \
                                        double *, int *, long long *);                         \
    template cudaError_t launch_unpack<R>(cudaStream_t, long long, const double *,             \
                                          const double *, const int *, const long long *,      \
                                          Particles<R>);                                       \
    template cudaError_t launch_field_unpack<R>(cudaStream_t, int,                             \
                                                const typename Rec<R>::vec4 *, double *);

PF_INSTANTIATE(double)
PF_INSTANTIATE(float)
template cudaError_t launch_adjoint_sp<double>(cudaStream_t, const AdjStep<double> &);
template cudaError_t launch_adjoint_sp<float>(cudaStream_t, const AdjStep<float> &);

}  // namespace pf
