/*
 * picfem_oracle.c -- plain FP64 CPU reference of the electrostatic FEM-PIC
 * cycle of Veske et al., Phys. Rev. E 101, 053307 (arXiv 1906.08125).
 *
 * TEST INFRASTRUCTURE ONLY: the CUDA library never links, loads or reads this
 * file.  It is the slow, obviously correct statement of what one PIC step
 * computes, against which the CUDA kernels are checked.  Compile with
 * -O2 -ffp-contract=off (no fused multiply-add, so every operation below is
 * one IEEE-754 double operation in the written order).
 *
 * Where the paper is silent the fixed readings are stated where they are used:
 *   - field at an SP: E = -grad(Phi_h), constant per tetrahedron (Sec. II.B.2,
 *     P1 shape functions);
 *   - walk: greedy exit through the face opposite the most negative
 *     barycentric coordinate, ties to the lowest local index, never back
 *     through the face just entered, stop once every other coordinate is >= 0;
 *   - deposit: barycentric weights quantised to integers of 2^-S (round half
 *     to even), the fourth weight taking the remainder so that every SP
 *     deposits exactly 2^S;
 *   - random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) keyed by
 *     (seed, step, quadrangle, SP index, draw slot);
 *   - emission current: closed-form Murphy-Good Fowler-Nordheim with Forbes'
 *     2006 barrier-function approximation (the paper uses GETELEC instead);
 *   - linear solver: Jacobi-preconditioned conjugate gradients, warm-started.
 *
 * Parity unpinned: the absolute current on tip geometries (GETELEC is not
 * available and the paper's figures are missing).
 *
 * Threads: built with -fopenmp, the loops whose iterations are independent
 * (tetrahedra of the field, rows of the SpMV and of the vector updates, SPs
 * of the push and walk, quadrangles of the injection, SPs of the deposit
 * with atomic int64 adds) run in parallel; every floating-point operation
 * and its order are the same as in the serial build (dot products stay one
 * sequential sum, compaction and the injection slots keep the serial
 * order), so the two builds give bit-identical results.
 */
#include "picfem_oracle.h"

#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

struct or_ctx {
    or_params p;
    /* mesh (copied) */
    int32_t n_nodes, n_tets, n_faces;
    double *xyz;
    int32_t *tet, *nbr, *pnbr;
    uint8_t *dir;
    int32_t *face_nodes, *face_tet;
    double *wf;
    /* derived geometry */
    double *jinv;   /* 9 per tet: rows of J^-1 */
    double *x0;     /* 3 per tet: vertex 0 */
    double *det;    /* det J per tet */
    double *shift;  /* 12 per tet: periodic shift for a crossing of face k */
    double *fnhat;  /* 3 per emitting face: unit normal metal -> vacuum */
    double *farea;  /* area per emitting face */
    /* linear system on free nodes */
    int32_t n_free;
    int32_t *dof;   /* node -> free dof or -1 */
    int32_t *rowptr, *col;
    double *val, *diag, *fN;
    double *gD;     /* per node: prescribed potential on Dirichlet nodes (0 elsewhere) */
    double *fD;     /* per free dof: load of the prescribed values, -sum_j M_ij gD_j */
    /* state */
    double *phi;    /* per node, gD on Dirichlet nodes */
    double *E;      /* 3 per tet */
    int64_t *W;     /* fixed-point node charge */
    int64_t np, n_fresh;
    double *r, *v;  /* 3 per SP */
    int32_t *cell;
    int64_t *id;
    int64_t step;
};

/* ------------------------------------------------------------------ */
/* small vector helpers (written out; no fusion)                       */
/* ------------------------------------------------------------------ */
static void sub3(const double *a, const double *b, double *o)
{
    o[0] = a[0] - b[0];
    o[1] = a[1] - b[1];
    o[2] = a[2] - b[2];
}
static void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double *a, const double *b)
{
    return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}

/* ------------------------------------------------------------------ */
/* random numbers: SplitMix64 output function, keyed chain              */
/* ------------------------------------------------------------------ */
#define OR_GAMMA 0x9E3779B97F4A7C15ULL
static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
uint64_t or_splitmix64_next(uint64_t *state)
{
    *state += OR_GAMMA;
    return mix64(*state);
}
/* uniform in [0,1): the four key words are folded in one after another,
 * h <- mix(h xor word + gamma), and the top 53 bits of the result scaled. */
double or_uniform(uint64_t seed, uint64_t step, uint64_t quad, uint64_t j,
                  uint64_t slot)
{
    uint64_t w[4];
    w[0] = seed;
    w[1] = step;
    w[2] = quad;
    w[3] = (j << 8) | (slot & 0xFF);
    uint64_t h = 0;
    for (int k = 0; k < 4; ++k)
        h = mix64((h ^ w[k]) + OR_GAMMA);
    return (double)(h >> 11) * 0x1.0p-53;
}

/* ------------------------------------------------------------------ */
/* Fowler-Nordheim current density [A/m^2] (Sec. II.B.3: J_e per        */
/* quadrangle).  Murphy-Good form with Forbes' approximations           */
/* v(f) = 1 - f + (f/6) ln f and t(f) = 1 + f/9 - (f/18) ln f, with the  */
/* first and second FN constants a, b and the Schottky constant c_S^2.  */
/* f is clamped to the barrier top, f <= 1.                             */
/* ------------------------------------------------------------------ */
double or_fn_current(double F, double phi, int model)
{
    const double a = 1.541434e-6;   /* A eV V^-2           */
    const double b = 6.830890;      /* eV^-3/2 V nm^-1      */
    const double cS2 = 1.439964;    /* eV^2 V^-1 nm         */
    if (!(F > 0.0))
        return 0.0;
    double Fn = F * 1e-9; /* V/nm */
    double v = 1.0, t = 1.0;
    if (model == OR_FN_MURPHY_GOOD) {
        double f = (cS2 * Fn) / (phi * phi);
        if (f > 1.0)
            f = 1.0;
        double lf = log(f);
        v = (1.0 - f) + (f / 6.0) * lf;
        t = (1.0 + f / 9.0) - (f / 18.0) * lf;
    }
    double pre = (a * Fn * Fn) / (phi * t * t);
    double expo = -((v * b) * (phi * sqrt(phi))) / Fn;
    return (pre * exp(expo)) * 1e18; /* A/nm^2 -> A/m^2 */
}

/* ------------------------------------------------------------------ */
/* geometry of a P1 tetrahedron: J = [x1-x0 | x2-x0 | x3-x0],           */
/* J^-1 = adj(J)/det J, rows (c2 x c3, c3 x c1, c1 x c2)/det             */
/* ------------------------------------------------------------------ */
static void tet_geometry(const double *X0, const double *X1, const double *X2,
                         const double *X3, double *jinv, double *det)
{
    double c1[3], c2[3], c3[3], k1[3], k2[3], k3[3];
    sub3(X1, X0, c1);
    sub3(X2, X0, c2);
    sub3(X3, X0, c3);
    cross3(c2, c3, k1);
    cross3(c3, c1, k2);
    cross3(c1, c2, k3);
    double d = dot3(c1, k1);
    for (int i = 0; i < 3; ++i) {
        jinv[0 + i] = k1[i] / d;
        jinv[3 + i] = k2[i] / d;
        jinv[6 + i] = k3[i] / d;
    }
    *det = d;
}

/* P1 gradients: g_{1..3} are the rows of J^-1, g_0 = -(g_1 + g_2 + g_3) */
static void tet_gradients(const double *jinv, double g[4][3])
{
    for (int i = 0; i < 3; ++i) {
        g[1][i] = jinv[0 + i];
        g[2][i] = jinv[3 + i];
        g[3][i] = jinv[6 + i];
        g[0][i] = -((jinv[0 + i] + jinv[3 + i]) + jinv[6 + i]);
    }
}

/* element stiffness K_ij = int grad N_i . grad N_j = V g_i . g_j (App. B) */
void or_element_stiffness(const double *x, double *k16)
{
    double jinv[9], det, g[4][3];
    tet_geometry(x, x + 3, x + 6, x + 9, jinv, &det);
    tet_gradients(jinv, g);
    double vol = det / 6.0;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
            k16[4 * i + j] = vol * dot3(g[i], g[j]);
}

/* barycentric coordinates: lambda_k = row_k(J^-1) . (r - x0), k = 1..3,
 * lambda_0 = ((1 - lambda_1) - lambda_2) - lambda_3 */
void or_barycentric(const or_ctx *c, int32_t t, const double *r, double *lam)
{
    const double *J = c->jinv + 9 * (size_t)t;
    const double *x0 = c->x0 + 3 * (size_t)t;
    double d[3];
    sub3(r, x0, d);
    lam[1] = (J[0] * d[0] + J[1] * d[1]) + J[2] * d[2];
    lam[2] = (J[3] * d[0] + J[4] * d[1]) + J[5] * d[2];
    lam[3] = (J[6] * d[0] + J[7] * d[1]) + J[8] * d[2];
    lam[0] = ((1.0 - lam[1]) - lam[2]) - lam[3];
}

/* the three nodes of face k of tet t (face k is opposite vertex k), in
 * increasing local order */
static void face_local_nodes(int k, int *o)
{
    int n = 0;
    for (int i = 0; i < 4; ++i)
        if (i != k)
            o[n++] = i;
}

/* ------------------------------------------------------------------ */
/* context                                                             */
/* ------------------------------------------------------------------ */
or_ctx *or_create(const or_params *p)
{
    or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
    if (!c)
        return NULL;
    c->p = *p;
    return c;
}

static void free_mesh(or_ctx *c)
{
    void *bufs[] = {c->xyz, c->tet, c->nbr, c->pnbr, c->dir, c->face_nodes,
                    c->face_tet, c->wf, c->jinv, c->x0, c->det, c->shift,
                    c->fnhat, c->farea, c->dof, c->rowptr, c->col, c->val,
                    c->diag, c->fN, c->phi, c->E, c->W, c->r, c->v, c->cell,
                    c->id, c->gD, c->fD};
    for (size_t i = 0; i < sizeof(bufs) / sizeof(bufs[0]); ++i)
        free(bufs[i]);
}

void or_destroy(or_ctx *c)
{
    if (!c)
        return;
    free_mesh(c);
    free(c);
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* position of column j in row i of the CSR pattern (binary search) */
static int64_t csr_find(const or_ctx *c, int32_t i, int32_t j)
{
    int64_t lo = c->rowptr[i], hi = c->rowptr[i + 1] - 1;
    while (lo <= hi) {
        int64_t m = (lo + hi) / 2;
        if (c->col[m] == j)
            return m;
        if (c->col[m] < j)
            lo = m + 1;
        else
            hi = m - 1;
    }
    return -1;
}

int or_mesh_load(or_ctx *c, int32_t n_nodes, const double *xyz,
                 int32_t n_tets, const int32_t *tet, const int32_t *nbr,
                 const int32_t *periodic_nbr, const uint8_t *node_dirichlet,
                 int32_t n_faces, const int32_t *face_nodes,
                 const int32_t *face_tet, const double *work_function_eV)
{
    if (n_nodes < 4 || n_tets < 1 || n_faces < 0 || (int64_t)n_faces * 3 >= (1 << 24))
        return OR_ERR_ARG;
    free_mesh(c);
    memset(&c->n_nodes, 0, sizeof(or_ctx) - offsetof(or_ctx, n_nodes));
    c->n_nodes = n_nodes;
    c->n_tets = n_tets;
    c->n_faces = n_faces;
    size_t N = (size_t)n_nodes, T = (size_t)n_tets, F = (size_t)n_faces;
    c->xyz = malloc(sizeof(double) * 3 * N);
    c->tet = malloc(sizeof(int32_t) * 4 * T);
    c->nbr = malloc(sizeof(int32_t) * 4 * T);
    c->pnbr = malloc(sizeof(int32_t) * 4 * T);
    c->dir = malloc(N);
    c->face_nodes = malloc(sizeof(int32_t) * 3 * (F + 1));
    c->face_tet = malloc(sizeof(int32_t) * (F + 1));
    c->wf = malloc(sizeof(double) * (F + 1));
    memcpy(c->xyz, xyz, sizeof(double) * 3 * N);
    memcpy(c->tet, tet, sizeof(int32_t) * 4 * T);
    memcpy(c->nbr, nbr, sizeof(int32_t) * 4 * T);
    if (periodic_nbr)
        memcpy(c->pnbr, periodic_nbr, sizeof(int32_t) * 4 * T);
    else
        for (size_t i = 0; i < 4 * T; ++i)
            c->pnbr[i] = -1;
    memcpy(c->dir, node_dirichlet, N);
    if (F) {
        memcpy(c->face_nodes, face_nodes, sizeof(int32_t) * 3 * F);
        memcpy(c->face_tet, face_tet, sizeof(int32_t) * F);
        memcpy(c->wf, work_function_eV, sizeof(double) * F);
    }

    /* validation: node indices, neighbour symmetry, boundary codes */
    for (size_t t = 0; t < T; ++t)
        for (int k = 0; k < 4; ++k) {
            int32_t a = c->tet[4 * t + k];
            if (a < 0 || a >= n_nodes)
                return OR_ERR_MESH;
            int32_t b = c->nbr[4 * t + k];
            if (b >= n_tets || b < OR_SIDE)
                return OR_ERR_MESH;
            if (b >= 0) {
                int back = 0;
                for (int m = 0; m < 4; ++m)
                    back += c->nbr[4 * (size_t)b + m] == (int32_t)t;
                if (back != 1)
                    return OR_ERR_MESH;
            }
            if (b == OR_SIDE) {
                int32_t pp = c->pnbr[4 * t + k];
                if (pp < 0 || pp >= n_tets)
                    return OR_ERR_MESH;
            }
        }
    for (size_t f = 0; f < F; ++f) {
        if (c->face_tet[f] < 0 || c->face_tet[f] >= n_tets)
            return OR_ERR_MESH;
        if (!(c->wf[f] > 0.0) || !isfinite(c->wf[f]))
            return OR_ERR_ARG;
        for (int k = 0; k < 3; ++k)
            if (c->face_nodes[3 * f + k] < 0 || c->face_nodes[3 * f + k] >= n_nodes)
                return OR_ERR_MESH;
    }

    /* geometry */
    c->jinv = malloc(sizeof(double) * 9 * T);
    c->x0 = malloc(sizeof(double) * 3 * T);
    c->det = malloc(sizeof(double) * T);
    for (size_t t = 0; t < T; ++t) {
        const int32_t *v = c->tet + 4 * t;
        tet_geometry(c->xyz + 3 * (size_t)v[0], c->xyz + 3 * (size_t)v[1],
                     c->xyz + 3 * (size_t)v[2], c->xyz + 3 * (size_t)v[3],
                     c->jinv + 9 * t, c->det + t);
        if (!(c->det[t] > 0.0))
            return OR_ERR_MESH;
        for (int i = 0; i < 3; ++i)
            c->x0[3 * t + i] = c->xyz[3 * (size_t)v[0] + i];
    }

    /* periodic shifts: a side face whose three nodes share x = xmin gets
     * +Lx (the SP reappears at the opposite side, Sec. II.B.1), x = xmax
     * gets -Lx, and likewise in y. */
    double lo[3], hi[3];
    for (int i = 0; i < 3; ++i)
        lo[i] = hi[i] = c->xyz[i];
    for (size_t n = 0; n < N; ++n)
        for (int i = 0; i < 3; ++i) {
            double q = c->xyz[3 * n + i];
            if (q < lo[i]) lo[i] = q;
            if (q > hi[i]) hi[i] = q;
        }
    c->shift = calloc(12 * T, sizeof(double));
    for (size_t t = 0; t < T; ++t)
        for (int k = 0; k < 4; ++k) {
            if (c->nbr[4 * t + k] != OR_SIDE)
                continue;
            int ln[3];
            face_local_nodes(k, ln);
            int found = 0;
            for (int ax = 0; ax < 2 && !found; ++ax) {
                int at_lo = 1, at_hi = 1;
                for (int m = 0; m < 3; ++m) {
                    double q = c->xyz[3 * (size_t)c->tet[4 * t + ln[m]] + ax];
                    at_lo &= q == lo[ax];
                    at_hi &= q == hi[ax];
                }
                if (at_lo) {
                    c->shift[12 * t + 3 * k + ax] = hi[ax] - lo[ax];
                    found = 1;
                } else if (at_hi) {
                    c->shift[12 * t + 3 * k + ax] = -(hi[ax] - lo[ax]);
                    found = 1;
                }
            }
            if (!found)
                return OR_ERR_MESH;
        }

    /* emitting-face geometry: normal (B-A) x (C-A) points into the vacuum */
    c->fnhat = malloc(sizeof(double) * 3 * (F + 1));
    c->farea = malloc(sizeof(double) * (F + 1));
    for (size_t f = 0; f < F; ++f) {
        const double *A = c->xyz + 3 * (size_t)c->face_nodes[3 * f + 0];
        const double *B = c->xyz + 3 * (size_t)c->face_nodes[3 * f + 1];
        const double *C = c->xyz + 3 * (size_t)c->face_nodes[3 * f + 2];
        double u[3], w[3], n[3];
        sub3(B, A, u);
        sub3(C, A, w);
        cross3(u, w, n);
        double len = sqrt(dot3(n, n));
        for (int i = 0; i < 3; ++i)
            c->fnhat[3 * f + i] = n[i] / len;
        c->farea[f] = 0.5 * len;
    }

    /* free DOFs: Dirichlet nodes (Phi = 0 on Gamma_3) are eliminated */
    c->dof = malloc(sizeof(int32_t) * N);
    int32_t nf = 0;
    for (size_t n = 0; n < N; ++n)
        c->dof[n] = c->dir[n] ? -1 : nf++;
    c->n_free = nf;

    /* CSR pattern of M on the free DOFs: row i holds every free j that
     * shares a tetrahedron with i, columns sorted */
    int32_t *cnt = calloc((size_t)nf + 1, sizeof(int32_t));
    for (size_t t = 0; t < T; ++t)
        for (int i = 0; i < 4; ++i) {
            int32_t di = c->dof[c->tet[4 * t + i]];
            if (di < 0)
                continue;
            for (int j = 0; j < 4; ++j)
                if (c->dof[c->tet[4 * t + j]] >= 0)
                    cnt[di]++;
        }
    int64_t *start = malloc(sizeof(int64_t) * ((size_t)nf + 1));
    start[0] = 0;
    for (int32_t i = 0; i < nf; ++i)
        start[i + 1] = start[i] + cnt[i];
    int32_t *raw = malloc(sizeof(int32_t) * (size_t)(start[nf] + 1));
    memset(cnt, 0, sizeof(int32_t) * ((size_t)nf + 1));
    for (size_t t = 0; t < T; ++t)
        for (int i = 0; i < 4; ++i) {
            int32_t di = c->dof[c->tet[4 * t + i]];
            if (di < 0)
                continue;
            for (int j = 0; j < 4; ++j) {
                int32_t dj = c->dof[c->tet[4 * t + j]];
                if (dj >= 0)
                    raw[start[di] + cnt[di]++] = dj;
            }
        }
    c->rowptr = malloc(sizeof(int32_t) * ((size_t)nf + 1));
    c->col = malloc(sizeof(int32_t) * (size_t)(start[nf] + 1));
    int64_t nnz = 0;
    for (int32_t i = 0; i < nf; ++i) {
        int32_t *seg = raw + start[i];
        qsort(seg, (size_t)cnt[i], sizeof(int32_t), cmp_i32);
        c->rowptr[i] = (int32_t)nnz;
        for (int32_t k = 0; k < cnt[i]; ++k)
            if (k == 0 || seg[k] != seg[k - 1])
                c->col[nnz++] = seg[k];
    }
    c->rowptr[nf] = (int32_t)nnz;
    free(raw);
    free(start);
    free(cnt);

    /* values: M_ij = sum over elements of V g_i . g_j, accumulated in
     * increasing element order (App. B, eq. poisson_mat) */
    c->val = calloc((size_t)nnz + 1, sizeof(double));
    for (size_t t = 0; t < T; ++t) {
        double g[4][3];
        tet_gradients(c->jinv + 9 * t, g);
        double vol = c->det[t] / 6.0;
        for (int i = 0; i < 4; ++i) {
            int32_t di = c->dof[c->tet[4 * t + i]];
            if (di < 0)
                continue;
            for (int j = 0; j < 4; ++j) {
                int32_t dj = c->dof[c->tet[4 * t + j]];
                if (dj < 0)
                    continue;
                c->val[csr_find(c, di, dj)] += vol * dot3(g[i], g[j]);
            }
        }
    }
    c->diag = malloc(sizeof(double) * ((size_t)nf + 1));
    for (int32_t i = 0; i < nf; ++i)
        c->diag[i] = c->val[csr_find(c, i, i)];

    /* Neumann load: int_{Gamma_1} N_i E0 dGamma = E0 A / 3 per vertex of
     * each top triangle, in increasing (tet, face) order */
    c->fN = calloc((size_t)nf + 1, sizeof(double));
    for (size_t t = 0; t < T; ++t)
        for (int k = 0; k < 4; ++k) {
            if (c->nbr[4 * t + k] != OR_TOP)
                continue;
            int ln[3];
            face_local_nodes(k, ln);
            const double *A = c->xyz + 3 * (size_t)c->tet[4 * t + ln[0]];
            const double *B = c->xyz + 3 * (size_t)c->tet[4 * t + ln[1]];
            const double *C = c->xyz + 3 * (size_t)c->tet[4 * t + ln[2]];
            double u[3], w[3], n[3];
            sub3(B, A, u);
            sub3(C, A, w);
            cross3(u, w, n);
            double area = 0.5 * sqrt(dot3(n, n));
            double contrib = (c->p.E0 * area) / 3.0;
            for (int m = 0; m < 3; ++m) {
                int32_t d = c->dof[c->tet[4 * t + ln[m]]];
                if (d >= 0)
                    c->fN[d] += contrib;
            }
        }

    c->gD = calloc(N, sizeof(double));
    c->fD = calloc((size_t)nf + 1, sizeof(double));
    c->phi = calloc(N, sizeof(double));
    c->E = calloc(3 * T, sizeof(double));
    c->W = calloc(N, sizeof(int64_t));
    size_t cap = (size_t)(c->p.capacity > 0 ? c->p.capacity : 1);
    c->r = malloc(sizeof(double) * 3 * cap);
    c->v = malloc(sizeof(double) * 3 * cap);
    c->cell = malloc(sizeof(int32_t) * cap);
    c->id = malloc(sizeof(int64_t) * cap);
    c->np = 0;
    c->n_fresh = 0;
    c->step = 0;
    return OR_OK;
}

int32_t or_n_free(const or_ctx *c) { return c->n_free; }
int64_t or_nnz(const or_ctx *c) { return c->rowptr[c->n_free]; }

void or_geometry(const or_ctx *c, double *jinv9, double *x0_3, double *vol)
{
    for (int32_t t = 0; t < c->n_tets; ++t) {
        if (jinv9)
            memcpy(jinv9 + 9 * (size_t)t, c->jinv + 9 * (size_t)t, 9 * sizeof(double));
        if (x0_3)
            memcpy(x0_3 + 3 * (size_t)t, c->x0 + 3 * (size_t)t, 3 * sizeof(double));
        if (vol)
            vol[t] = c->det[t] / 6.0;
    }
}

void or_matrix(const or_ctx *c, int32_t *dof_of_node, int32_t *rowptr,
               int32_t *col, double *val, double *f_neumann)
{
    int64_t nnz = c->rowptr[c->n_free];
    if (dof_of_node)
        memcpy(dof_of_node, c->dof, sizeof(int32_t) * (size_t)c->n_nodes);
    if (rowptr)
        memcpy(rowptr, c->rowptr, sizeof(int32_t) * ((size_t)c->n_free + 1));
    if (col)
        memcpy(col, c->col, sizeof(int32_t) * (size_t)nnz);
    if (val)
        memcpy(val, c->val, sizeof(double) * (size_t)nnz);
    if (f_neumann)
        memcpy(f_neumann, c->fN, sizeof(double) * (size_t)c->n_free);
}

/* ------------------------------------------------------------------ */
/* field: E_t = -sum_i Phi_{v_i} g_i, constant in each tetrahedron       */
/* ------------------------------------------------------------------ */
static void compute_field(or_ctx *c)
{
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < (int64_t)c->n_tets; ++t) {
        double g[4][3];
        tet_gradients(c->jinv + 9 * t, g);
        const int32_t *v = c->tet + 4 * t;
        for (int i = 0; i < 3; ++i) {
            double s = ((c->phi[v[0]] * g[0][i] + c->phi[v[1]] * g[1][i]) +
                        c->phi[v[2]] * g[2][i]) + c->phi[v[3]] * g[3][i];
            c->E[3 * t + i] = -s;
        }
    }
}

void or_get_potential(const or_ctx *c, double *phi)
{
    memcpy(phi, c->phi, sizeof(double) * (size_t)c->n_nodes);
}
void or_set_potential(or_ctx *c, const double *phi)
{
    for (int32_t n = 0; n < c->n_nodes; ++n)
        c->phi[n] = c->dir[n] ? c->gD[n] : phi[n];
    compute_field(c);
}

/* Prescribed potential on the Dirichlet nodes (App. B: the weak form is taken
 * for Phi = Phi_free + Phi_D with Phi_D carrying the prescribed values, so the
 * free equations gain the load -sum_{j Dirichlet} M_ij g_j).  M_ij is summed
 * element by element, V_e g_i . g_j, in increasing element order and, within
 * an element, in increasing local index j. */
void or_set_dirichlet(or_ctx *c, const double *g)
{
    for (int32_t n = 0; n < c->n_nodes; ++n)
        c->gD[n] = c->dir[n] ? g[n] : 0.0;
    memset(c->fD, 0, sizeof(double) * ((size_t)c->n_free + 1));
    for (size_t t = 0; t < (size_t)c->n_tets; ++t) {
        double gr[4][3];
        tet_gradients(c->jinv + 9 * t, gr);
        double vol = c->det[t] / 6.0;
        for (int i = 0; i < 4; ++i) {
            int32_t di = c->dof[c->tet[4 * t + i]];
            if (di < 0)
                continue;
            for (int j = 0; j < 4; ++j) {
                int32_t nj = c->tet[4 * t + j];
                if (!c->dir[nj])
                    continue;
                c->fD[di] = c->fD[di] - (vol * dot3(gr[i], gr[j])) * c->gD[nj];
            }
        }
    }
    for (int32_t n = 0; n < c->n_nodes; ++n)
        if (c->dir[n])
            c->phi[n] = c->gD[n];
    compute_field(c);
}
void or_get_field(const or_ctx *c, double *E3)
{
    memcpy(E3, c->E, sizeof(double) * 3 * (size_t)c->n_tets);
}
int64_t or_num_particles(const or_ctx *c) { return c->np; }
void or_get_particles(const or_ctx *c, double *r3, double *v3, int32_t *cell,
                      int64_t *id)
{
    size_t n = (size_t)c->np;
    if (r3) memcpy(r3, c->r, sizeof(double) * 3 * n);
    if (v3) memcpy(v3, c->v, sizeof(double) * 3 * n);
    if (cell) memcpy(cell, c->cell, sizeof(int32_t) * n);
    if (id) memcpy(id, c->id, sizeof(int64_t) * n);
}
int or_set_particles(or_ctx *c, int64_t n, const double *r3, const double *v3,
                     const int32_t *cell, const int64_t *id)
{
    if (n < 0 || n > c->p.capacity)
        return OR_ERR_CAPACITY;
    for (int64_t i = 0; i < n; ++i)
        if (cell[i] < 0 || cell[i] >= c->n_tets)
            return OR_ERR_ARG;
    memcpy(c->r, r3, sizeof(double) * 3 * (size_t)n);
    memcpy(c->v, v3, sizeof(double) * 3 * (size_t)n);
    memcpy(c->cell, cell, sizeof(int32_t) * (size_t)n);
    memcpy(c->id, id, sizeof(int64_t) * (size_t)n);
    c->np = n;
    c->n_fresh = 0;
    return OR_OK;
}
void or_get_charge(const or_ctx *c, int64_t *W)
{
    memcpy(W, c->W, sizeof(int64_t) * (size_t)c->n_nodes);
}
int64_t or_step_index(const or_ctx *c) { return c->step; }
void or_set_step_index(or_ctx *c, int64_t step) { c->step = step; }
void or_set_work_function(or_ctx *c, const double *wf)
{
    memcpy(c->wf, wf, sizeof(double) * (size_t)c->n_faces);
}

/* ------------------------------------------------------------------ */
/* Jacobi-preconditioned CG on M Phi = f (eq. poisson_mat), warm start   */
/* from the current potential; plain sequential dot products            */
/* ------------------------------------------------------------------ */
static double vdot(const double *a, const double *b, int32_t n)
{
    double s = 0.0;
    for (int32_t i = 0; i < n; ++i)
        s += a[i] * b[i];
    return s;
}
static void spmv(const or_ctx *c, const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < c->n_free; ++i) {
        double s = 0.0;
        for (int32_t k = c->rowptr[i]; k < c->rowptr[i + 1]; ++k)
            s += c->val[k] * x[c->col[k]];
        y[i] = s;
    }
}

static int pcg(or_ctx *c, const double *f, double *x, int32_t *iters,
               double *relres)
{
    int32_t n = c->n_free;
    size_t sz = sizeof(double) * ((size_t)n + 1);
    double *r = malloc(sz), *z = malloc(sz), *p = malloc(sz), *Ap = malloc(sz);
    int status = OR_OK;
    spmv(c, x, Ap);
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) {
        r[i] = f[i] - Ap[i];
        z[i] = r[i] / c->diag[i];
        p[i] = z[i];
    }
    double ff = vdot(f, f, n);
    double rz = vdot(r, z, n);
    double rr = vdot(r, r, n);
    int32_t it = 0;
    if (ff == 0.0) {
        for (int32_t i = 0; i < n; ++i)
            x[i] = 0.0;
        rr = 0.0;
        ff = 1.0;
    }
    double tol = c->p.pcg_rtol * sqrt(ff);
    while (sqrt(rr) > tol) {
        if (it >= c->p.pcg_max_iter) {
            status = OR_ERR_NOT_CONVERGED;
            break;
        }
        spmv(c, p, Ap);
        double alpha = rz / vdot(p, Ap, n);
#pragma omp parallel for schedule(static)
        for (int32_t i = 0; i < n; ++i) {
            x[i] = x[i] + alpha * p[i];
            r[i] = r[i] - alpha * Ap[i];
            z[i] = r[i] / c->diag[i];
        }
        double rz_new = vdot(r, z, n);
        rr = vdot(r, r, n);
        double beta = rz_new / rz;
        rz = rz_new;
#pragma omp parallel for schedule(static)
        for (int32_t i = 0; i < n; ++i)
            p[i] = z[i] + beta * p[i];
        ++it;
    }
    if (iters)
        *iters = it;
    if (relres)
        *relres = sqrt(rr) / sqrt(ff);
    free(r);
    free(z);
    free(p);
    free(Ap);
    return status;
}

/* M x = f for a right-hand side of the caller's (free DOFs, the numbering of
 * or_matrix), by the same Jacobi-PCG from the x given, to ||f - M x|| <=
 * rtol ||f|| (App. B, eq. poisson_mat); used by the reverse pass of the
 * adjoint reference on systems too large for a direct factorisation */
int or_solve(or_ctx *c, const double *f, double *x, double rtol, int32_t max_iter,
             int32_t *iters, double *relres)
{
    const double rtol0 = c->p.pcg_rtol;
    const int32_t max0 = c->p.pcg_max_iter;
    c->p.pcg_rtol = rtol;
    c->p.pcg_max_iter = max_iter;
    int status = pcg(c, f, x, iters, relres);
    c->p.pcg_rtol = rtol0;
    c->p.pcg_max_iter = max0;
    return status;
}

/* RHS f_i = (q w_sp / eps) sum_j N_i(r_j) + int_{Gamma_1} N_i E0 (eq.
 * poisson_rhs); the particle sum is the fixed-point W_i * 2^-S */
int or_poisson_solve(or_ctx *c, int32_t *iters, double *relres)
{
    int32_t n = c->n_free;
    double *f = malloc(sizeof(double) * ((size_t)n + 1));
    double *x = malloc(sizeof(double) * ((size_t)n + 1));
    double coef = (c->p.q * c->p.w_sp) / c->p.eps0;
#pragma omp parallel for schedule(static)
    for (int32_t node = 0; node < c->n_nodes; ++node) {
        int32_t d = c->dof[node];
        if (d < 0)
            continue;
        f[d] = (coef * ldexp((double)c->W[node], -c->p.quant_bits) + c->fN[d]) + c->fD[d];
        x[d] = c->phi[node];
    }
    int st = pcg(c, f, x, iters, relres);
    for (int32_t node = 0; node < c->n_nodes; ++node) {
        int32_t d = c->dof[node];
        c->phi[node] = d < 0 ? c->gD[node] : x[d];
    }
    compute_field(c);
    free(f);
    free(x);
    return st;
}

int or_init_potential(or_ctx *c, int32_t *iters, double *relres)
{
    for (int32_t n = 0; n < c->n_nodes; ++n)
        c->phi[n] = c->dir[n] ? c->gD[n] : 0.0;
    memset(c->W, 0, sizeof(int64_t) * (size_t)c->n_nodes);
    return or_poisson_solve(c, iters, relres);
}

/* ------------------------------------------------------------------ */
/* injection (Sec. II.B.3 eqs. nsp, rnd_nsp, sp_velocity,                */
/* sp_displacement; App. E eq. rnd_point)                                */
/* ------------------------------------------------------------------ */
/* the emission of every quadrangle (F, J_FN and n_sp of eq. nsp) from the
 * per-tetrahedron field E3 [n_tets*3]: the context's own field, or any
 * other field of the same mesh (e.g. one read from another code, to
 * evaluate where its rounding decisions of eq. rnd_nsp may differ) */
void or_quad_emission_field(const or_ctx *c, const double *E3, double *Fout, double *Jout,
                            double *nout)
{
#pragma omp parallel for schedule(static)
    for (int32_t f = 0; f < c->n_faces; ++f) {
        const double *E = E3 + 3 * (size_t)c->face_tet[f];
        double F = -dot3(E, c->fnhat + 3 * (size_t)f);
        if (!(F > 0.0))
            F = 0.0;
        double J = or_fn_current(F, c->wf[f], c->p.fn_model);
        double Aq = c->farea[f] / 3.0;
        double nsp = ((J * Aq) * c->p.dt) / (c->p.e_charge * c->p.w_sp);
        for (int k = 0; k < 3; ++k) {
            if (Fout) Fout[3 * (size_t)f + k] = F;
            if (Jout) Jout[3 * (size_t)f + k] = J;
            if (nout) nout[3 * (size_t)f + k] = nsp;
        }
    }
}

void or_quad_emission(const or_ctx *c, double *Fout, double *Jout, double *nout)
{
    or_quad_emission_field(c, c->E, Fout, Jout, nout);
}

#define OR_ID_QUAD_SHIFT 18
#define OR_ID_STEP_SHIFT 42
#define OR_MAX_PER_QUAD ((int64_t)1 << OR_ID_QUAD_SHIFT)
#define OR_MAX_ATTEMPTS 64

int or_inject(or_ctx *c, int64_t step, int64_t *n_injected)
{
    int64_t nq = 3 * (int64_t)c->n_faces;
    double *nsp = malloc(sizeof(double) * (size_t)(nq + 1));
    int64_t *cnt = malloc(sizeof(int64_t) * (size_t)(nq + 1));
    or_quad_emission(c, NULL, NULL, nsp);
    int64_t total = 0;
    for (int64_t q = 0; q < nq; ++q) {
        double R0 = or_uniform(c->p.seed, (uint64_t)step, (uint64_t)q, 0, 0);
        double fl = floor(nsp[q]);
        double frac = nsp[q] - fl;
        cnt[q] = (int64_t)fl + (R0 >= frac ? 0 : 1);
        if (cnt[q] >= OR_MAX_PER_QUAD || !(nsp[q] >= 0.0)) {
            free(nsp);
            free(cnt);
            return OR_ERR_CAPACITY;
        }
        total += cnt[q];
    }
    if (c->np + total > c->p.capacity) {
        free(nsp);
        free(cnt);
        return OR_ERR_CAPACITY;
    }
    double qmdt = c->p.q_over_m * c->p.dt;
    double dt = c->p.dt;
    int status = OR_OK;
    /* slot of the first SP of each quadrangle: quadrangles in order, then j */
    int64_t *slot = malloc(sizeof(int64_t) * (size_t)(nq + 1));
    slot[0] = c->np;
    for (int64_t q = 0; q < nq; ++q)
        slot[q + 1] = slot[q] + cnt[q];
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < nq; ++q) {
        if (cnt[q] == 0)
            continue;
        int32_t f = (int32_t)(q / 3);
        int vtx = (int)(q % 3);
        const double *V = c->xyz + 3 * (size_t)c->face_nodes[3 * f + vtx];
        const double *Vn = c->xyz + 3 * (size_t)c->face_nodes[3 * f + (vtx + 1) % 3];
        const double *Vp = c->xyz + 3 * (size_t)c->face_nodes[3 * f + (vtx + 2) % 3];
        double m1[3], m2[3];
        for (int i = 0; i < 3; ++i) {
            m1[i] = (V[i] + Vn[i]) * 0.5;
            m2[i] = (V[i] + Vp[i]) * 0.5;
        }
        const double *E = c->E + 3 * (size_t)c->face_tet[f];
        for (int64_t j = 0; j < cnt[q]; ++j) {
            double R1 = 0.0, R2 = 0.0;
            int ok = 0;
            for (int a = 0; a < OR_MAX_ATTEMPTS && !ok; ++a) {
                R1 = or_uniform(c->p.seed, (uint64_t)step, (uint64_t)q, (uint64_t)j, (uint64_t)(1 + 2 * a));
                R2 = or_uniform(c->p.seed, (uint64_t)step, (uint64_t)q, (uint64_t)j, (uint64_t)(2 + 2 * a));
                /* triangle barycentrics of V + R1 (m1 - V) + R2 (m2 - V) */
                double l_next = R1 * 0.5, l_prev = R2 * 0.5;
                double l_v = (1.0 - l_next) - l_prev;
                ok = l_v >= l_next && l_v >= l_prev;
            }
            if (!ok) {
#pragma omp atomic write
                status = OR_ERR_ARG;
                break;
            }
            double R3 = or_uniform(c->p.seed, (uint64_t)step, (uint64_t)q, (uint64_t)j, 255);
            double s = qmdt * (0.5 + R3);
            double tR = dt * R3;
            size_t k = (size_t)(slot[q] + j);
            for (int i = 0; i < 3; ++i) {
                double pnt = (V[i] + R1 * (m1[i] - V[i])) + R2 * (m2[i] - V[i]);
                double v0 = s * E[i];
                c->v[3 * k + i] = v0;
                c->r[3 * k + i] = pnt + v0 * tR;
            }
            c->cell[k] = c->face_tet[f];
            c->id[k] = (step << OR_ID_STEP_SHIFT) | (q << OR_ID_QUAD_SHIFT) | j;
        }
    }
    if (status == OR_OK) {
        c->np += total;
        c->n_fresh += total;
    }
    if (n_injected)
        *n_injected = total;
    free(slot);
    free(nsp);
    free(cnt);
    return status;
}

/* ------------------------------------------------------------------ */
/* relocation by the neighbour walk (Sec. II.B.2)                        */
/* ------------------------------------------------------------------ */
enum { FATE_ALIVE = 0, FATE_COLLECTED = 1, FATE_ABSORBED = 2 };

/* local index of the face of tet `into` that is shared with tet `from` */
static int entry_face(const or_ctx *c, int32_t into, int32_t from, int periodic,
                      const double *shift_used)
{
    for (int m = 0; m < 4; ++m) {
        if (!periodic && c->nbr[4 * (size_t)into + m] == from)
            return m;
        if (periodic && c->nbr[4 * (size_t)into + m] == OR_SIDE &&
            c->pnbr[4 * (size_t)into + m] == from) {
            const double *s = c->shift + 12 * (size_t)into + 3 * m;
            if (s[0] == -shift_used[0] && s[1] == -shift_used[1])
                return m;
        }
    }
    return -1;
}

static int walk(const or_ctx *c, double *r, int32_t *cell, int *fate,
                int32_t *len, int64_t *wraps)
{
    int32_t t = *cell;
    int entered = -1;
    int32_t steps = 0;
    for (;;) {
        double lam[4];
        or_barycentric(c, t, r, lam);
        int k = -1;
        double m = 0.0;
        for (int i = 0; i < 4; ++i) {
            if (i == entered)
                continue;
            if (k < 0 || lam[i] < m) {
                k = i;
                m = lam[i];
            }
        }
        if (m >= 0.0) {
            *fate = FATE_ALIVE;
            break;
        }
        if (steps >= c->p.walk_max_steps) {
            *cell = t;
            *len = steps;
            return OR_ERR_WALK_LIMIT;
        }
        ++steps;
        int32_t nb = c->nbr[4 * (size_t)t + k];
        if (nb == OR_TOP) {
            *fate = FATE_COLLECTED;
            break;
        }
        if (nb == OR_CATHODE) {
            *fate = FATE_ABSORBED;
            break;
        }
        if (nb == OR_SIDE) {
            const double *s = c->shift + 12 * (size_t)t + 3 * k;
            for (int i = 0; i < 3; ++i)
                r[i] = r[i] + s[i];
            int32_t pt = c->pnbr[4 * (size_t)t + k];
            entered = entry_face(c, pt, t, 1, s);
            t = pt;
            if (wraps)
                ++*wraps;
            continue;
        }
        entered = entry_face(c, nb, t, 0, NULL);
        t = nb;
    }
    *cell = t;
    *len = steps;
    return OR_OK;
}

int or_locate(const or_ctx *c, int64_t n, double *r3, int32_t *cell,
              int32_t *fate, int32_t *walk_len)
{
    for (int64_t i = 0; i < n; ++i) {
        int fa = 0;
        int32_t len = 0;
        int st = walk(c, r3 + 3 * i, cell + i, &fa, &len, NULL);
        if (st != OR_OK)
            return st;
        if (fate) fate[i] = fa;
        if (walk_len) walk_len[i] = len;
    }
    return OR_OK;
}

/* leapfrog (eqs. leapfrog1-3) with the closing half kick of step k-1 and
 * the opening half kick of step k merged into one kick by 2Q E_k,
 * Q = (q/m) dt / 2; then the drift r += dt v; then the walk.  SPs injected
 * in this step are not kicked (they were injected between leapfrog1 and
 * leapfrog2) but drift. */
int or_push_relocate(or_ctx *c, int64_t step, or_stats *st)
{
    (void)step;
    double qmdt = c->p.q_over_m * c->p.dt;
    double dt = c->p.dt;
    int64_t n_old = c->np - c->n_fresh;
    int64_t collected = 0, absorbed = 0, wraps = 0, crossings = 0;
    int32_t max_walk = 0;
    int64_t out = 0;
    int status = OR_OK;
    /* every SP on its own (kick, drift, walk), in place ... */
    int8_t *fate = malloc((size_t)c->np + 1);
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : wraps, crossings) reduction(max : max_walk)
    for (int64_t k = 0; k < c->np; ++k) {
        double *r = c->r + 3 * k, *v = c->v + 3 * k;
        if (k < n_old) {
            const double *E = c->E + 3 * (size_t)c->cell[k];
            for (int i = 0; i < 3; ++i)
                v[i] = v[i] + qmdt * E[i];
        }
        for (int i = 0; i < 3; ++i)
            r[i] = r[i] + dt * v[i];
        int fa = 0;
        int32_t len = 0;
        int32_t t = c->cell[k];
        int64_t w = 0;
        int s = walk(c, r, &t, &fa, &len, &w);
        if (s != OR_OK) {
#pragma omp atomic write
            status = s;
            fa = FATE_ALIVE;
        }
        wraps += w;
        crossings += len;
        if (len > max_walk)
            max_walk = len;
        c->cell[k] = t;
        fate[k] = (int8_t)fa;
    }
    if (status != OR_OK) {
        free(fate);
        return status;
    }
    /* ... then the survivors kept in order */
    for (int64_t k = 0; k < c->np; ++k) {
        if (fate[k] == FATE_COLLECTED) {
            ++collected;
            continue;
        }
        if (fate[k] == FATE_ABSORBED) {
            ++absorbed;
            continue;
        }
        if (out != k) {
            for (int i = 0; i < 3; ++i) {
                c->r[3 * out + i] = c->r[3 * k + i];
                c->v[3 * out + i] = c->v[3 * k + i];
            }
            c->cell[out] = c->cell[k];
            c->id[out] = c->id[k];
        }
        ++out;
    }
    free(fate);
    c->np = out;
    c->n_fresh = 0;
    if (st) {
        st->collected = collected;
        st->absorbed = absorbed;
        st->wrapped = wraps;
        st->crossings = crossings;
        st->max_walk = max_walk;
        st->alive = out;
        st->collected_charge = (c->p.q * c->p.w_sp) * (double)collected;
    }
    return OR_OK;
}

/* deposit (eq. poisson_rhs): each SP adds N_i(r_j) to the four nodes of its
 * tetrahedron, as integers of 2^-S: w_i = rint(lambda_i 2^S) for i = 0..2,
 * w_3 = 2^S - w_0 - w_1 - w_2 */
int or_deposit(or_ctx *c)
{
    int S = c->p.quant_bits;
    int64_t one = (int64_t)1 << S;
    memset(c->W, 0, sizeof(int64_t) * (size_t)c->n_nodes);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < c->np; ++k) {
        double lam[4];
        int32_t t = c->cell[k];
        or_barycentric(c, t, c->r + 3 * k, lam);
        int64_t w0 = llrint(ldexp(lam[0], S));
        int64_t w1 = llrint(ldexp(lam[1], S));
        int64_t w2 = llrint(ldexp(lam[2], S));
        int64_t w3 = ((one - w0) - w1) - w2;
        const int32_t *v = c->tet + 4 * (size_t)t;
        /* int64 sums: the same totals in any order */
#pragma omp atomic
        c->W[v[0]] += w0;
#pragma omp atomic
        c->W[v[1]] += w1;
#pragma omp atomic
        c->W[v[2]] += w2;
#pragma omp atomic
        c->W[v[3]] += w3;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Monte Carlo binary collisions between SPs of the same cell (App. F,   */
/* after Takizuka & Abe 1977): group the SPs by cell, pair them at       */
/* random, collide each pair elastically with a Gaussian scattering      */
/* angle.                                                                */
/* ------------------------------------------------------------------ */
#define OR_PI 3.14159265358979323846           /* pi, rounded to double */
#define OR_COLL_DOMAIN ((uint64_t)1 << 40)  /* key words never used by a quadrangle */
#define OR_SHUF_DOMAIN ((uint64_t)1 << 41)

/* the keyed chain of or_uniform, all 64 bits */
static uint64_t hash4(uint64_t w0, uint64_t w1, uint64_t w2, uint64_t w3)
{
    uint64_t w[4] = {w0, w1, w2, w3};
    uint64_t h = 0;
    for (int k = 0; k < 4; ++k)
        h = mix64((h ^ w[k]) + OR_GAMMA);
    return h;
}

typedef struct {
    int32_t cell;
    uint64_t key;
    int64_t id;
    int64_t idx;
} coll_rec;

static int cmp_coll(const void *pa, const void *pb)
{
    const coll_rec *a = pa, *b = pb;
    if (a->cell != b->cell)
        return a->cell < b->cell ? -1 : 1;
    if (a->key != b->key)
        return a->key < b->key ? -1 : 1;
    return a->id < b->id ? -1 : (a->id > b->id);
}

/* One elastic collision (eqs. vel12, scat_vel, rot_mat, sin_theta): the
 * relative velocity w = u_a - u_b turns by theta about a random azimuth phi,
 * w' = w + M(theta, phi) w, and v_{a,b} = u_{a,b} +- M w / 2 (equal masses).
 * delta = tan(theta/2) ~ N(0, <delta^2>) with <delta^2> = C / |w|^3
 * (eq. variance, C holding everything but the speed). */
static void collide_pair(double *va, double *vb, double C, double U1, double U2, double U3)
{
    double w[3] = {va[0] - vb[0], va[1] - vb[1], va[2] - vb[2]};
    double u = sqrt(dot3(w, w));
    if (!(u > 0.0))
        return;
    double var = C / ((u * u) * u);
    double delta = sqrt(var) * (sqrt(-2.0 * log(1.0 - U1)) * cos((2.0 * OR_PI) * U2));
    double phi = (2.0 * OR_PI) * U3;
    double dd = delta * delta;
    double s = (2.0 * delta) / (1.0 + dd);       /* sin theta     */
    double c1 = (2.0 * dd) / (1.0 + dd);         /* 1 - cos theta */
    double sp = sin(phi), cp = cos(phi);
    double wp = sqrt(w[0] * w[0] + w[1] * w[1]);
    double d[3];
    if (wp > 0.0) {
        double a = (s * sp) * (u / wp);
        double bx = (s * cp) * (w[0] / wp), by = (s * cp) * (w[1] / wp);
        d[0] = (-c1 * w[0] + a * w[1]) + bx * w[2];
        d[1] = (-a * w[0] - c1 * w[1]) + by * w[2];
        d[2] = (-bx * w[0] - by * w[1]) - c1 * w[2];
    } else {
        d[0] = (s * cp) * w[2];
        d[1] = (s * sp) * w[2];
        d[2] = -c1 * w[2];
    }
    for (int i = 0; i < 3; ++i) {
        va[i] = va[i] + 0.5 * d[i];
        vb[i] = vb[i] - 0.5 * d[i];
    }
}

/* All collisions of a step.  In a cell with n >= 2 SPs, ordered by a
 * random key of (seed, step, id): an odd n collides the first three as the
 * pairs (0,1), (1,2), (2,0) with half the variance, then (3,4), (5,6), ...;
 * an even n collides (0,1), (2,3), ...  The variance uses the real electron
 * density n w_sp / V_cell and the relative speed of the pair. */
void or_collide(or_ctx *c, int64_t step)
{
    int64_t n = c->np;
    if (n < 2)
        return;
    coll_rec *rec = malloc(sizeof(coll_rec) * (size_t)n);
    for (int64_t k = 0; k < n; ++k) {
        rec[k].cell = c->cell[k];
        rec[k].id = c->id[k];
        rec[k].key = hash4(c->p.seed, (uint64_t)step, OR_SHUF_DOMAIN, (uint64_t)c->id[k]);
        rec[k].idx = k;
    }
    qsort(rec, (size_t)n, sizeof(coll_rec), cmp_coll);
    const double q = c->p.q, m = c->p.q / c->p.q_over_m;
    const double q2 = q * q;
    for (int64_t g0 = 0; g0 < n;) {
        int64_t g1 = g0;
        while (g1 < n && rec[g1].cell == rec[g0].cell)
            ++g1;
        int64_t cnt = g1 - g0;
        int32_t t = rec[g0].cell;
        if (cnt >= 2) {
            double vol = c->det[t] / 6.0;
            double nreal = (double)cnt * c->p.w_sp;
            double num = ((q2 * q2) * nreal) * (c->p.coulomb_log * c->p.dt);
            double den = ((2.0 * OR_PI) * (c->p.eps0 * c->p.eps0)) * ((m * m) * vol);
            double C = num / den;
            uint64_t kq = OR_COLL_DOMAIN | (uint64_t)t;
            int64_t ci = 0, k0 = 0;
            if (cnt & 1) {
                const int tri[3][2] = {{0, 1}, {1, 2}, {2, 0}};
                for (int e = 0; e < 3; ++e, ++ci) {
                    double *va = c->v + 3 * rec[g0 + tri[e][0]].idx;
                    double *vb = c->v + 3 * rec[g0 + tri[e][1]].idx;
                    collide_pair(va, vb, 0.5 * C, or_uniform(c->p.seed, (uint64_t)step, kq, (uint64_t)ci, 1),
                                 or_uniform(c->p.seed, (uint64_t)step, kq, (uint64_t)ci, 2),
                                 or_uniform(c->p.seed, (uint64_t)step, kq, (uint64_t)ci, 3));
                }
                k0 = 3;
            }
            for (int64_t k = k0; k + 1 < cnt; k += 2, ++ci) {
                double *va = c->v + 3 * rec[g0 + k].idx;
                double *vb = c->v + 3 * rec[g0 + k + 1].idx;
                collide_pair(va, vb, C, or_uniform(c->p.seed, (uint64_t)step, kq, (uint64_t)ci, 1),
                             or_uniform(c->p.seed, (uint64_t)step, kq, (uint64_t)ci, 2),
                             or_uniform(c->p.seed, (uint64_t)step, kq, (uint64_t)ci, 3));
            }
        }
        g0 = g1;
    }
    free(rec);
}

/* threads of the parallel loops (an OpenMP build only); returns the number
 * in use, 1 in a serial build */
int or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* one PIC step in the order of Sec. II.B: E_k (already held), kick,
 * inject, drift + walk, deposit, Poisson solve for Phi_{k+1} */
int or_step(or_ctx *c, int64_t n_steps, or_stats *stats)
{
    for (int64_t s = 0; s < n_steps; ++s) {
        or_stats st;
        memset(&st, 0, sizeof(st));
        int64_t k = c->step;
        int e = or_inject(c, k, &st.injected);
        if (e != OR_OK)
            return e;
        e = or_push_relocate(c, k, &st);
        if (e != OR_OK)
            return e;
        if (c->p.collisions)
            or_collide(c, k);
        or_deposit(c);
        e = or_poisson_solve(c, &st.pcg_iters, &st.pcg_relres);
        if (e != OR_OK)
            return e;
        c->step = k + 1;
        if (stats)
            stats[s] = st;
    }
    return OR_OK;
}
