// setup.cu -- one-time mesh kernels of mesh_load: per-tetrahedron geometry,
// stiffness-matrix values, Neumann load and emitting-face geometry.
// Compiled with --fmad=false: every expression is evaluated as written, one
// IEEE double operation at a time, so the values are reproducible bit for bit.
#include "common.cuh"

namespace pf {

// J = [x1-x0 | x2-x0 | x3-x0]; J^-1 = adj(J) / det J whose rows are
// (c2 x c3, c3 x c1, c1 x c2) / det; det = c1 . (c2 x c3).  The P1 gradients
// of N_1..N_3 are these rows and grad N_0 = -(sum of them) (App. B).
__global__ void k_geometry(int T, const double *__restrict__ xyz, const int4 *__restrict__ tet,
                           const int4 *__restrict__ nb, TetRec64 *rec64, TetRec32 *rec32,
                           double *det_out)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T)
        return;
    int4 v = tet[t];
    const double *X0 = xyz + 3 * (size_t)v.x, *X1 = xyz + 3 * (size_t)v.y;
    const double *X2 = xyz + 3 * (size_t)v.z, *X3 = xyz + 3 * (size_t)v.w;
    double c1[3], c2[3], c3[3];
    for (int i = 0; i < 3; ++i) {
        c1[i] = X1[i] - X0[i];
        c2[i] = X2[i] - X0[i];
        c3[i] = X3[i] - X0[i];
    }
    double k1[3] = {c2[1] * c3[2] - c2[2] * c3[1], c2[2] * c3[0] - c2[0] * c3[2],
                    c2[0] * c3[1] - c2[1] * c3[0]};
    double k2[3] = {c3[1] * c1[2] - c3[2] * c1[1], c3[2] * c1[0] - c3[0] * c1[2],
                    c3[0] * c1[1] - c3[1] * c1[0]};
    double k3[3] = {c1[1] * c2[2] - c1[2] * c2[1], c1[2] * c2[0] - c1[0] * c2[2],
                    c1[0] * c2[1] - c1[1] * c2[0]};
    double d = (c1[0] * k1[0] + c1[1] * k1[1]) + c1[2] * k1[2];
    TetRec64 r;
    for (int i = 0; i < 3; ++i) {
        r.j[0 + i] = k1[i] / d;
        r.j[3 + i] = k2[i] / d;
        r.j[6 + i] = k3[i] / d;
        r.x0[i] = X0[i];
    }
    int4 n = nb[t];
    r.nb[0] = n.x;
    r.nb[1] = n.y;
    r.nb[2] = n.z;
    r.nb[3] = n.w;
    rec64[t] = r;
    if (rec32) {
        TetRec32 q;
        for (int i = 0; i < 9; ++i)
            q.j[i] = (float)r.j[i];
        for (int i = 0; i < 3; ++i)
            q.x0[i] = (float)r.x0[i];
        for (int i = 0; i < 4; ++i)
            q.nb[i] = r.nb[i];
        rec32[t] = q;
    }
    det_out[t] = d;
}

__device__ __forceinline__ void grad_row(const TetRec64 &r, int i, double g[3])
{
    if (i == 0) {
        for (int c = 0; c < 3; ++c)
            g[c] = -((r.j[0 + c] + r.j[3 + c]) + r.j[6 + c]);
    } else {
        for (int c = 0; c < 3; ++c)
            g[c] = r.j[3 * (i - 1) + c];
    }
}

// M_ij = sum over elements e (increasing) of V_e grad N_i . grad N_j with
// V_e = det / 6 (App. B, eq. poisson_mat).  One thread per nonzero; the
// contributions of a nonzero are listed in increasing element order, so the
// sum is accumulated in a fixed order.
__global__ void k_matrix_values(long long nnz, const long long *__restrict__ cptr,
                                const int *__restrict__ contrib, const TetRec64 *__restrict__ rec,
                                const double *__restrict__ det, const long long *__restrict__ sell_pos,
                                const int *__restrict__ slot_row, const int *__restrict__ slot_col,
                                double *val64, float *val32, double *dinv64, float *dinv32)
{
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= nnz)
        return;
    double sum = 0.0;
    for (long long k = cptr[s]; k < cptr[s + 1]; ++k) {
        int c = contrib[k];
        int t = c >> 4, i = (c >> 2) & 3, j = c & 3;
        TetRec64 r = rec[t];
        double gi[3], gj[3];
        grad_row(r, i, gi);
        grad_row(r, j, gj);
        double vol = det[t] / 6.0;
        double dot = (gi[0] * gj[0] + gi[1] * gj[1]) + gi[2] * gj[2];
        sum += vol * dot;
    }
    long long p = sell_pos[s];
    val64[p] = sum;
    val32[p] = (float)sum;
    int row = slot_row[s];
    if (row == slot_col[s]) {
        dinv64[row] = 1.0 / sum;
        dinv32[row] = (float)(1.0 / sum);
    }
}

// Neumann load int_{Gamma_1} N_i E0 dGamma = E0 A / 3 for each vertex i of a
// top triangle (eq. poisson_rhs, second term), summed over the triangles of
// free DOF i in increasing (tetrahedron, face) order.
__global__ void k_neumann(int n_rows, const int *__restrict__ fptr, const int *__restrict__ fcontrib,
                          const int4 *__restrict__ tet, const double *__restrict__ xyz,
                          const int *__restrict__ tet_rep, const double *__restrict__ E0_rep,
                          double *fN)
{
    int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= n_rows)
        return;
    double sum = 0.0;
    for (int k = fptr[d]; k < fptr[d + 1]; ++k) {
        int c = fcontrib[k];
        int t = c >> 2, face = c & 3;
        int4 v4 = tet[t];
        int v[4] = {v4.x, v4.y, v4.z, v4.w};
        int ln[3], m = 0;
        for (int i = 0; i < 4; ++i)
            if (i != face)
                ln[m++] = v[i];
        const double *A = xyz + 3 * (size_t)ln[0], *B = xyz + 3 * (size_t)ln[1];
        const double *C = xyz + 3 * (size_t)ln[2];
        double u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        double w[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
        double n[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2],
                       u[0] * w[1] - u[1] * w[0]};
        double area = 0.5 * sqrt((n[0] * n[0] + n[1] * n[1]) + n[2] * n[2]);
        sum += (E0_rep[tet_rep[t]] * area) / 3.0;
    }
    fN[d] = sum;
}

// Load of the prescribed Dirichlet values on free row d:
// fD_d = -sum (V_e grad N_i . grad N_j) g_j over the contributions listed for
// the row (element e, local i = the row's node, local j a Dirichlet node), in
// increasing (element, j) order.
__global__ void k_dirichlet_load(int n_rows, const int *__restrict__ dptr,
                                 const int *__restrict__ dcon, const TetRec64 *__restrict__ rec,
                                 const double *__restrict__ det, const int4 *__restrict__ tet,
                                 const double *__restrict__ gD, double *fD)
{
    int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= n_rows)
        return;
    double sum = 0.0;
    for (int k = dptr[d]; k < dptr[d + 1]; ++k) {
        int c = dcon[k];
        int t = c >> 4, i = (c >> 2) & 3, j = c & 3;
        TetRec64 r = rec[t];
        double gi[3], gj[3];
        grad_row(r, i, gi);
        grad_row(r, j, gj);
        double vol = det[t] / 6.0;
        double dot = (gi[0] * gj[0] + gi[1] * gj[1]) + gi[2] * gj[2];
        int4 v4 = tet[t];
        int v[4] = {v4.x, v4.y, v4.z, v4.w};
        sum = sum - (vol * dot) * gD[v[j]];
    }
    fD[d] = sum;
}

// Emitting face: unit normal (B-A)x(C-A)/|.| into the vacuum, area |.|/2.
__global__ void k_face_geometry(int F, const int *__restrict__ fnodes, const double *__restrict__ xyz,
                                double *nhat, double *area)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F)
        return;
    const double *A = xyz + 3 * (size_t)fnodes[3 * f + 0];
    const double *B = xyz + 3 * (size_t)fnodes[3 * f + 1];
    const double *C = xyz + 3 * (size_t)fnodes[3 * f + 2];
    double u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    double w[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
    double n[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2],
                   u[0] * w[1] - u[1] * w[0]};
    double len = sqrt((n[0] * n[0] + n[1] * n[1]) + n[2] * n[2]);
    for (int i = 0; i < 3; ++i)
        nhat[3 * f + i] = n[i] / len;
    area[f] = 0.5 * len;
}

static inline unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

cudaError_t launch_geometry(cudaStream_t s, int T, const double *xyz, const int4 *tet,
                            const int4 *nb, TetRec64 *rec64, TetRec32 *rec32, double *det)
{
    if (T <= 0)
        return cudaSuccess;
    k_geometry<<<blocks_for(T, 128), 128, 0, s>>>(T, xyz, tet, nb, rec64, rec32, det);
    return cudaGetLastError();
}

cudaError_t launch_matrix_values(cudaStream_t s, long long nnz, const long long *cptr,
                                 const int *contrib, const TetRec64 *rec, const double *det,
                                 const long long *sell_pos, const int *slot_row,
                                 const int *slot_col, double *val64, float *val32,
                                 double *dinv64, float *dinv32)
{
    if (nnz <= 0)
        return cudaSuccess;
    k_matrix_values<<<blocks_for(nnz, 256), 256, 0, s>>>(nnz, cptr, contrib, rec, det, sell_pos,
                                                         slot_row, slot_col, val64, val32,
                                                         dinv64, dinv32);
    return cudaGetLastError();
}

cudaError_t launch_neumann(cudaStream_t s, int n_rows, const int *fptr, const int *fcontrib,
                           const int4 *tet, const double *xyz, const int *tet_rep,
                           const double *E0_rep, double *fN)
{
    if (n_rows <= 0)
        return cudaSuccess;
    k_neumann<<<blocks_for(n_rows, 256), 256, 0, s>>>(n_rows, fptr, fcontrib, tet, xyz, tet_rep,
                                                      E0_rep, fN);
    return cudaGetLastError();
}

cudaError_t launch_dirichlet_load(cudaStream_t s, int n_rows, const int *dptr, const int *dcon,
                                  const TetRec64 *rec, const double *det, const int4 *tet,
                                  const double *gD, double *fD)
{
    if (n_rows <= 0)
        return cudaSuccess;
    k_dirichlet_load<<<blocks_for(n_rows, 256), 256, 0, s>>>(n_rows, dptr, dcon, rec, det, tet, gD,
                                                             fD);
    return cudaGetLastError();
}

cudaError_t launch_face_geometry(cudaStream_t s, int F, const int *face_nodes,
                                 const double *xyz, double *nhat, double *area)
{
    if (F <= 0)
        return cudaSuccess;
    k_face_geometry<<<blocks_for(F, 128), 128, 0, s>>>(F, face_nodes, xyz, nhat, area);
    return cudaGetLastError();
}

}  // namespace pf
