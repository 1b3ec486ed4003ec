// common.cuh -- device data layout and kernel entry points shared by the
// translation units of libpicfem (the GB300 FEM-PIC cycle).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "picfem.h"

namespace pf {

// ---------------------------------------------------------------------------
// Per-tetrahedron walk record: the rows of J^-1 (J = [x1-x0|x2-x0|x3-x0]),
// the vertex x0, and the packed neighbour of each face.  One record is one
// 128-byte line in FP64 and half a line in FP32, so a walk step is a single
// line fetch.
//
// Packed neighbour nb[k] of face k (opposite vertex k):
//   nb >= 0          interior: (neighbour << 2) | local index of the shared
//                    face in the neighbour (the face the walk enters by)
//   nb == NB_TOP     Gamma_1, the SP is collected
//   nb == NB_CATHODE Gamma_3, the SP is absorbed
//   nb <= NB_SIDE    Gamma_2: v = NB_SIDE - nb = (partner << 4) |
//                    (shift << 2) | entry face; shift 0:+Lx 1:-Lx 2:+Ly 3:-Ly
// ---------------------------------------------------------------------------
constexpr int NB_TOP = -1;
constexpr int NB_CATHODE = -2;
constexpr int NB_SIDE = -16;

struct __align__(128) TetRec64 {
    double j[9];
    double x0[3];
    int nb[4];
};
struct __align__(64) TetRec32 {
    float j[9];
    float x0[3];
    int nb[4];
};
static_assert(sizeof(TetRec64) == 128, "one line per FP64 record");
static_assert(sizeof(TetRec32) == 64, "half a line per FP32 record");

// field of one tetrahedron, padded to one 32-byte load
struct __align__(32) Vec4d {
    double x, y, z, w;
};
__host__ __device__ inline Vec4d make_vec4d(double x, double y, double z, double w)
{
    return Vec4d{x, y, z, w};
}

template <typename R> struct Rec;
template <> struct Rec<double> { using type = TetRec64; using vec4 = Vec4d; };
template <> struct Rec<float> { using type = TetRec32; using vec4 = float4; };

// SP id layout: (step << 42) | (quadrangle << 18) | index in the quadrangle
constexpr int ID_QUAD_SHIFT = 18;
constexpr int ID_STEP_SHIFT = 42;
constexpr long long MAX_PER_QUAD = 1LL << ID_QUAD_SHIFT;
constexpr int MAX_ATTEMPTS = 64;

// Particle store: structure of arrays, one buffer of `capacity` SPs.
template <typename R> struct Particles {
    R *x, *y, *z, *vx, *vy, *vz;
    int *cell;
    long long *id;
};

// Mesh data the particle kernels read.
template <typename R> struct MeshView {
    const typename Rec<R>::type *rec;   // [T]
    const int4 *tet;                    // [T] node indices
    const typename Rec<R>::vec4 *E;     // [T] field of the current Phi
    const int *face_nodes;              // [F*3]
    const int *face_tet;                // [F]
    const double *face_nhat;            // [F*3]
    const double *face_area;            // [F]
    const double *wf;                   // [F]
    const double *xyz;                  // [N*3]
    int n_faces;
    // replicas (a batch; one replica for a single mesh)
    const int *tet_rep;                 // [T] replica of each tetrahedron
    const int *face_rep;                // [F] replica of each emitting face
    const int *rep_face_off;            // [R+1] first face of each replica
    const double *rep_L;                // [2R] periodic box length in x and y
};

// Run constants of the particle kernels.
struct RunConst {
    double dt, qmdt;       // dt and (q/m) dt = 2Q
    double w_sp, e_charge;
    double scale;          // 2^S
    uint64_t seed;
    long long capacity;
    int fn_model;
    int walk_max;
};

// Device-side bookkeeping of one context.
// slices per aggregate of the general solver's coarse correction
constexpr int PCG_AGG_SLICES = 32;
// multigrid hierarchy of the resident solver: pairwise-matching passes for
// level 1 and level 2, the most level-2 rows (dense inverse), and the
// Chebyshev smoothing degrees of the fine level and of level 1
constexpr int MG_PASSES0 = 3;
constexpr int MG_PASSES1 = 4;
constexpr int MG_MAX_COARSE = 2048;
constexpr int MG_DEGREE0 = 3;
constexpr int MG_DEGREE1 = 3;
// multigrid hierarchy of the general kernels: at most GMG_MAX_LEVELS levels
// below the fine one, coarsened until every system has at most
// GMG_MAX_COARSE rows on the coarsest (solved with a dense inverse); the
// smoothing degree is at most GMG_MAX_DEG
constexpr int GMG_MAX_LEVELS = 6;
constexpr int GMG_MAX_COARSE = 1024;
constexpr int GMG_MAX_DEG = 8;
constexpr int GMG_DEGREE0 = 1;
constexpr int GMG_DEGREE1 = 3;

// One level of the general kernels' V-cycle as the device reads it (an array
// in device memory, level 0 = the fine matrix).  Rows are laid out in 32-row
// slices like the fine level, each system's rows in its own slices
// [gsl[g], gsl[g+1]); padding rows have 1/diagonal 0 and no entries.
struct GmgLevel {
    int n_slices;
    const int *sptr, *col;          // sliced ELLPACK (element offsets, level rows)
    const float *val32, *dinv32;    // values, 1 / diagonal
    const double *val64, *dinv64;
    const int *gsl;                 // [systems + 1] slices of each system
    const int *agg;                 // next finer level's rows -> this level's (-1: none)
    const int *mptr, *midx;         // next finer level's rows in each row's aggregate
    void *x, *rc, *d[2];            // correction, residual, Chebyshev steps (the
                                    // solver's precision: float or double)
    double c1[GMG_MAX_DEG], c2[GMG_MAX_DEG], inv_theta;   // Chebyshev coefficients
    float c1f[GMG_MAX_DEG], c2f[GMG_MAX_DEG], inv_thetaf;
};

// Step bookkeeping kept on the device, so that a whole step can be captured
// in a CUDA graph and replayed: the index of the step being run (key of the
// random numbers and part of the SP ids) and the per-step statistics array of
// the current pic_step call.  The last kernel of a step copies the step's
// statistics into ring[step - step0] and advances step.
struct StepHdr {
    long long step;
    long long step0;
    pic_step_stats *ring;
    long long ring_cap;
};

struct DevState {
    unsigned long long cnt[2];  // SPs in particle buffer 0 / 1
    long long n_new;            // SPs injected in this step (after the scan)
    long long base;             // split API: first slot of the fresh SPs
    long long n_fresh;          // split API: fresh SPs at the end of the buffer
    int err;                    // first device-side error (PIC_ERR_*), 0 if none
    int pad;
    unsigned bar_count, bar_gen;  // grid barrier of the persistent PCG
    unsigned long long work;      // next unclaimed SP of the fused step (work queue)
    StepHdr hdr;
};

// ---------------------------------------------------------------------------
// kernel launchers (each returns the cudaError_t of the launch)
// ---------------------------------------------------------------------------
// setup (mesh_load)
cudaError_t launch_geometry(cudaStream_t s, int T, const double *xyz, const int4 *tet,
                            const int4 *nb, TetRec64 *rec64, TetRec32 *rec32, double *det);
cudaError_t launch_matrix_values(cudaStream_t s, long long nnz, const long long *cptr,
                                 const int *contrib, const TetRec64 *rec, const double *det,
                                 const long long *sell_pos, const int *slot_row,
                                 const int *slot_col, double *val64, float *val32,
                                 double *dinv64, float *dinv32);
cudaError_t launch_dirichlet_load(cudaStream_t s, int n_rows, const int *dptr, const int *dcon,
                                  const TetRec64 *rec, const double *det, const int4 *tet,
                                  const double *gD, double *fD);
cudaError_t launch_neumann(cudaStream_t s, int n_rows, const int *fptr, const int *fcontrib,
                           const int4 *tet, const double *xyz, const int *tet_rep,
                           const double *E0_rep, double *fN);
cudaError_t launch_face_geometry(cudaStream_t s, int F, const int *face_nodes,
                                 const double *xyz, double *nhat, double *area);

// particles
template <typename R>
cudaError_t launch_field(cudaStream_t s, int T, const typename Rec<R>::type *rec,
                         const int4 *tet, const double *phi, typename Rec<R>::vec4 *E,
                         DevState *end_step, pic_step_stats *slot);
template <typename R>
cudaError_t launch_inject_count(cudaStream_t s, int nq, MeshView<R> m, RunConst c,
                                const long long *step, int *qcount, int *err);
cudaError_t launch_inject_scan(cudaStream_t s, int nq, const int *qcount, long long *qoff,
                               DevState *st, int buf, long long capacity, int split_mode,
                               pic_step_stats *stats);
template <typename R>
cudaError_t launch_inject_emit(cudaStream_t s, int grid, MeshView<R> m, RunConst c,
                               const long long *step, int nq, const long long *qoff,
                               Particles<R> P, DevState *st);
template <typename R>
cudaError_t launch_push_relocate(cudaStream_t s, int grid, MeshView<R> m, RunConst c,
                                 Particles<R> A, Particles<R> B, int a, DevState *st,
                                 pic_step_stats *stats, int *dest = nullptr);
template <typename R>
cudaError_t launch_deposit(cudaStream_t s, int grid, MeshView<R> m, RunConst c,
                           Particles<R> A, int a, DevState *st, unsigned long long *W);
// walk_form: WALK_FORM_AUTO (persistent lanes for FP64, coherent warps for
// FP32), WALK_FORM_COHERENT, WALK_FORM_PERSISTENT or WALK_FORM_ROUNDS
enum { WALK_FORM_AUTO = 0, WALK_FORM_COHERENT = 1, WALK_FORM_PERSISTENT = 2, WALK_FORM_ROUNDS = 3 };
template <typename R>
cudaError_t launch_step_fused(cudaStream_t s, int grid, int walk_form, MeshView<R> m, RunConst c,
                              const long long *step, int nq, const long long *qoff, Particles<R> A,
                              Particles<R> B, int a, DevState *st, unsigned long long *W,
                              pic_step_stats *stats);
template <typename R>
cudaError_t launch_pack(cudaStream_t s, long long n, Particles<R> A, double *r, double *v,
                        int *cell, long long *id);
template <typename R>
cudaError_t launch_unpack(cudaStream_t s, long long n, const double *r, const double *v,
                          const int *cell, const long long *id, Particles<R> A);
template <typename R>
cudaError_t launch_field_unpack(cudaStream_t s, int T, const typename Rec<R>::vec4 *E,
                                double *out);

// Poisson solve
// polls a device-side wait of the solver (grid barrier, tagged halo word)
// makes before it gives up with PIC_ERR_TIMEOUT, unless pic_tuning.wait_limit
// sets another limit
constexpr long long PCG_SPIN_LIMIT_DEFAULT = 1LL << 25;

struct PcgArgs {
    int n, n_pad, n_slices;
    const int *slice_ptr;     // [n_slices+1], element offsets (multiples of 32)
    const int *col;           // sliced ELLPACK columns
    const double *val64;
    const float *val32;
    const double *dinv64;     // 1 / M_ii, 0 on padding rows
    const float *dinv32;
    const double *fN;         // Neumann load per free DOF
    const unsigned long long *W;  // fixed-point node charge
    const int *dof_node;      // node of each free DOF, -1 on padding rows
    double coef;              // q w_sp / eps0
    double wscale;            // 2^-S
    double *x;                // [n_pad] potential on free DOFs (warm start in, out)
    double *phi;              // [n_nodes] receives x on the free nodes
    double *f, *r, *z, *p0, *p1, *ap;          // FP64 work vectors [n_pad]
    float *r32, *z32, *p32_0, *p32_1, *ap32, *dx32;  // FP32 work vectors [n_pad]
    double *partials;         // [2][grid][4]
    double *part8;            // [2][grid][8] (resident one-reduction CG)
    DevState *st;
    pic_step_stats *stats;    // nullable
    const unsigned long long *alive;  // nullable: SPs in flight -> stats->alive
    double rtol, inner_rtol;
    int max_iter;
    int precision;
    long long spin_limit;     // polls of one device-side wait before PIC_ERR_TIMEOUT
    int max_rows;             // resident kernels: see PcgLaunch
    long long max_chunk;
    int variant;              // FP32_IR inner solver (PIC_PCG_*)
    int inner_max;            // FP32_IR inner iterations per refinement (0 = no cap)
    const int *lcol;          // resident kernels: block-local column of every stored entry
    const int *halo_ptr;      // [grid+1] first halo column of each block
    const int *halo_idx;      // global rows of the halo columns, sorted per block
    int max_local;            // most own rows + halo columns of one block
    int cheb_degree;          // <= 1: Jacobi; k >= 2: Chebyshev polynomial preconditioner
    double cheb_a, cheb_b;    // Chebyshev interval of D^-1 M
    // coefficients of the Chebyshev steps (computed on the host):
    // d_1 = D^-1 r / theta;  d_{j+1} = c1[j] d_j + c2[j] D^-1 r_j
    double cheb_c1[32], cheb_c2[32], cheb_inv_theta;
    float cheb_c1f[32], cheb_c2f[32], cheb_inv_thetaf;
    double *d0, *d1;          // FP64 halo buffers of the Chebyshev steps [n_pad]
    float *d32_0, *d32_1;     // FP32 halo buffers of the Chebyshev steps [n_pad]
    // resident FP32 kernels: the Chebyshev steps' neighbour exchange without a
    // grid barrier.  dtag[k][row] = value bits | tag << 32, written in one
    // 64-bit store; readers poll until the tag is the one they expect.  Tags
    // carry a per-launch epoch (*epoch, advanced once per launch, never
    // saved or restored with the state).  null: grid barriers instead.
    unsigned long long *dtag[2];
    unsigned *epoch;
    // independent systems solved side by side (a batch of replicas): group g
    // owns slices [grp[4g], grp[4g+1]) and blocks [grp[4g+2], +grp[4g+3]);
    // n_groups == 0 means one system over the whole grid
    int n_groups;
    const int *grp;           // [4 * n_groups]
    const int *blk_grp;       // [grid] group of each block
    unsigned *grp_bar;        // [n_groups] barrier counters, zero at launch
    int *grp_iters;           // [n_groups] iterations of each system's last solve (or null)
    int stream_matrix;        // general kernels: 1 stream the matrix past L2 (it does not fit)
    int cheb_local;           // resident kernels: 1 block-local Chebyshev preconditioner,
                              // 2 block-local + coarse correction over the blocks
    const float *coarse_inv;  // [G*G] inverse of the blocks' coarse matrix (or null)
    double *coarse_r;         // [2G] the blocks' sums of r (and of A p: merged form)
    // general kernels' coarse correction (null agg_inv: none)
    const int *agg_off;       // [groups + 1] first aggregate of each group
    const long long *inv_off; // [groups] offset of each group's A0^-1 in agg_inv
    const float *agg_inv;     // the groups' A0^-1, row-major
    double *slice_r, *agg_r, *agg_z;   // [n_slices], [n_agg], [n_agg]
    const double *rhs;        // null: f from W and the Neumann load; else f[row] = rhs[row]
    const double *fD;         // load of the prescribed Dirichlet values (rows)
    // Multigrid V-cycle of the resident kernels (cheb_local == 4, mg_n1 > 0):
    // level 1 aggregates the fine rows, level 2 the level-1 rows, every
    // aggregate inside one block; Chebyshev smoothing of degree mg_deg0 on the
    // fine level (the fine coefficients above) and mg_deg1 on level 1; level 2
    // solved with a dense inverse.  Block b owns level-1 rows
    // [mg_l1_off[b], mg_l1_off[b+1]) and level-2 rows [mg_l2_off[b], ..+1]).
    int mg_n1, mg_n2, mg_deg0, mg_deg1;
    int mg_max_l1_local, mg_max_l1_own, mg_max_l2_own;
    size_t mg_smem_off;       // byte offset of the V-cycle's arrays in dynamic shared memory
    const int *mg_agg0;       // [n_pad] fine row -> block-local level-1 row, -1 on padding
    const int *mg_l1_off, *mg_l2_off;  // [G+1]
    const int *mg_m0_ptr, *mg_m0_idx;  // [n1+1]: fine rows (block-local) of each level-1 row
    const int *mg_a1_ptr, *mg_a1_col;  // level-1 matrix: CSR rows, block-local columns
    const float *mg_a1_val32;
    const double *mg_a1_val64;
    const float *mg_dinv1_32;
    const double *mg_dinv1_64;
    const int *mg_h1_ptr, *mg_h1_idx;  // [G+1] / global level-1 rows of each block's halo
    const int *mg_agg1;       // [n1] level-1 row -> block-local level-2 row
    const int *mg_m1_ptr, *mg_m1_idx;  // [n2+1]: level-1 rows (block-local) of each level-2 row
    const float *mg_a2inv;    // [n2*n2] inverse of the level-2 matrix, row-major
    float *mg_r2f;            // [n2] level-2 right-hand side (FP32 kernels)
    double *mg_r2d;           // [n2] (FP64 kernels)
    unsigned long long *mg_dtag1;  // [2*n1] tagged level-1 exchange words
    float *mg_g1f[2];         // [n1] level-1 exchange through a grid barrier (FP32)
    double *mg_g1d[2];        // (FP64)
    double mg_c1[32], mg_c2[32], mg_inv_theta;   // level-1 Chebyshev coefficients
    float mg_c1f[32], mg_c2f[32], mg_inv_thetaf;
    // Multigrid V-cycle of the general kernels (gmg_nlev > 0): levels
    // gmg[0] (fine) .. gmg[gmg_nlev] (coarsest, solved per system with the
    // dense inverse gmg_inv + gmg_ioff[g] of order gmg_cn[g]); Chebyshev
    // smoothing of degree gmg_deg0 on the fine level, gmg_deg1 below
    int gmg_nlev, gmg_deg0, gmg_deg1;
    const GmgLevel *gmg;
    const float *gmg_inv;
    const long long *gmg_ioff;
    const int *gmg_cn;
};
// Host-side product of mg_build: the multigrid hierarchy of the resident
// solver (see mg.cu), with the layout of the PcgArgs fields above.
struct MgHost {
    int n1 = 0, n2 = 0;
    std::vector<int> agg0, l1_off, l2_off, m0_ptr, m0_idx, a1_ptr, a1_col, h1_ptr, h1_idx;
    std::vector<int> agg1, m1_ptr, m1_idx;
    std::vector<double> a1_val, dinv1;
    std::vector<float> a2inv;
    double lmax1 = 2.0;
    int max_l1_local = 0, max_l1_own = 0, max_l2_own = 0;
};
// Build the hierarchy from the fine matrix in sliced ELLPACK (host copies of
// slice_ptr, columns, FP64 values and 1/diagonal, 0 on padding rows) split
// over G blocks as the resident kernels split it: passes0 matching passes
// for level 1, passes1 (more while it has over max_coarse rows) for level 2.
// false when the hierarchy cannot be built (the caller keeps the other
// preconditioners).
bool mg_build(const int *sptr, const int *scol, const double *sval, const double *dinv,
              int n_slices, int G, int passes0, int passes1, int max_coarse, MgHost *out);
// dynamic shared memory of the V-cycle's arrays (bytes, elements of `elem` bytes)
// Host-side product of gmg_build: the general kernels' hierarchy.  lev[0]
// stands for the fine level (empty); lev[1..L] hold the coarse levels in the
// device layout of GmgLevel (the coarsest without a matrix); the coarsest
// level's matrix of each system is inverted (FP64 Cholesky, stored in FP32).
struct GmgLevelHost {
    int n_slices = 0;
    std::vector<int> sptr, col, gsl, agg, mptr, midx;
    std::vector<double> val, dinv;
    double lmax = 2.0;
};
struct GmgHost {
    std::vector<GmgLevelHost> lev;
    std::vector<int> cn;
    std::vector<long long> ioff;
    std::vector<float> inv;
};
// Build it from the fine matrix (sliced ELLPACK as for mg_build) of n_sys
// independent systems, system g on slices [sys_slices[g], sys_slices[g+1]):
// passes0 matching passes for level 1, passes1 for each further level, until
// every system has at most max_coarse rows (at most max_levels levels).
// false when that cannot be reached.
bool gmg_build(const int *sptr, const int *scol, const double *sval, const double *dinv,
               int n_slices, int n_sys, const int *sys_slices, int passes0, int passes1,
               int max_coarse, int max_levels, GmgHost *out);
inline size_t mg_smem_bytes(const MgHost &m, size_t elem)
{
    return elem * ((size_t)m.max_l1_local + 4 * (size_t)m.max_l1_own + (size_t)m.max_l2_own) + 16;
}
struct PcgLaunch {
    int grid, block;
    int resident;          // 1: rows owned in registers, own segments in shared memory
    int rpt;               // resident: row slots per thread (1, 2, 4 or 8)
    int smem_matrix;       // resident: the block's matrix slices live in shared memory
    size_t smem_bytes;     // resident: dynamic shared memory per block
    int max_rows;          // resident: 32 * most slices owned by one block
    long long max_chunk;   // resident: most stored matrix entries owned by one block
    int max_local;         // resident: most own rows + halo columns of one block
    int halo_symmetric;    // resident: block b reads block o's rows iff o reads b's
    int n_groups;          // general: independent systems (0: one system, whole grid)
    size_t mg_off;         // resident with a multigrid hierarchy: where its shared arrays start
};
// Host-side tables: local column indices and halos of the resident kernels;
// group tables of the general kernels when several systems are solved side
// by side.
struct PcgHalo {
    std::vector<int> lcol, halo_ptr, halo_idx;
    std::vector<int> grp, blk_grp;
};
// message returned by pic_last_error(NULL)
void set_global_error(const char *msg);

// grp_slices[g] .. grp_slices[g+1]: slices of system g (n_sys >= 1)
// blocks_per_sm > 0 caps the blocks of a batch solve at blocks_per_sm per SM;
// a batch's blocks are shared out in proportion to grp_work (null: to the
// systems' slices)
cudaError_t pcg_plan(const int *slice_ptr_host, const int *col_host, int n_slices,
                     int num_sms, int precision, int variant, int n_sys, const int *grp_slices,
                     const double *grp_work, int blocks_per_sm, PcgLaunch *plan, PcgHalo *halo);
// the most blocks a batch solve can use (its partial-sum buffer is sized for it)
int pcg_max_group_blocks(int precision, int num_sms);
// grid of the one-system general kernels: a slice per warp at most, at most
// blocks_per_sm blocks per SM (0: as many as fit); 0 on error
int pcg_general_grid(int precision, int n_slices, int num_sms, int blocks_per_sm);
cudaError_t launch_pcg(cudaStream_t s, const PcgLaunch &plan, const PcgArgs &a);
// Grow a resident plan's dynamic shared memory by the multigrid arrays
// (`extra` bytes); *ok = false (plan unchanged) when the block would no
// longer fit on an SM.
cudaError_t pcg_plan_mg(PcgLaunch *plan, int precision, int variant, size_t extra, bool *ok);

// ---------------------------------------------------------------------------
// adjoint (pic_adjoint)
// ---------------------------------------------------------------------------
// where the push put SP i: its slot in the other buffer, or one of these
enum { DEST_COLLECTED = -1, DEST_ABSORBED = -2 };

// adjoint of the SP state (position, velocity, weight), FP64, structure of arrays
struct AdjSP {
    double *rx, *ry, *rz, *vx, *vy, *vz, *w;
};

// One step of the reverse pass over the SPs of a recorded step: `pre` holds
// the step's SPs before the push (the n_old old ones, then the injected
// ones), `dest` where the push sent each, `post` the buffer it wrote.
template <typename R> struct AdjStep {
    long long n, n_old;
    Particles<R> pre, post;
    const int *dest;
    AdjSP in;                  // adjoint of the post-push state, by slot
    AdjSP out;                 // adjoint of the pre-step state of the old SPs
    const TetRec64 *rec64;
    const int4 *tet;
    const Vec4d *E;            // E_k in FP64
    const double *fbar;        // node adjoint of the RHS of the solve after the step
    double coef;               // q w_sp / eps0
    double *Ebar;              // [3T] adjoint of E_k (accumulated)
    double *gwf;               // [F] dQ/dphi_f (accumulated)
    const int *face_tet, *face_rep, *rep_face_off;
    const double *fnhat, *wf;
    uint64_t seed;
    int fn_model;
    double qmdt, dt, qw;       // q/m dt, dt, q w_sp
};
template <typename R> cudaError_t launch_adjoint_sp(cudaStream_t s, const AdjStep<R> &g);
// Phi_bar += E^T Ebar (E = -grad Phi per tetrahedron)
cudaError_t launch_field_adjoint(cudaStream_t s, int T, const TetRec64 *rec, const int4 *tet,
                                 const double *Ebar, double *phibar);
// Stable compaction after an ordered push (dest[i] = 1 for a survivor held at
// B[i], else DEST_*): survivors move to A[0..n_alive) in index order, dest[i]
// becomes the survivor's slot, st->cnt[a] = n_alive, st->n_fresh = 0.
// scratch: 2 * ceil(n / 1024) + 2 ints.
template <typename R>
cudaError_t launch_compact(cudaStream_t s, long long n, int *dest, Particles<R> B, Particles<R> A,
                           DevState *st, int a, int *scratch);
// out[i] = sum_{j<i} in[j] for i <= n (scratch: 2 ceil(n / 1024) + 2 ints)
cudaError_t launch_exclusive_scan(cudaStream_t s, long long n, const int *in, int *out,
                                  int *scratch);

// Monte Carlo binary collisions of the SPs of each cell (App. F)
template <typename R> struct CollArgs {
    Particles<R> P;                  // the SPs in flight
    const unsigned long long *n;     // their count (device)
    const long long *step;           // the step index (device)
    int T;
    const double *det;               // [T] det J (volume = det / 6)
    const int *tet_rep, *rep_tet_off;   // replica of a tetrahedron, first tetrahedron of a replica
    int *cnt, *off, *fill;           // [T], [T + 1], [T] scratch
    int *perm;                       // [capacity] SPs grouped by cell
    unsigned long long *key;         // [capacity] random order key of each SP
    int *scan;                       // scan scratch
    uint64_t seed;
    double w_sp, coulomb_log, dt, q, m, eps0;
    int grid;                        // blocks of the SP passes
};
template <typename R> cudaError_t launch_collide(cudaStream_t s, const CollArgs<R> &g);
// B (count *nB) -> A ordered by cell, *nA = *nB; scratch cnt [T], off [T + 1],
// rank [capacity], scan (scan scratch for T)
template <typename R>
cudaError_t launch_sort_by_cell(cudaStream_t s, int grid, int T, Particles<R> B, Particles<R> A,
                                const unsigned long long *nB, unsigned long long *nA, int *cnt,
                                int *off, int *rank, int *scan);
// rows of a node vector (0 on padding rows)
cudaError_t launch_gather_rows(cudaStream_t s, int n_rows, const int *dof_node,
                               const double *node_v, double *rows);
// gE0[r] += sum over the rows of replica r of x_row fN_row / E0_r
cudaError_t launch_dE0(cudaStream_t s, int n_rows, const double *x, const double *fN,
                       const int *rep_slice, int n_rep, const double *E0_rep, double *gE0);

}  // namespace pf
