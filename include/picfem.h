/*
 * picfem.h -- C ABI of libpicfem, the GB300 (sm_103a) electrostatic FEM-PIC
 * cycle of Veske et al., "Dynamic coupling between particle-in-cell and
 * atomistic simulations", Phys. Rev. E 101, 053307 (arXiv 1906.08125).
 *
 * One PIC step (Sec. II.B, eqs. leapfrog1-3 and Fig. 3):
 *   inject        field-emission injection from the cathode quadrangles
 *                 (Sec. II.B.3, eqs. nsp, rnd_nsp, sp_velocity,
 *                 sp_displacement; App. E eq. rnd_point)
 *   push_relocate leapfrog kick with E_k = -grad Phi_k (P1, constant per
 *                 tetrahedron), drift, and relocation by walking tetrahedron
 *                 neighbours; absorption at Gamma_1 / Gamma_3, periodic wrap
 *                 on Gamma_2 (Sec. II.B.1-2)
 *   deposit       charge to mesh nodes with the same P1 shape functions,
 *                 as int64 fixed point (Sec. II.B.2, eq. poisson_rhs)
 *   poisson_solve preconditioned CG on the P1 stiffness matrix (eqs. poisson,
 *                 poisson_bc; App. B eq. poisson_mat) -> Phi_{k+1}
 * pic_step runs the four in that order, n times, with fused kernels.
 *
 * Conventions for every entry point:
 *  - Return value: PIC_OK (0) or a negative PIC_ERR_* code; the message is
 *    available from pic_last_error().  No exception crosses the ABI.
 *  - Host input arrays are copied; the caller keeps ownership.
 *  - "device" pointers are CUDA device (or managed) memory on the context's
 *    device, e.g. torch.Tensor.data_ptr(); the copy is queued on the
 *    context's stream and is complete when the call returns unless stated
 *    otherwise.  "host or device" pointers may be either (CUDA unified
 *    addressing decides the direction).
 *  - Calls that return host scalars synchronise the context's stream.
 *  - The context owns all internal device buffers (freed by pic_destroy).
 *  - Units are SI: m, s, V, V/m, C, kg.
 *  - A context is not thread safe; use one context per host thread.
 */
#ifndef PICFEM_H
#define PICFEM_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define PIC_OK 0
#define PIC_ERR_ARG (-1)             /* bad argument or non-finite input     */
#define PIC_ERR_CUDA (-2)            /* a CUDA runtime call failed            */
#define PIC_ERR_MESH (-3)            /* inconsistent or inverted mesh         */
#define PIC_ERR_CAPACITY (-4)        /* more SPs than particle_capacity       */
#define PIC_ERR_WALK_LIMIT (-5)      /* an SP walked more than walk_max_steps */
#define PIC_ERR_NOT_CONVERGED (-6)   /* PCG reached pcg_max_iter              */
#define PIC_ERR_NOT_IMPLEMENTED (-7)
#define PIC_ERR_TIMEOUT (-8)         /* a device-side wait ran out            */

/* neighbour-table boundary codes (nbr[t*4+k] < 0; face k is opposite vertex k) */
#define PIC_BND_TOP (-1)      /* Gamma_1: far-field Neumann face, SPs collected */
#define PIC_BND_CATHODE (-2)  /* Gamma_3: Dirichlet Phi = 0, SPs absorbed       */
#define PIC_BND_SIDE (-3)     /* Gamma_2: laterally periodic for SPs            */

/* arithmetic of the push and of the Poisson solve */
#define PIC_PREC_FP64 0     /* FP64 throughout (bit-exact with the FP64 oracle)   */
#define PIC_PREC_FP32_IR 1  /* FP32 push/SpMV; PCG wrapped in FP64 iterative
                               refinement (FP64 residual, dot products, update) */

/* Fowler-Nordheim model for the emission current density J_e */
#define PIC_FN_MURPHY_GOOD 0  /* Murphy-Good with Forbes' 2006 v(f), t(f)   */
#define PIC_FN_ELEMENTARY 1   /* v = t = 1                                    */

typedef struct pic_ctx_s *pic_ctx;

typedef struct {
    double dt;             /* PIC time step Delta t [s] (eqs. leapfrog1-3)      */
    double E0;             /* applied field on Gamma_1 [V/m] (eq. poisson_bc)   */
    double w_sp;           /* SP weight (real particles per SP)                 */
    double q;              /* charge of one real particle [C], -e for electrons */
    double q_over_m;       /* charge-to-mass ratio [C/kg] (eq. newton)          */
    double eps0;           /* permittivity [F/m] (eq. poisson)                  */
    double e_charge;       /* elementary charge [C] (eq. nsp)                   */
    double pcg_rtol;       /* stop when ||f - M Phi||_2 <= rtol ||f||_2         */
    int32_t pcg_max_iter;  /* PCG iteration cap -> PIC_ERR_NOT_CONVERGED        */
    int32_t fn_model;      /* PIC_FN_*                                          */
    uint64_t seed;         /* key of the counter-based random numbers           */
    int64_t capacity;      /* maximum SPs in flight -> PIC_ERR_CAPACITY         */
    int32_t walk_max_steps;/* face crossings per SP per step -> PIC_ERR_WALK_LIMIT */
    int32_t quant_bits;    /* S: deposit weights in units of 2^-S, 1 <= S <= 40 */
    int32_t precision;     /* PIC_PREC_*                                        */
    int32_t pcg_variant;   /* FP32_IR inner solver: PIC_PCG_STANDARD,
                              PIC_PCG_PIPELINED, PIC_PCG_MERGED or
                              PIC_PCG_SINGLE                                    */
    double ir_inner_rtol;  /* FP32_IR: the most the inner FP32 PCG is asked to
                              reduce its residual in one refinement (e.g. 1e-4);
                              it stops earlier once the FP64 target is met     */
    int32_t ir_inner_max_iter; /* FP32_IR: inner iterations per refinement
                              before the FP64 residual is recomputed (0 = no cap) */
    int32_t pcg_cheb_degree;   /* preconditioner: <= 1 Jacobi; k >= 2 Chebyshev
                              polynomial of degree k in D^-1 M (k - 1 extra SpMVs
                              per CG iteration, no extra reductions)             */
    double pcg_cheb_ratio;     /* Chebyshev interval [b / ratio, b], b the
                              Gershgorin bound of D^-1 M (e.g. 30)               */
    int32_t graph;             /* 1: pic_step captures one step per buffer parity
                              in a CUDA graph and replays it (not while
                              profiling); 0: launches every kernel directly      */
    int32_t collisions;        /* 1: Monte Carlo binary collisions of the SPs of
                              each cell after every push (App. F; see pic_collide) */
    double coulomb_log;        /* Lambda of the scattering variance (App. F: 13)   */
} pic_params;

/* inner solver of the FP32_IR Poisson solve */
#define PIC_PCG_STANDARD 0   /* two grid reductions per iteration            */
#define PIC_PCG_PIPELINED 1  /* one (Ghysels & Vanroose 2014), less accurate  */
#define PIC_PCG_MERGED 2     /* the standard iteration with p.Ap summed on the
                                Chebyshev polynomial's first grid barrier (its
                                first step split by linearity into D^-1 r and
                                D^-1 A p): degree k >= 2 over the whole matrix,
                                k grid barriers per iteration instead of k + 1.
                                Single systems on the resident solver only;
                                otherwise the standard form runs            */
#define PIC_PCG_SINGLE 3     /* Chronopoulos & Gear: one reduction (r.u, Au.u,
                                r.r) per iteration, A p carried as s = w + beta s;
                                with the tagged exchange and a whole-matrix
                                Chebyshev polynomial (degree >= 2) one grid
                                barrier per iteration.  Single systems on the
                                resident solver only; otherwise standard     */

typedef struct {
    int64_t injected;         /* SPs injected in the step                      */
    int64_t collected;        /* SPs that left through Gamma_1                 */
    int64_t absorbed;         /* SPs that left through Gamma_3                 */
    int64_t wrapped;          /* periodic crossings of Gamma_2                 */
    int64_t crossings;        /* face crossings of all SPs in the walk         */
    int64_t alive;            /* SPs in flight after the step                  */
    int32_t max_walk;         /* longest walk (face crossings) of one SP       */
    int32_t pcg_iters;        /* CG iterations (FP32_IR: inner iterations)     */
    double pcg_relres;        /* final ||f - M Phi|| / ||f||                    */
    double collected_charge;  /* q * w_sp * collected [C]                      */
    int32_t pcg_outer;        /* FP32_IR refinements (FP64: 0)                 */
    int32_t reserved;
    int64_t walk_warp_iters;  /* walk iterations summed over warps: a warp of
                                 the coherent form spends its longest walk on
                                 each group of 32 SPs, one of the persistent
                                 form its loop iterations; 32 x this / crossings
                                 is the lane slots per useful walk step      */
} pic_step_stats;

typedef struct {
    int32_t n_nodes, n_tets, n_faces, n_free;
    int64_t nnz;              /* nonzeros of the stiffness matrix on free DOFs  */
    int64_t sell_len;         /* stored entries incl. slice padding            */
    int32_t pcg_grid;         /* blocks of the persistent PCG launch           */
    int32_t particle_grid;    /* blocks of the particle kernels                */
    double box_lo[3], box_hi[3];  /* over all replicas                          */
    int32_t n_rep;            /* replicas (1 after mesh_load)                  */
    int32_t n_rows;           /* solver rows: free DOFs + per-replica padding  */
    int32_t pcg_resident;     /* 1: one-system resident PCG kernel             */
    int32_t graph;            /* pic_step: 1 replays a captured CUDA graph per
                                 step, 0 not yet captured or params.graph = 0,
                                 -1 the capture was refused (direct launches)  */
    int32_t mg_levels;        /* multigrid hierarchy built at mesh_load for the
                                 solver in use (pcg_cheb_local = 4): levels
                                 below the fine one, 0 when there is none     */
    int32_t mg_coarse_rows;   /* rows of its coarsest level (the largest over
                                 the replicas of a batch)                     */
} pic_info;

/* Create a context on the current CUDA device.  `stream` is a cudaStream_t
 * (NULL = legacy default stream) on which every kernel and copy is queued. */
int pic_create(pic_ctx *out, const pic_params *p, void *stream);
int pic_destroy(pic_ctx ctx);
/* Message of the last failed call on ctx (static storage when ctx is NULL). */
const char *pic_last_error(pic_ctx ctx);
/* Library version string. */
const char *pic_version(void);

/*
 * mesh_load: the vacuum domain Omega_1 as P1 tetrahedra (Sec. II.A, App. B).
 * All pointers are HOST arrays and are copied.
 *   xyz[n_nodes*3]         node coordinates [m]
 *   tet[n_tets*4]          node indices, positively oriented
 *                          (det[x1-x0, x2-x0, x3-x0] > 0, else PIC_ERR_MESH)
 *   nbr[n_tets*4]          tetrahedron across the face opposite vertex k, or a
 *                          PIC_BND_* code; interior entries must be mutual
 *   periodic_nbr[n_tets*4] partner across a PIC_BND_SIDE face (nullable when
 *                          there are none); the side faces must lie on the
 *                          bounding-box planes x = min/max or y = min/max
 *   node_dirichlet[n_nodes] 1 for nodes on Gamma_3 (Phi = 0)
 *   face_nodes[n_faces*3]  emitting cathode triangles (A, B, C) with
 *                          (B-A)x(C-A) pointing into the vacuum; each gives
 *                          three quadrangles, one per vertex (Sec. II.B.3)
 *   face_tet[n_faces]      tetrahedron on the vacuum side of each face
 *   work_function_eV[n_faces] > 0
 * Builds the per-tetrahedron walk records, the stiffness matrix (sliced
 * ELLPACK), the Neumann load E0 A/3 per top-face vertex, and resets the
 * state (no SPs, Phi = 0, step 0).
 */
int mesh_load(pic_ctx ctx, int32_t n_nodes, const double *xyz, int32_t n_tets,
              const int32_t *tet, const int32_t *nbr, const int32_t *periodic_nbr,
              const uint8_t *node_dirichlet, int32_t n_faces, const int32_t *face_nodes,
              const int32_t *face_tet, const double *work_function_eV);

/*
 * mesh_load_batch: n_rep independent simulations (replicas) in one context,
 * stepped together by every call below.  The arrays are those of mesh_load
 * for the union of the replicas' meshes, each replica a contiguous block:
 *   rep_node_off[n_rep+1]  replica r owns nodes [rep_node_off[r], rep_node_off[r+1])
 *   rep_tet_off[n_rep+1]   and tetrahedra [rep_tet_off[r], rep_tet_off[r+1]);
 *                          both start at 0 and end at n_nodes / n_tets
 *   E0_rep[n_rep]          applied field of each replica [V/m] (params.E0 is
 *                          not used by a batch)
 * No tetrahedron, neighbour, periodic partner or face may reach into another
 * replica, and the emitting faces must be listed replica by replica
 * (PIC_ERR_MESH otherwise).  Each replica's periodic box is its own bounding
 * box in x and y.  Replica r draws its random numbers from seed + r with its
 * own quadrangle numbering, so it reproduces a one-replica run of its mesh
 * with seed + r; SP ids carry the batch-wide quadrangle index.  The Poisson
 * systems are solved together, each block of the solver working on one
 * replica, and each replica's CG stops at its own relative residual.
 * Statistics of pic_step / push_relocate are sums over replicas; the PCG
 * iteration count is the maximum.  All pointers are HOST arrays, copied.
 */
int mesh_load_batch(pic_ctx ctx, int32_t n_rep, const int32_t *rep_node_off,
                    const int32_t *rep_tet_off, const double *E0_rep, int32_t n_nodes,
                    const double *xyz, int32_t n_tets, const int32_t *tet, const int32_t *nbr,
                    const int32_t *periodic_nbr, const uint8_t *node_dirichlet, int32_t n_faces,
                    const int32_t *face_nodes, const int32_t *face_tet,
                    const double *work_function_eV);

/*
 * Launch tuning (an autotuner's knobs; none changes what is computed except
 * pcg_cheb_degree, which changes the preconditioner but not the stopping
 * rule, so the potential meets the same tolerance):
 *   particle_blocks_per_sm  blocks of 256 threads per SM of the particle
 *                           kernels (1..64; default 24 for FP32_IR, 8 for FP64)
 *   walk_form               fused step: 0 by precision (FP64 persistent lanes,
 *                           FP32 coherent warps), 1 coherent warps (a warp
 *                           walks 32 consecutive SPs to the end), 2 persistent
 *                           lanes (a lane takes the next SP from its warp's
 *                           queue), 3 rounds (a warp walks a contiguous range
 *                           of the SPs, shared out evenly over the warps, in
 *                           rounds of at most 16 face crossings, lanes that
 *                           finished taking the range's next SPs after each
 *                           round); the SP results are identical
 *   pcg_blocks_per_sm       batch solve (mesh_load_batch): at most this many
 *                           blocks per SM (0 = as many as fit; 0..64), and
 *                           the same for one system too large for the
 *                           resident kernels; the resident solver ignores it
 *   pcg_cheb_degree         as pic_params.pcg_cheb_degree (0..32)
 *   pcg_balance             batch solve: 1 (default) shares the blocks out in
 *                           proportion to each replica's slices x the CG
 *                           iterations of its last solve, re-planned at the
 *                           start of every pic_step call; 0 by slices only
 *   pcg_cheb_local          one-system (resident) solver: 0 applies the
 *                           Chebyshev polynomial (or Jacobi) to the whole
 *                           matrix; 1 to each solver block's own diagonal block
 *                           of D^-1 M (no grid barrier inside the
 *                           preconditioner); 2 adds to 1 the coarse correction
 *                           R0^T A0^-1 R0 r over the blocks (R0 sums a block's
 *                           rows, A0 = R0 M R0^T; one grid barrier); 3 is the
 *                           whole-matrix polynomial plus that coarse
 *                           correction; 4 a three-level multigrid V-cycle:
 *                           aggregates of the matrix rows by three passes of
 *                           pairwise matching within each solver block (level
 *                           1), four more on level 1 (level 2, solved with a
 *                           dense inverse), Galerkin coarse matrices,
 *                           Chebyshev smoothing of degree 3 before and after
 *                           the coarse correction on the fine level and on
 *                           level 1 (built at mesh_load for the resident
 *                           solver).  The general solver (batches, systems
 *                           too large for the resident blocks) builds its
 *                           own hierarchy for 4: the same matching over the
 *                           whole matrix of each replica, three passes for
 *                           level 1 and four for each further level until
 *                           every replica has at most 1024 rows (at most six
 *                           levels), the coarsest solved with a dense
 *                           inverse per replica, smoothing of degree
 *                           pcg_mg_degree0 on the fine level and
 *                           pcg_mg_degree1 on every coarser one, in FP32 or
 *                           FP64 with the solver.  PIC_ERR_ARG where no
 *                           hierarchy was built.  The
 *                           default is 4 where the hierarchy exists and
 *                           pcg_cheb_degree >= 2, else 3 when pcg_cheb_degree
 *                           >= 2, otherwise 0.  All are SPD; the stopping rule
 *                           is unchanged
 *   sort_cells              pic_step: 1 (default) orders the surviving SPs by
 *                           cell after every step (a counting sort; the
 *                           neighbouring SPs' walks then share walk records in
 *                           L1); 0 leaves them in the order the step appended
 *                           them.  Nothing computed depends on the order
 *   pcg_halo_sync           one-system FP32 solver, whole-matrix Chebyshev
 *                           steps: 1 (default) exchanges the step directions
 *                           with the neighbouring blocks through tagged
 *                           64-bit words (value | step tag), each block
 *                           waiting only for the values it reads; 0 with a
 *                           grid barrier per step.  Identical results
 *   wait_limit              polls one device-side wait of the solver (a grid
 *                           barrier, a tagged halo word) makes before the
 *                           kernel gives up, records PIC_ERR_TIMEOUT and
 *                           returns; 0 (default) = 2^25 polls, else 1..2^30.
 *                           For tests and diagnosis of the failure path: a
 *                           small limit makes a solve fail with
 *                           PIC_ERR_TIMEOUT, and the context stays usable
 *   pcg_mg_degree0/1        multigrid V-cycle (pcg_cheb_local = 4): degree of
 *                           the Chebyshev smoothing on the fine level / on
 *                           the coarser levels, before and after the coarse
 *                           correction
 *                           (1..8; 0 = the default: 3 and 3 for the
 *                           resident solver, 1 and 3 for the general one,
 *                           whose fine-level products stream the matrix
 *                           from HBM).  Changes the preconditioner, not the
 *                           stopping rule
 * pic_set_tuning takes effect from the next call and drops captured graphs;
 * PIC_ERR_ARG for a value out of range.  t: HOST.
 */
typedef struct {
    int32_t particle_blocks_per_sm;
    int32_t walk_form;
    int32_t pcg_blocks_per_sm;
    int32_t pcg_cheb_degree;
    int32_t pcg_balance;
    int32_t pcg_cheb_local;
    int32_t sort_cells;
    int32_t pcg_halo_sync;
    int32_t wait_limit;
    int32_t pcg_mg_degree0;
    int32_t pcg_mg_degree1;
} pic_tuning;
int pic_get_tuning(pic_ctx ctx, pic_tuning *t);
int pic_set_tuning(pic_ctx ctx, const pic_tuning *t);

/* Per replica (HOST arrays [n_rep], each nullable): CG iterations of its
 * last solve in a batch (inner iterations in the FP32_IR form; 0 when the
 * context holds one mesh), stored matrix entries (sliced ELLPACK, padding
 * included), solver rows (a multiple of 32) and free DOFs. */
int pic_replica_info(pic_ctx ctx, int32_t *pcg_iters, int64_t *stored, int32_t *rows,
                     int32_t *free_dofs);

/* Sizes of the loaded mesh and of the launches (info: HOST). */
int pic_mesh_info(pic_ctx ctx, pic_info *info);

/* Charge-free potential: Phi_0 from M Phi = f_Neumann (W = 0). */
int pic_init_potential(pic_ctx ctx, int32_t *iters, double *rel_res);

/*
 * inject: for every quadrangle q of every emitting face, F = max(0, -E.n),
 * J_e = J_FN(F, phi_face) (closed form; the paper uses GETELEC),
 * n_sp = J_e A_q dt / (e w_sp), stochastically rounded with R0 (eq. rnd_nsp);
 * each new SP gets a uniform point of the quadrangle by rejection from the
 * parallelogram (App. E), v0 = (q/m) E dt (1/2 + R3) and r = point + v0 dt R3
 * (eqs. sp_velocity, sp_displacement).  New SPs are appended and marked
 * fresh: the next push_relocate drifts them without the kick.
 * SP ids: (step << 42) | (quad << 18) | j.
 * n_injected: HOST, nullable (non-NULL synchronises).
 */
int inject(pic_ctx ctx, int64_t step, int64_t *n_injected);

/*
 * push_relocate: v += (q/m) dt E_cell for non-fresh SPs (the closing half kick
 * of the previous step merged with the opening half kick, eqs. leapfrog3 +
 * leapfrog1), then r += dt v for all, then the neighbour walk to the
 * containing tetrahedron; SPs leaving through Gamma_1 / Gamma_3 are removed,
 * through Gamma_2 wrapped.  out: HOST, nullable (non-NULL synchronises).
 */
int push_relocate(pic_ctx ctx, int64_t step, pic_step_stats *out);

/*
 * deposit: W_i = sum over SPs of the fixed-point weight of node i (eq.
 * poisson_rhs; w = rint(lambda 2^S) for three vertices, the fourth takes the
 * remainder, so every SP adds exactly 2^S).  node_charge_fx: DEVICE int64
 * [n_nodes], nullable; receives W.
 */
int deposit(pic_ctx ctx, int64_t *node_charge_fx);

/*
 * poisson_solve: f = (q w_sp / eps0) W 2^-S + f_Neumann on the free nodes;
 * preconditioned CG warm-started from the current Phi (precision, inner form
 * and preconditioner per pic_params and pic_tuning: Jacobi, or a Chebyshev
 * polynomial in D^-1 M with the two-level coarse correction; FP32_IR runs
 * FP32 inner solves inside FP64 iterative refinement); updates Phi and E.  phi: DEVICE double [n_nodes], nullable; iters and
 * rel_res: HOST, nullable (non-NULL synchronises).
 */
int poisson_solve(pic_ctx ctx, double *phi, int32_t *iters, double *rel_res);

/*
 * pic_step: n_steps full PIC steps from the current state (inject, push,
 * walk, deposit, solve), step index advancing by one each.  stats: host or
 * device array [n_steps], nullable.  A host array synchronises at the end
 * (and reports device-side errors); a device array is filled asynchronously
 * (collected_charge left 0) and errors surface at the next pic_sync.
 */
int pic_step(pic_ctx ctx, int64_t n_steps, pic_step_stats *stats);

/*
 * pic_adjoint: the charge Q collected through Gamma_1 over n_steps steps from
 * the current state, and its derivatives with respect to the applied field
 * of each replica and the work function of each emitting face, by reverse
 * mode over the steps of Sec. II.B.
 *
 * The run starts with a deposit and a Poisson solve of the SPs present (so
 * Phi_0 follows E0 too) and then takes n_steps ordinary steps; the context is
 * left in the state after them.  Q is piecewise constant in the parameters
 * (stochastic rounding of the SP counts, eq. rnd_nsp; discrete cell crossings
 * and exits), so the derivative is that of the smooth model obtained by
 * freezing the discrete decisions of this run: every SP injected from
 * quadrangle q carries the weight n_sp,q(theta) / n_sp,q(theta0) (eq. nsp,
 * n_sp proportional to J_FN(F_q, phi_f)); counts, random numbers, cells at
 * the start of each step, fates, final cells and periodic shifts are those of
 * the run; the deposit is taken without the integer rounding; the potential
 * is the solution of M Phi = f.  Q = q w_sp sum over collected SPs of the
 * weight.
 *
 * Memory: the state is kept every ckpt_every steps (SPs and Phi); the reverse
 * pass recomputes one segment at a time and keeps its per-step SP arrays, so
 * device memory grows with ckpt_every, not with n_steps.  The adjoint Poisson
 * solves (M is symmetric: adjoint CG is CG on the same matrix) use the
 * context's solver with relative residual 1e-10 (FP64 in the FP32_IR form
 * through its FP64 refinement).
 *
 *   Q        HOST double [1]: collected charge [C] (nullable)
 *   dQ_dE0   HOST double [n_rep]: dQ/dE0 of each replica [C m/V] (nullable)
 *   dQ_dphi  HOST double [n_faces]: dQ/dphi_f [C/eV] (nullable)
 * PIC_ERR_ARG for n_steps < 1 or ckpt_every < 1; device errors of the steps
 * as in pic_step.
 */
int pic_adjoint(pic_ctx ctx, int64_t n_steps, int32_t ckpt_every, double *Q, double *dQ_dE0,
                double *dQ_dphi);

/*
 * pic_collide: Monte Carlo binary collisions of the SPs in flight (App. F,
 * after Takizuka & Abe): the SPs of each cell, ordered by a random key of
 * (seed, step, id), are paired (an odd count collides its first three as
 * (0,1), (1,2), (2,0) with half the variance); each pair's relative velocity
 * w = u_a - u_b turns by theta about a uniform azimuth phi (eq. rot_mat),
 * v_{a,b} = u_{a,b} +- M w / 2 (eq. vel12, equal masses: energy and momentum
 * conserved), with delta = tan(theta/2) ~ N(0, q^4 n Lambda dt /
 * (2 pi eps0^2 m^2 |w|^3 V_cell)) (eqs. sin_theta, variance), n the real
 * electrons in the cell (SPs x w_sp).  pic_step runs it after every push
 * when params.collisions = 1 (pic_adjoint then refuses:
 * PIC_ERR_NOT_IMPLEMENTED).  Random keys: replica seed, step, 2^40 + cell
 * index within the replica, collision index, slots 1..3.
 */
int pic_collide(pic_ctx ctx, int64_t step);

/* Prescribed potential on the Dirichlet nodes (node_dirichlet of mesh_load):
 * HOST double [n_nodes], values on other nodes ignored; default 0.  The free
 * equations gain the load -sum_{j Dirichlet} M_ij g_j (the prescribed part of
 * the P1 solution moved to the right-hand side, App. B); Phi takes the values
 * at once, the free part is not re-solved.  A Dirichlet anode is the top
 * plane's nodes marked Dirichlet with g = V (SPs still leave through
 * Gamma_1 as collected). */
int pic_set_dirichlet(pic_ctx ctx, const double *values);

/* Applied field of each replica (E0 of the Neumann condition on Gamma_1,
 * eq. poisson_bc): HOST double [n_rep]; the Neumann load is rebuilt as in
 * mesh_load, the potential is not re-solved. */
int pic_set_applied_field(pic_ctx ctx, const double *E0);

/* ---- state (checkpoint / resume, parity) ---- */
int pic_get_step(pic_ctx ctx, int64_t *step);
int pic_set_step(pic_ctx ctx, int64_t step);
/* phi: host or device double [n_nodes]; Dirichlet nodes read/write as 0 */
int pic_get_potential(pic_ctx ctx, double *phi);
/* The same copy queued on the context's stream without waiting for it: phi
 * (host memory should be pinned, else the driver stages it synchronously,
 * or device) holds the potential once the stream has passed the call --
 * after pic_sync, or after an event the caller records on the context's
 * stream following the call.  Lets a caller read step k's result while
 * step k + 1 runs. */
int pic_get_potential_async(pic_ctx ctx, double *phi);
int pic_set_potential(pic_ctx ctx, const double *phi);
/* E: host or device double [n_tets*3], the field of the current Phi */
int pic_get_field(pic_ctx ctx, double *E);
/* W of the last deposit: host or device int64 [n_nodes] */
int pic_get_charge(pic_ctx ctx, int64_t *W);
/* number of SPs in flight (synchronises) */
int pic_num_particles(pic_ctx ctx, int64_t *n);
/* r, v: host or device double [n*3] (xyz interleaved); cell: int32 [n];
 * id: int64 [n]; n = pic_num_particles; any pointer nullable.  The order of
 * SPs is unspecified (sort by id to compare). */
int pic_get_particles(pic_ctx ctx, double *r, double *v, int32_t *cell, int64_t *id);
/* replace the SPs (none fresh); cell must hold the tetrahedron containing r */
int pic_set_particles(pic_ctx ctx, int64_t n, const double *r, const double *v,
                      const int32_t *cell, const int64_t *id);
/* work function per emitting face: host or device double [n_faces] */
int pic_set_work_function(pic_ctx ctx, const double *work_function_eV);

/* ---- counters ---- */
/* Number of this library's kernel launches since the context was created. */
int pic_launch_count(pic_ctx ctx, int64_t *launches);
/* Per-kernel device time recorded with CUDA events on the context's stream
 * while profiling is enabled.  names[i] points to static strings. */
#define PIC_PROF_MAX 16
typedef struct {
    int32_t n;
    const char *name[PIC_PROF_MAX];
    int64_t launches[PIC_PROF_MAX];
    double ms[PIC_PROF_MAX];
} pic_profile_report;
int pic_profile_enable(pic_ctx ctx, int32_t enable);  /* also clears */
int pic_profile_read(pic_ctx ctx, pic_profile_report *out); /* synchronises */
/* Wait for all queued work; returns the first device-side error, if any. */
int pic_sync(pic_ctx ctx);

/* Measurement probe, not part of the cycle: the FP64 fused-multiply-add rate
 * of the current device (2 flops per FMA), measured with a kernel of
 * independent FMA chains on `stream` (a cudaStream_t, nullable: the default
 * stream) over `iters` (>= 1) iterations per chain, timed with CUDA events
 * after one untimed launch; the FP64 form's roofline (the FP64 walk, Sec.
 * II.B.2) is set against it.  *tflops: HOST, TFLOP/s.  Allocates and frees
 * its own scratch and synchronises `stream`; PIC_ERR_ARG for iters < 1 or a
 * null tflops, PIC_ERR_CUDA on a CUDA error. */
int pic_measure_fp64_rate(void *stream, int32_t iters, double *tflops);

/*
 * pic_pcg_solve_static: Jacobi-preconditioned CG on a caller-supplied sparse
 * symmetric positive definite system A x = b that allocates no device memory
 * (the paper has no counterpart; this serves callers of the library, not the
 * method).  It is for callers that cannot call cudaMalloc -- an application
 * that runs inside a device arena it manages itself, or under an allocator
 * that is locked or budgeted elsewhere -- and so cannot create a pic_ctx.
 * The caller passes every input and output; the solver's work vectors live
 * in one file-scope device array of PIC_STATIC_MAX_ROWS rows (about 10 MiB)
 * that each GPU loading the library holds until the process exits.
 *   n                     rows, 1 <= n <= PIC_STATIC_MAX_ROWS (else PIC_ERR_ARG,
 *                         nothing is launched)
 *   rowptr[n+1], col[nnz] DEVICE int32 CSR pattern, 0-based: rowptr starts
 *                         at 0, never decreases and ends at nnz (the length
 *                         of col and val); every column in [0, n); the
 *                         diagonal must be stored.  A decreasing rowptr or a
 *                         column outside [0, n) is found by the kernel
 *                         before any value is read through it and gives
 *                         PIC_ERR_ARG; a rowptr whose last entry exceeds
 *                         the arrays' length cannot be detected.
 *   val[nnz], b[n]        DEVICE double
 *   x[n]                  DEVICE double: initial guess in, solution out
 *   rtol, max_iter        stop when ||b - A x||_2 <= rtol ||b||_2 (recursive
 *                         residual), PIC_ERR_NOT_CONVERGED at max_iter (iters
 *                         = max_iter) or on a CG breakdown (p.Ap <= 0, or a
 *                         non-finite value during the iterations)
 *   iters, rel_res        HOST, nullable
 *   stream                cudaStream_t (NULL = legacy default stream)
 * A non-finite value in A, b or the initial x gives PIC_ERR_ARG (it reaches
 * the first pass's sums; x is then left as it was).  Every call copies its
 * status words to the host and synchronises `stream` before it returns.
 * The first call on a device, with that
 * device current, looks up the device address of the scratch array and the
 * resident grid size; make that first call before any stream capture.  All
 * calls on a device share the scratch array (each clears the words that must
 * start at zero): calls whose kernels overlap on the GPU race, so serialise
 * them.  Errors: PIC_ERR_ARG, PIC_ERR_CUDA, PIC_ERR_NOT_CONVERGED,
 * PIC_ERR_TIMEOUT; the message is in pic_last_error(NULL).
 */
#define PIC_STATIC_MAX_ROWS 262144
int pic_pcg_solve_static(int32_t n, const int32_t *rowptr, const int32_t *col,
                         const double *val, const double *b, double *x, double rtol,
                         int32_t max_iter, int32_t *iters, double *rel_res, void *stream);

#ifdef __cplusplus
}
#endif
#endif
