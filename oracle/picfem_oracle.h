/*
 * picfem_oracle.h -- plain FP64 CPU reference of the electrostatic FEM-PIC cycle
 * of Veske et al., "Dynamic coupling between particle-in-cell and atomistic
 * simulations" (Phys. Rev. E 101, 053307; arXiv 1906.08125).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA library
 * against the paper.  Only the test suite, the smoke entry and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or helper
 * with the CUDA library, and it never reads anything the CUDA library wrote.
 *
 * Every routine is written for a reader to check against the paper by eye:
 * sequential loops, no blocking, no reordering beyond what the cited
 * equation fixes.  Build with -ffp-contract=off so that no multiply-add is
 * fused.
 *
 * Parity unpinned: the absolute emission current on tip geometries (the paper
 * takes it from the external GETELEC code and its figures are not available);
 * only the closed-form Fowler-Nordheim expression is pinned.
 */
#ifndef PICFEM_ORACLE_H
#define PICFEM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
enum {
    OR_OK = 0,
    OR_ERR_ARG = -1,
    OR_ERR_MESH = -3,
    OR_ERR_CAPACITY = -4,
    OR_ERR_WALK_LIMIT = -5,
    OR_ERR_NOT_CONVERGED = -6
};

/* boundary codes stored in the neighbour table (face i is opposite vertex i) */
enum { OR_TOP = -1, OR_CATHODE = -2, OR_SIDE = -3 };

/* Fowler-Nordheim model */
enum { OR_FN_MURPHY_GOOD = 0, OR_FN_ELEMENTARY = 1 };

typedef struct {
    double dt;           /* PIC time step [s]                                   */
    double E0;           /* applied far field [V/m] (Neumann data on Gamma_1)    */
    double w_sp;         /* superparticle weight (real electrons per SP)         */
    double q;            /* charge of one real particle [C] (-e for electrons)   */
    double q_over_m;     /* charge-to-mass ratio [C/kg]                          */
    double eps0;         /* vacuum permittivity [F/m]                            */
    double e_charge;     /* elementary charge [C] used in eq. (nsp)              */
    double pcg_rtol;     /* ||r||_2 <= rtol ||f||_2                              */
    int32_t pcg_max_iter;
    int32_t fn_model;    /* OR_FN_*                                              */
    uint64_t seed;
    int64_t capacity;    /* maximum number of SPs in flight                      */
    int32_t walk_max_steps;
    int32_t quant_bits;  /* S: deposit weights are integers of 2^-S              */
    int32_t collisions;  /* 1: binary collisions after each push (App. F)         */
    int32_t pad;
    double coulomb_log;  /* Lambda of the scattering variance (App. F: 13)         */
} or_params;

typedef struct {
    int64_t injected;
    int64_t collected;    /* left through Gamma_1 (top)                         */
    int64_t absorbed;     /* left through Gamma_3 (cathode)                     */
    int64_t wrapped;      /* periodic crossings of Gamma_2                      */
    int64_t crossings;    /* face crossings summed over all SPs                 */
    int64_t alive;        /* SPs in flight after the step                       */
    int32_t max_walk;     /* longest walk of one SP (face crossings)            */
    int32_t pcg_iters;
    double  pcg_relres;
    double  collected_charge; /* q * w_sp * collected [C]                       */
} or_stats;

typedef struct or_ctx or_ctx;

or_ctx *or_create(const or_params *p);
void or_destroy(or_ctx *c);

int or_mesh_load(or_ctx *c, int32_t n_nodes, const double *xyz,
                 int32_t n_tets, const int32_t *tet, const int32_t *nbr,
                 const int32_t *periodic_nbr, const uint8_t *node_dirichlet,
                 int32_t n_faces, const int32_t *face_nodes,
                 const int32_t *face_tet, const double *work_function_eV);

/* derived data, for the pins */
int32_t or_n_free(const or_ctx *c);
int64_t or_nnz(const or_ctx *c);
void or_geometry(const or_ctx *c, double *jinv9, double *x0_3, double *vol);
void or_matrix(const or_ctx *c, int32_t *dof_of_node, int32_t *rowptr,
               int32_t *col, double *val, double *f_neumann);
void or_element_stiffness(const double *x4x3, double *k16);

/* pure functions */
double or_fn_current(double F_V_per_m, double phi_eV, int model);
double or_uniform(uint64_t seed, uint64_t step, uint64_t quad, uint64_t j,
                  uint64_t slot);
uint64_t or_splitmix64_next(uint64_t *state);

/* state */
int or_init_potential(or_ctx *c, int32_t *iters, double *relres);
void or_get_potential(const or_ctx *c, double *phi);
void or_set_potential(or_ctx *c, const double *phi);
void or_set_dirichlet(or_ctx *c, const double *g);
void or_get_field(const or_ctx *c, double *E3);
int64_t or_num_particles(const or_ctx *c);
void or_get_particles(const or_ctx *c, double *r3, double *v3, int32_t *cell,
                      int64_t *id);
int or_set_particles(or_ctx *c, int64_t n, const double *r3, const double *v3,
                     const int32_t *cell, const int64_t *id);
void or_get_charge(const or_ctx *c, int64_t *W);
int64_t or_step_index(const or_ctx *c);
void or_set_step_index(or_ctx *c, int64_t step);
void or_set_work_function(or_ctx *c, const double *wf);

/* the steps of the cycle, in the order of one PIC step */
int or_inject(or_ctx *c, int64_t step, int64_t *n_injected);
int or_push_relocate(or_ctx *c, int64_t step, or_stats *st);
int or_deposit(or_ctx *c);
int or_poisson_solve(or_ctx *c, int32_t *iters, double *relres);
/* M x = f for a caller's right-hand side f (free DOFs in or_matrix's
 * numbering), Jacobi-PCG from the x given to ||f - M x|| <= rtol ||f|| */
int or_solve(or_ctx *c, const double *f, double *x, double rtol, int32_t max_iter,
             int32_t *iters, double *relres);
int or_step(or_ctx *c, int64_t n_steps, or_stats *stats);
void or_collide(or_ctx *c, int64_t step);

/* point location by the neighbour walk alone (no push): for the pins */
int or_locate(const or_ctx *c, int64_t n, double *r3, int32_t *cell,
              int32_t *fate, int32_t *walk_len);
/* barycentric coordinates of r in tet t */
void or_barycentric(const or_ctx *c, int32_t t, const double *r, double *lam4);

/* per-quadrangle emission numbers of the current field (for the pins) */
void or_quad_emission(const or_ctx *c, double *F, double *J, double *n_sp);
/* threads of the parallel loops of an OpenMP build (n <= 0: unchanged);
 * returns the number in use (1 in a serial build) */
int or_set_threads(int n);
/* the same numbers from a given per-tetrahedron field E3 [n_tets*3] */
void or_quad_emission_field(const or_ctx *c, const double *E3, double *F, double *J,
                            double *n_sp);

#ifdef __cplusplus
}
#endif
#endif
