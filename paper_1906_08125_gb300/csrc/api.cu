// api.cu -- the C ABI of libpicfem (include/picfem.h): context, mesh loading
// (validation, topology tables and the sparsity pattern are built on the
// host; geometry and matrix values are computed by kernels), state access and
// the orchestration of one PIC step on the context's stream.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

using namespace pf;

namespace {

enum KernelId {
    K_FIELD,
    K_INJECT_COUNT,
    K_INJECT_SCAN,
    K_INJECT_EMIT,
    K_PUSH_RELOCATE,
    K_DEPOSIT,
    K_STEP_FUSED,
    K_PCG,
    K_UTIL,
    K_COMPACT,
    K_ADJ_FIELD,
    K_ADJ_ROWS,
    K_ADJ_SP,
    K_COLLIDE,
    K_SORT,
    K_NUM
};
const char *const kKernelNames[K_NUM] = {"field",          "inject_count", "inject_scan",
                                         "inject_emit",    "push_relocate", "deposit",
                                         "step_fused",     "pcg",          "util",
                                         "compact",        "adj_field",    "adj_rows",
                                         "adj_sp",         "collide",      "sort"};

struct ProfRec {
    int kid;
    cudaEvent_t a, b;
};

}  // namespace

struct pic_ctx_s {
    pic_params p{};
    cudaStream_t s = nullptr;
    int dev = 0, num_sms = 0, l2_bytes = 0;
    std::string err;
    // sizes
    int N = 0, T = 0, F = 0, NQ = 0, n_free = 0, n_pad = 0, n_slices = 0;
    long long sell_len = 0, nnz = 0;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    bool loaded = false;
    std::vector<void *> allocs;  // mesh-lifetime device buffers
    // mesh
    double *xyz = nullptr;
    int4 *tet4 = nullptr;
    TetRec64 *rec64 = nullptr;
    TetRec32 *rec32 = nullptr;
    double *det = nullptr;
    unsigned char *dir = nullptr;
    int *face_nodes = nullptr, *face_tet = nullptr;
    double *wf = nullptr, *fnhat = nullptr, *farea = nullptr;
    int *dof_node = nullptr, *slice_ptr = nullptr, *col = nullptr;
    int *lcol = nullptr, *halo_ptr = nullptr, *halo_idx = nullptr;
    double *val64 = nullptr, *dinv64 = nullptr, *fN = nullptr;
    float *val32 = nullptr, *dinv32 = nullptr;
    // state
    double *phi = nullptr, *x = nullptr;
    void *E = nullptr;
    unsigned long long *W = nullptr;
    void *pbuf[2][6] = {{nullptr}};
    int *cell[2] = {nullptr, nullptr};
    long long *id[2] = {nullptr, nullptr};
    int a = 0;
    DevState *st = nullptr;
    int *qcount = nullptr;
    long long *qoff = nullptr;
    // pcg
    double *f = nullptr, *r = nullptr, *z = nullptr, *p0 = nullptr, *p1 = nullptr, *ap = nullptr;
    float *r32 = nullptr, *z32 = nullptr, *p32_0 = nullptr, *p32_1 = nullptr, *ap32 = nullptr,
          *dx32 = nullptr;
    double *d0 = nullptr, *d1 = nullptr;
    float *d32_0 = nullptr, *d32_1 = nullptr;
    unsigned long long *dtag = nullptr;   // [2 * n_pad] tagged Chebyshev halo values
    unsigned *pcg_epoch = nullptr;        // launches of the resident solver (mod 255)
    double cheb_b = 2.0;   // Gershgorin bound of D^-1 M
    const float *coarse_inv = nullptr;   // two-level preconditioner: A0^-1 of the blocks
    double *coarse_r = nullptr;
    // general kernels' coarse correction: aggregates per group and their A0^-1
    const int *agg_off = nullptr;
    const long long *inv_off = nullptr;
    const float *agg_inv = nullptr;
    double *slice_r = nullptr, *agg_r = nullptr, *agg_z = nullptr;
    // multigrid hierarchy of the resident solver (mg.cu; n1 == 0: none)
    struct {
        int n1 = 0, n2 = 0, max_l1_local = 0, max_l1_own = 0, max_l2_own = 0;
        double lmax1 = 2.0;
        int *agg0 = nullptr, *l1_off = nullptr, *l2_off = nullptr, *m0_ptr = nullptr,
            *m0_idx = nullptr, *a1_ptr = nullptr, *a1_col = nullptr, *h1_ptr = nullptr,
            *h1_idx = nullptr, *agg1 = nullptr, *m1_ptr = nullptr, *m1_idx = nullptr;
        float *a1_val32 = nullptr, *dinv1_32 = nullptr, *a2inv = nullptr, *r2f = nullptr;
        double *a1_val64 = nullptr, *dinv1_64 = nullptr, *r2d = nullptr;
        float *g1f[2] = {nullptr, nullptr};
        double *g1d[2] = {nullptr, nullptr};
        unsigned long long *dtag1 = nullptr;
    } mg;
    // multigrid hierarchy of the general kernels (mg.cu gmg_build; nlev == 0: none)
    struct {
        int nlev = 0, coarse_max = 0;
        const GmgLevel *levels = nullptr;   // [nlev + 1], device
        const float *inv = nullptr;
        const long long *ioff = nullptr;
        const int *cn = nullptr;
    } gmg;
    // replicas of a batch (1 for a single mesh)
    int n_rep = 1, n_rows = 0;
    int *tet_rep = nullptr, *face_rep = nullptr, *rep_face_off = nullptr;
    double *rep_L = nullptr, *E0_rep = nullptr;
    int *grp = nullptr, *blk_grp = nullptr;
    unsigned *grp_bar = nullptr;
    double *partials = nullptr;
    double *part8 = nullptr;   // [2][grid][8] block values of the one-reduction CG
    PcgLaunch plan{};
    pic_step_stats *dstats = nullptr;  // per-step stats of pic_step
    long long dstats_cap = 0;
    pic_step_stats *sstats = nullptr;  // scratch stats of the split calls
    pic_step_stats *slot = nullptr;    // statistics of the step in progress
    // CUDA graphs of one step, one per particle-buffer parity (graph_state:
    // 1 captured, 0 not tried, -1 capture refused: direct launches)
    cudaStream_t cap_s = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    long long glaunch[2] = {0, 0};
    int gnext[2] = {1, 0};   // buffer parity after a replay of each graph
    int graph_state = 0;
    // staging
    void *stage[4] = {nullptr, nullptr, nullptr, nullptr};
    size_t stage_sz[4] = {0, 0, 0, 0};
    int64_t step = 0;
    long long launches = 0;
    int pgrid = 0;
    // launch tuning (pic_set_tuning)
    int walk_form = WALK_FORM_AUTO, pcg_bps = 0, pcg_balance = 1, cheb_local = 0, sort_cells = 1,
        halo_sync = 1, wait_limit = 0, mg_deg0 = 0, mg_deg1 = 0;   // 0: the default
    int *scnt = nullptr, *soff = nullptr, *srank = nullptr, *sscan = nullptr;   // sort scratch
    std::vector<int> rep_slice;   // first slice of each replica (batch solve plan)
    int *grp_iters = nullptr;     // iterations of each replica's last solve
    int *nfptr = nullptr, *nfcon = nullptr;   // Neumann contributions per row
    int *dptr = nullptr, *dcon = nullptr;     // Dirichlet couplings per row
    double *gD = nullptr, *fD = nullptr;      // prescribed values (nodes), their load (rows)
    std::vector<unsigned char> dir_h;         // Dirichlet flags (host copy)
    int *rep_tet_off_d = nullptr;             // first tetrahedron of each replica
    // collision scratch (allocated with the mesh when params.collisions, else on
    // the first pic_collide)
    int *ccnt = nullptr, *coff = nullptr, *cfill = nullptr, *cperm = nullptr, *cscan = nullptr;
    unsigned long long *ckey = nullptr;
    int *rep_slice_d = nullptr;   // rep_slice on the device
    std::vector<long long> rep_sell;   // stored matrix entries of each replica
    std::vector<int> rep_free;         // free DOFs of each replica
    std::vector<int> grp_h, blk_grp_h;   // the batch plan's tables (host copies)
    // profiling
    bool prof = false;
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> ev_pool;
    double prof_ms[K_NUM] = {0};
    long long prof_n[K_NUM] = {0};
};

namespace {

std::string g_err;

int fail(pic_ctx c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    else
        g_err = buf;
    return code;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(c, PIC_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                            \
    } while (0)

cudaEvent_t take_event(pic_ctx c)
{
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct ProfScope {
    pic_ctx c;
    int kid;
    cudaEvent_t a = nullptr;
    ProfScope(pic_ctx c_, int k) : c(c_), kid(k)
    {
        if (c->prof) {
            a = take_event(c);
            cudaEventRecord(a, c->s);
        }
    }
    ~ProfScope()
    {
        if (a) {
            cudaEvent_t b = take_event(c);
            cudaEventRecord(b, c->s);
            c->prof_recs.push_back({kid, a, b});
        }
    }
};

#define LAUNCH(kid, call)                                                                  \
    do {                                                                                   \
        ProfScope ps_(c, kid);                                                             \
        cudaError_t e_ = (call);                                                           \
        ++c->launches;                                                                     \
        if (e_ != cudaSuccess)                                                             \
            return fail(c, PIC_ERR_CUDA, "launch %s: %s", kKernelNames[kid],               \
                        cudaGetErrorString(e_));                                           \
    } while (0)

template <typename T> cudaError_t dalloc(pic_ctx c, T **p, size_t n)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, n ? n * sizeof(T) : 16);
    if (e == cudaSuccess) {
        c->allocs.push_back(q);
        *p = (T *)q;
    }
    return e;
}

void free_graphs(pic_ctx c)
{
    for (int a = 0; a < 2; ++a) {
        if (c->gexec[a])
            cudaGraphExecDestroy(c->gexec[a]);
        c->gexec[a] = nullptr;
        c->glaunch[a] = 0;
    }
    c->graph_state = 0;
}

void free_mesh(pic_ctx c)
{
    free_graphs(c);
    for (void *q : c->allocs)
        cudaFree(q);
    c->allocs.clear();
    c->loaded = false;
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

cudaError_t stage(pic_ctx c, int slot, size_t bytes, void **out)
{
    if (c->stage_sz[slot] < bytes) {
        if (c->stage[slot])
            cudaFree(c->stage[slot]);
        c->stage[slot] = nullptr;
        c->stage_sz[slot] = 0;
        cudaError_t e = cudaMalloc(&c->stage[slot], bytes);
        if (e != cudaSuccess)
            return e;
        c->stage_sz[slot] = bytes;
    }
    *out = c->stage[slot];
    return cudaSuccess;
}

int check_device_error(pic_ctx c)
{
    DevState h;
    CK(cudaMemcpyAsync(&h, c->st, sizeof h, cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    if (h.err) {
        const char *what = h.err == PIC_ERR_CAPACITY        ? "particle capacity exceeded"
                           : h.err == PIC_ERR_WALK_LIMIT    ? "an SP exceeded walk_max_steps"
                           : h.err == PIC_ERR_NOT_CONVERGED ? "PCG reached pcg_max_iter"
                           : h.err == PIC_ERR_TIMEOUT       ? "device-side wait timed out"
                           : h.err == PIC_ERR_ARG           ? "injection rejection limit"
                                                            : "device error";
        int code = h.err;
        int zero = 0;
        cudaMemcpy(&c->st->err, &zero, sizeof zero, cudaMemcpyHostToDevice);
        return fail(c, code, "%s (device status %d)", what, code);
    }
    return PIC_OK;
}

bool fp64(pic_ctx c) { return c->p.precision == PIC_PREC_FP64; }

template <typename R> Particles<R> parts(pic_ctx c, int b)
{
    Particles<R> P;
    P.x = (R *)c->pbuf[b][0];
    P.y = (R *)c->pbuf[b][1];
    P.z = (R *)c->pbuf[b][2];
    P.vx = (R *)c->pbuf[b][3];
    P.vy = (R *)c->pbuf[b][4];
    P.vz = (R *)c->pbuf[b][5];
    P.cell = c->cell[b];
    P.id = c->id[b];
    return P;
}

template <typename R> MeshView<R> view(pic_ctx c)
{
    MeshView<R> m;
    if constexpr (sizeof(R) == 8)
        m.rec = (const typename Rec<R>::type *)c->rec64;
    else
        m.rec = (const typename Rec<R>::type *)c->rec32;
    m.tet = c->tet4;
    m.E = (const typename Rec<R>::vec4 *)c->E;
    m.face_nodes = c->face_nodes;
    m.face_tet = c->face_tet;
    m.face_nhat = c->fnhat;
    m.face_area = c->farea;
    m.wf = c->wf;
    m.xyz = c->xyz;
    m.n_faces = c->F;
    m.tet_rep = c->tet_rep;
    m.face_rep = c->face_rep;
    m.rep_face_off = c->rep_face_off;
    m.rep_L = c->rep_L;
    return m;
}

RunConst run_const(pic_ctx c)
{
    RunConst k;
    k.dt = c->p.dt;
    k.qmdt = c->p.q_over_m * c->p.dt;
    k.w_sp = c->p.w_sp;
    k.e_charge = c->p.e_charge;
    k.scale = std::ldexp(1.0, c->p.quant_bits);
    k.seed = c->p.seed;
    k.capacity = c->p.capacity;
    k.fn_model = c->p.fn_model;
    k.walk_max = c->p.walk_max_steps;
    return k;
}

__global__ void k_phi_to_x(int n, const int *dof_node, const double *phi, double *x)
{
    int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d < n)
        x[d] = dof_node[d] >= 0 ? phi[dof_node[d]] : 0.0;
}
// Phi on the Dirichlet nodes: the prescribed values (0 unless pic_set_dirichlet)
__global__ void k_set_dirichlet(int N, const unsigned char *dir, const double *gD, double *phi)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N && dir[i])
        phi[i] = gD[i];
}

// E from Phi; at the end of a pic_step step it also files the step's
// statistics and advances the device-side step index.
int refresh_field(pic_ctx c, bool end_of_step = false)
{
    DevState *st = end_of_step ? c->st : nullptr;
    if (fp64(c))
        LAUNCH(K_FIELD, launch_field<double>(c->s, c->T, c->rec64, c->tet4, c->phi, (Vec4d *)c->E,
                                             st, c->slot));
    else
        LAUNCH(K_FIELD, launch_field<float>(c->s, c->T, c->rec32, c->tet4, c->phi, (float4 *)c->E,
                                            st, c->slot));
    return PIC_OK;
}

// Smoothing degree of the V-cycle on the fine level (k = 0) or below (k = 1):
// the tuned value, else the default of the solver in use (the resident one
// smooths both levels with degree 3; the general one, whose fine-level
// products stream the matrix from HBM, smooths the fine level with degree 1,
// a scaled Jacobi step, and the coarser ones with degree 3)
static int mg_degree(pic_ctx c, int k)
{
    const int t = k == 0 ? c->mg_deg0 : c->mg_deg1;
    if (t > 0)
        return t;
    if (c->plan.resident)
        return k == 0 ? MG_DEGREE0 : MG_DEGREE1;
    return k == 0 ? GMG_DEGREE0 : GMG_DEGREE1;
}

// Chebyshev iteration on [lo, hi] (Saad, Alg. 12.1): theta, delta, sigma and
// the recurrence rho_j = 1 / (2 sigma - rho_j-1), rho_0 = 1 / sigma; the steps
// d_j+1 = c1[j] d_j + c2[j] D^-1 r_j after d_1 = D^-1 r / theta
static void cheb_coefficients(double lo, double hi, int n, double *c1, double *c2,
                              double *inv_theta)
{
    const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
    const double sigma = delta > 0 ? theta / delta : 1.0;
    double rho = 1.0 / sigma;
    *inv_theta = 1.0 / theta;
    for (int j = 0; j < n; ++j) {
        const double rho_new = 1.0 / (2.0 * sigma - rho);
        c1[j] = rho_new * rho;
        c2[j] = delta > 0 ? 2.0 * rho_new / delta : 0.0;
        rho = rho_new;
    }
}

// A solve with a right-hand side of the caller's (the adjoint solves): f =
// rhs (rows), iterate and result in x (rows, warm start), scattered to the
// node array out; stopping at relative residual rtol.
struct SolveOverride {
    const double *rhs;
    double *x;
    double *out;
    double rtol;
};

int run_pcg(pic_ctx c, pic_step_stats *stats, const unsigned long long *alive,
            const SolveOverride *ov = nullptr)
{
    PcgArgs g{};
    g.n = c->n_rows;
    g.n_pad = c->n_pad;
    g.n_slices = c->n_slices;
    g.slice_ptr = c->slice_ptr;
    g.col = c->col;
    g.val64 = c->val64;
    g.val32 = c->val32;
    g.dinv64 = c->dinv64;
    g.dinv32 = c->dinv32;
    g.fN = c->fN;
    g.W = c->W;
    g.dof_node = c->dof_node;
    g.coef = (c->p.q * c->p.w_sp) / c->p.eps0;
    g.wscale = std::ldexp(1.0, -c->p.quant_bits);
    g.x = c->x;
    g.phi = c->phi;
    g.f = c->f;
    g.r = c->r;
    g.z = c->z;
    g.p0 = c->p0;
    g.p1 = c->p1;
    g.ap = c->ap;
    g.r32 = c->r32;
    g.z32 = c->z32;
    g.p32_0 = c->p32_0;
    g.p32_1 = c->p32_1;
    g.ap32 = c->ap32;
    g.dx32 = c->dx32;
    g.partials = c->partials;
    g.part8 = c->part8;
    g.st = c->st;
    g.stats = stats;
    g.alive = alive;
    g.rtol = c->p.pcg_rtol;
    g.inner_rtol = c->p.ir_inner_rtol;
    g.max_iter = c->p.pcg_max_iter;
    g.precision = c->p.precision;
    g.max_rows = c->plan.max_rows;
    g.max_chunk = c->plan.max_chunk;
    g.variant = c->p.pcg_variant;
    g.lcol = c->lcol;
    g.halo_ptr = c->halo_ptr;
    g.halo_idx = c->halo_idx;
    g.max_local = c->plan.max_local;
    g.cheb_degree = c->p.pcg_cheb_degree;
    g.cheb_b = c->cheb_b;
    g.cheb_a = (c->p.pcg_cheb_degree >= 2 || (c->cheb_local == 4 && c->mg.n1 > 0))
                   ? c->cheb_b / c->p.pcg_cheb_ratio
                   : 0.0;
    cheb_coefficients(g.cheb_a, g.cheb_b, 32, g.cheb_c1, g.cheb_c2, &g.cheb_inv_theta);
    g.cheb_inv_thetaf = (float)g.cheb_inv_theta;
    for (int j = 0; j < 32; ++j) {
        g.cheb_c1f[j] = (float)g.cheb_c1[j];
        g.cheb_c2f[j] = (float)g.cheb_c2[j];
    }
    g.d0 = c->d0;
    g.d1 = c->d1;
    g.d32_0 = c->d32_0;
    g.d32_1 = c->d32_1;
    g.dtag[0] = g.dtag[1] = nullptr;
    if (c->dtag && c->halo_sync == 1 && c->plan.resident && c->plan.halo_symmetric) {
        g.dtag[0] = c->dtag;
        g.dtag[1] = c->dtag + c->n_pad;
    }
    g.epoch = c->pcg_epoch;
    g.spin_limit = c->wait_limit > 0 ? (long long)c->wait_limit : PCG_SPIN_LIMIT_DEFAULT;
    g.inner_max = c->p.ir_inner_max_iter;
    g.n_groups = c->plan.n_groups;
    g.grp = c->grp;
    g.blk_grp = c->blk_grp;
    g.grp_bar = c->grp_bar;
    g.grp_iters = c->grp_iters;
    // stream the matrix past L2 when it does not fit in about half of it
    const double mat_bytes = (double)c->sell_len * (fp64(c) ? 12.0 : 8.0);
    g.stream_matrix = mat_bytes > 0.5 * (double)c->l2_bytes ? 1 : 0;
    g.rhs = nullptr;
    g.fD = c->fD;
    g.cheb_local = c->cheb_local;
    if (c->mg.n1 > 0 && c->cheb_local == 4) {
        g.mg_n1 = c->mg.n1;
        g.mg_n2 = c->mg.n2;
        g.mg_deg0 = mg_degree(c, 0);
        g.mg_deg1 = mg_degree(c, 1);
        g.mg_max_l1_local = c->mg.max_l1_local;
        g.mg_max_l1_own = c->mg.max_l1_own;
        g.mg_max_l2_own = c->mg.max_l2_own;
        g.mg_smem_off = c->plan.mg_off;
        g.mg_agg0 = c->mg.agg0;
        g.mg_l1_off = c->mg.l1_off;
        g.mg_l2_off = c->mg.l2_off;
        g.mg_m0_ptr = c->mg.m0_ptr;
        g.mg_m0_idx = c->mg.m0_idx;
        g.mg_a1_ptr = c->mg.a1_ptr;
        g.mg_a1_col = c->mg.a1_col;
        g.mg_a1_val32 = c->mg.a1_val32;
        g.mg_a1_val64 = c->mg.a1_val64;
        g.mg_dinv1_32 = c->mg.dinv1_32;
        g.mg_dinv1_64 = c->mg.dinv1_64;
        g.mg_h1_ptr = c->mg.h1_ptr;
        g.mg_h1_idx = c->mg.h1_idx;
        g.mg_agg1 = c->mg.agg1;
        g.mg_m1_ptr = c->mg.m1_ptr;
        g.mg_m1_idx = c->mg.m1_idx;
        g.mg_a2inv = c->mg.a2inv;
        g.mg_r2f = c->mg.r2f;
        g.mg_r2d = c->mg.r2d;
        g.mg_dtag1 = (!fp64(c) && c->halo_sync == 1) ? c->mg.dtag1 : nullptr;
        for (int k = 0; k < 2; ++k) {
            g.mg_g1f[k] = c->mg.g1f[k];
            g.mg_g1d[k] = c->mg.g1d[k];
        }
        // level-1 Chebyshev coefficients on [lmax1 / ratio, lmax1]
        const double b1 = c->mg.lmax1;
        cheb_coefficients(b1 / c->p.pcg_cheb_ratio, b1, 32, g.mg_c1, g.mg_c2, &g.mg_inv_theta);
        g.mg_inv_thetaf = (float)g.mg_inv_theta;
        for (int j = 0; j < 32; ++j) {
            g.mg_c1f[j] = (float)g.mg_c1[j];
            g.mg_c2f[j] = (float)g.mg_c2[j];
        }
    }
    if (c->gmg.nlev > 0 && c->cheb_local == 4 && !c->plan.resident) {
        g.gmg_nlev = c->gmg.nlev;
        g.gmg_deg0 = mg_degree(c, 0);
        g.gmg_deg1 = mg_degree(c, 1);
        g.gmg = c->gmg.levels;
        g.gmg_inv = c->gmg.inv;
        g.gmg_ioff = c->gmg.ioff;
        g.gmg_cn = c->gmg.cn;
    }
    g.coarse_inv = c->coarse_inv;
    g.coarse_r = c->coarse_r;
    g.agg_inv = c->cheb_local == 3 ? c->agg_inv : nullptr;
    g.agg_off = c->agg_off;
    g.inv_off = c->inv_off;
    g.slice_r = c->slice_r;
    g.agg_r = c->agg_r;
    g.agg_z = c->agg_z;
    if (ov) {
        g.rhs = ov->rhs;
        g.x = ov->x;
        g.phi = ov->out;
        g.rtol = ov->rtol;
        g.grp_iters = nullptr;    // the balance follows the forward solves
    }
    CK(cudaMemsetAsync(&c->st->bar_count, 0, sizeof(unsigned), c->s));
    if (c->plan.n_groups > 0)
        CK(cudaMemsetAsync(c->grp_bar, 0, sizeof(unsigned) * c->plan.n_groups, c->s));
    LAUNCH(K_PCG, launch_pcg(c->s, c->plan, g));
    return PIC_OK;
}

int ensure_dstats(pic_ctx c, long long n)
{
    if (c->dstats_cap < n) {
        if (c->dstats)
            cudaFree(c->dstats);
        c->dstats = nullptr;
        c->dstats_cap = 0;
        CK(cudaMalloc(&c->dstats, sizeof(pic_step_stats) * (size_t)n));
        c->dstats_cap = n;
    }
    return PIC_OK;
}

#define REQUIRE_MESH()                                                                   \
    do {                                                                                 \
        if (!c)                                                                          \
            return fail(nullptr, PIC_ERR_ARG, "null context");                           \
        if (!c->loaded)                                                                  \
            return fail(c, PIC_ERR_ARG, "mesh_load has not been called");               \
        CK(cudaSetDevice(c->dev));                                                       \
    } while (0)

}  // namespace

void pf::set_global_error(const char *msg) { g_err = msg; }

// ===========================================================================
// context
// ===========================================================================
extern "C" const char *pic_version(void) { return "libpicfem 0.1 (sm_103a)"; }

extern "C" const char *pic_last_error(pic_ctx c) { return c ? c->err.c_str() : g_err.c_str(); }

extern "C" int pic_create(pic_ctx *out, const pic_params *p, void *stream)
{
    pic_ctx c = nullptr;
    if (!out || !p)
        return fail(nullptr, PIC_ERR_ARG, "pic_create: null argument");
    const pic_params &q = *p;
    if (!(q.dt > 0) || !std::isfinite(q.dt) || !std::isfinite(q.E0) || !(q.w_sp > 0) ||
        !std::isfinite(q.w_sp) || !std::isfinite(q.q) || !std::isfinite(q.q_over_m) ||
        !(q.eps0 > 0) || !(q.e_charge > 0) || !(q.pcg_rtol >= 0) || q.pcg_max_iter < 0 ||
        q.capacity < 1 || q.walk_max_steps < 1 || q.quant_bits < 1 || q.quant_bits > 40 ||
        (q.precision != PIC_PREC_FP64 && q.precision != PIC_PREC_FP32_IR) ||
        (q.fn_model != PIC_FN_MURPHY_GOOD && q.fn_model != PIC_FN_ELEMENTARY) ||
        (q.precision == PIC_PREC_FP32_IR && !(q.ir_inner_rtol > 0 && q.ir_inner_rtol < 1)) ||
        (q.pcg_variant < PIC_PCG_STANDARD || q.pcg_variant > PIC_PCG_SINGLE) ||
        q.ir_inner_max_iter < 0 || q.pcg_cheb_degree < 0 || q.pcg_cheb_degree > 32 ||
        (q.pcg_cheb_degree >= 2 && !(q.pcg_cheb_ratio > 1.0)))
        return fail(nullptr, PIC_ERR_ARG, "pic_create: invalid parameters");
    c = new pic_ctx_s();
    c->p = q;
    c->s = (cudaStream_t)stream;
    if (cudaGetDevice(&c->dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->dev) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return fail(nullptr, PIC_ERR_CUDA, "pic_create: no CUDA device");
    }
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->dev);
    if (!coop) {
        delete c;
        return fail(nullptr, PIC_ERR_CUDA, "pic_create: device lacks cooperative launch");
    }
    // particle kernels: 16 blocks of 256 per SM for the FP32 walk (more SPs
    // claimed in flight hides more of its record-fetch latency), 8 for FP64
    c->pgrid = c->num_sms * (q.precision == PIC_PREC_FP32_IR ? 24 : 8);
    // a Chebyshev-preconditioned solve gets the coarse correction over the
    // solver blocks by default (the plain Jacobi form stays plain)
    c->cheb_local = q.pcg_cheb_degree >= 2 ? 3 : 0;
    cudaDeviceGetAttribute(&c->l2_bytes, cudaDevAttrL2CacheSize, c->dev);
    *out = c;
    return PIC_OK;
}

extern "C" int pic_destroy(pic_ctx c)
{
    if (!c)
        return PIC_OK;
    cudaSetDevice(c->dev);
    cudaStreamSynchronize(c->s);
    free_mesh(c);
    for (int i = 0; i < 4; ++i)
        if (c->stage[i])
            cudaFree(c->stage[i]);
    if (c->dstats)
        cudaFree(c->dstats);
    for (auto &r : c->prof_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : c->ev_pool)
        cudaEventDestroy(e);
    if (c->cap_s)
        cudaStreamDestroy(c->cap_s);
    delete c;
    return PIC_OK;
}

// ===========================================================================
// mesh
// ===========================================================================
// Inverse of a symmetric positive definite n x n matrix (row-major, FP64) by
// Cholesky A = L L^T and one forward/back substitution per column; false if
// A is not positive definite.
static bool spd_inverse(const std::vector<double> &A, int n, float *inv)
{
    std::vector<double> L(A);
    for (int j = 0; j < n; ++j) {
        double d = L[(size_t)j * n + j];
        for (int k = 0; k < j; ++k)
            d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(d > 0.0))
            return false;
        d = std::sqrt(d);
        L[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double v = L[(size_t)i * n + j];
            for (int k = 0; k < j; ++k)
                v -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = v / d;
        }
    }
    std::vector<double> col((size_t)n);
    for (int c0 = 0; c0 < n; ++c0) {
        for (int i = 0; i < n; ++i) {
            double v = i == c0 ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k)
                v -= L[(size_t)i * n + k] * col[k];
            col[i] = v / L[(size_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double v = col[i];
            for (int k = i + 1; k < n; ++k)
                v -= L[(size_t)k * n + i] * col[k];
            col[i] = v / L[(size_t)i * n + i];
        }
        for (int i = 0; i < n; ++i)
            inv[(size_t)i * n + c0] = (float)col[i];
    }
    return true;
}

// copy of a host vector into new device memory of element type T
template <typename T, typename U>
static int upload_vec(pic_ctx c, T **dst, const std::vector<U> &v)
{
    CK(dalloc(c, dst, v.size() + 1));
    if (!v.empty()) {
        std::vector<T> tmp(v.begin(), v.end());
        CK(cudaMemcpy(*dst, tmp.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    }
    return PIC_OK;
}

// the multigrid hierarchy on the device (tables, level-1 matrix in FP32 and
// FP64, the level-2 inverse, exchange buffers)
static int upload_mg(pic_ctx c, const MgHost &m)
{
    auto &d = c->mg;
    int rc = 0;
    if ((rc = upload_vec(c, &d.agg0, m.agg0)) || (rc = upload_vec(c, &d.l1_off, m.l1_off)) ||
        (rc = upload_vec(c, &d.l2_off, m.l2_off)) || (rc = upload_vec(c, &d.m0_ptr, m.m0_ptr)) ||
        (rc = upload_vec(c, &d.m0_idx, m.m0_idx)) || (rc = upload_vec(c, &d.a1_ptr, m.a1_ptr)) ||
        (rc = upload_vec(c, &d.a1_col, m.a1_col)) || (rc = upload_vec(c, &d.h1_ptr, m.h1_ptr)) ||
        (rc = upload_vec(c, &d.h1_idx, m.h1_idx)) || (rc = upload_vec(c, &d.agg1, m.agg1)) ||
        (rc = upload_vec(c, &d.m1_ptr, m.m1_ptr)) || (rc = upload_vec(c, &d.m1_idx, m.m1_idx)) ||
        (rc = upload_vec(c, &d.a1_val32, m.a1_val)) || (rc = upload_vec(c, &d.a1_val64, m.a1_val)) ||
        (rc = upload_vec(c, &d.dinv1_32, m.dinv1)) || (rc = upload_vec(c, &d.dinv1_64, m.dinv1)) ||
        (rc = upload_vec(c, &d.a2inv, m.a2inv)))
        return rc;
    CK(dalloc(c, &d.r2f, (size_t)m.n2));
    CK(dalloc(c, &d.r2d, (size_t)m.n2));
    for (int k = 0; k < 2; ++k) {
        CK(dalloc(c, &d.g1f[k], (size_t)m.n1));
        CK(dalloc(c, &d.g1d[k], (size_t)m.n1));
    }
    CK(dalloc(c, &d.dtag1, 2 * (size_t)m.n1));
    // all-ones tags: no epoch (< 255) produces them
    CK(cudaMemset(d.dtag1, 0xFF, sizeof(unsigned long long) * 2 * (size_t)m.n1));
    d.n1 = m.n1;
    d.n2 = m.n2;
    d.max_l1_local = m.max_l1_local;
    d.max_l1_own = m.max_l1_own;
    d.max_l2_own = m.max_l2_own;
    d.lmax1 = m.lmax1;
    return PIC_OK;
}

// the general kernels' hierarchy on the device: level 0 points at the fine
// matrix and at the solver's own vectors (z, the preconditioner's scratch and
// its two step buffers), levels 1.. at their own tables and vectors (in the
// solver's precision, zeroed), the level records and the coarsest inverses
static int upload_gmg(pic_ctx c, const GmgHost &h)
{
    const bool f64 = fp64(c);
    const size_t elem = f64 ? sizeof(double) : sizeof(float);
    const int L = (int)h.lev.size() - 1;
    std::vector<GmgLevel> rec((size_t)L + 1);
    for (auto &r : rec)
        r = GmgLevel{};
    auto coefs = [&](GmgLevel &r, double lmax) {
        double c1[GMG_MAX_DEG], c2[GMG_MAX_DEG], it;
        cheb_coefficients(lmax / c->p.pcg_cheb_ratio, lmax, GMG_MAX_DEG, c1, c2, &it);
        for (int j = 0; j < GMG_MAX_DEG; ++j) {
            r.c1[j] = c1[j];
            r.c2[j] = c2[j];
            r.c1f[j] = (float)c1[j];
            r.c2f[j] = (float)c2[j];
        }
        r.inv_theta = it;
        r.inv_thetaf = (float)it;
    };
    int rc = 0;
    {
        GmgLevel &f = rec[0];
        f.n_slices = c->n_slices;
        f.sptr = c->slice_ptr;
        f.col = c->col;
        f.val32 = c->val32;
        f.val64 = c->val64;
        f.dinv32 = c->dinv32;
        f.dinv64 = c->dinv64;
        int *gsl = nullptr;
        if ((rc = upload_vec(c, &gsl, c->rep_slice)))
            return rc;
        f.gsl = gsl;
        f.x = f64 ? (void *)c->z : (void *)c->z32;
        f.rc = f64 ? (void *)c->ap : (void *)c->ap32;
        f.d[0] = f64 ? (void *)c->d0 : (void *)c->d32_0;
        f.d[1] = f64 ? (void *)c->d1 : (void *)c->d32_1;
        coefs(f, c->cheb_b);
    }
    for (int l = 1; l <= L; ++l) {
        const GmgLevelHost &H = h.lev[l];
        GmgLevel &r = rec[l];
        r.n_slices = H.n_slices;
        int *sptr = nullptr, *col = nullptr, *gsl = nullptr, *agg = nullptr, *mptr = nullptr,
            *midx = nullptr;
        if ((rc = upload_vec(c, &gsl, H.gsl)) || (rc = upload_vec(c, &agg, H.agg)) ||
            (rc = upload_vec(c, &mptr, H.mptr)) || (rc = upload_vec(c, &midx, H.midx)))
            return rc;
        r.gsl = gsl;
        r.agg = agg;
        r.mptr = mptr;
        r.midx = midx;
        if (l < L) {
            if ((rc = upload_vec(c, &sptr, H.sptr)) || (rc = upload_vec(c, &col, H.col)))
                return rc;
            r.sptr = sptr;
            r.col = col;
            if (f64) {
                double *v = nullptr, *d = nullptr;
                if ((rc = upload_vec(c, &v, H.val)) || (rc = upload_vec(c, &d, H.dinv)))
                    return rc;
                r.val64 = v;
                r.dinv64 = d;
            } else {
                float *v = nullptr, *d = nullptr;
                if ((rc = upload_vec(c, &v, H.val)) || (rc = upload_vec(c, &d, H.dinv)))
                    return rc;
                r.val32 = v;
                r.dinv32 = d;
            }
            coefs(r, H.lmax);
        }
        const size_t rows = 32 * (size_t)H.n_slices;
        void **vec[4] = {&r.x, &r.rc, &r.d[0], &r.d[1]};
        for (void **v : vec) {
            unsigned char *q = nullptr;
            CK(dalloc(c, &q, rows * elem));
            CK(cudaMemset(q, 0, rows * elem));
            *v = q;
        }
    }
    GmgLevel *dl = nullptr;
    CK(dalloc(c, &dl, rec.size()));
    CK(cudaMemcpy(dl, rec.data(), sizeof(GmgLevel) * rec.size(), cudaMemcpyHostToDevice));
    float *inv = nullptr;
    long long *ioff = nullptr;
    int *cn = nullptr;
    if ((rc = upload_vec(c, &inv, h.inv)) || (rc = upload_vec(c, &ioff, h.ioff)) ||
        (rc = upload_vec(c, &cn, h.cn)))
        return rc;
    c->gmg.levels = dl;
    c->gmg.inv = inv;
    c->gmg.ioff = ioff;
    c->gmg.cn = cn;
    c->gmg.nlev = L;
    c->gmg.coarse_max = 0;
    for (int v : h.cn)
        c->gmg.coarse_max = std::max(c->gmg.coarse_max, v);
    return PIC_OK;
}

// scratch of the binary collisions: per-cell counts, offsets and fill
// counters, the SPs grouped by cell and their order keys
static int alloc_collision_scratch(pic_ctx c)
{
    const size_t T = (size_t)c->T, cap = (size_t)c->p.capacity;
    CK(dalloc(c, &c->ccnt, T));
    CK(dalloc(c, &c->coff, T + 1));
    CK(dalloc(c, &c->cfill, T));
    CK(dalloc(c, &c->cperm, cap));
    CK(dalloc(c, &c->ckey, cap));
    CK(dalloc(c, &c->cscan, 2 * ((T + 1023) / 1024) + 2));
    return PIC_OK;
}

template <typename R> static CollArgs<R> coll_args(pic_ctx c)
{
    CollArgs<R> g;
    g.P = parts<R>(c, c->a);
    g.n = &c->st->cnt[c->a];
    g.step = &c->st->hdr.step;
    g.T = c->T;
    g.det = c->det;
    g.tet_rep = c->tet_rep;
    g.rep_tet_off = c->rep_tet_off_d;
    g.cnt = c->ccnt;
    g.off = c->coff;
    g.fill = c->cfill;
    g.perm = c->cperm;
    g.key = c->ckey;
    g.scan = c->cscan;
    g.seed = c->p.seed;
    g.w_sp = c->p.w_sp;
    g.coulomb_log = c->p.coulomb_log;
    g.dt = c->p.dt;
    g.q = c->p.q;
    g.m = c->p.q / c->p.q_over_m;
    g.eps0 = c->p.eps0;
    g.grid = c->pgrid;
    return g;
}

// Loads R meshes (replicas) given as one set of arrays with global indices;
// replica r owns nodes [rno[r], rno[r+1]) and tetrahedra [rto[r], rto[r+1]),
// its faces are contiguous, E0r[r] is its applied field.  A single mesh is
// the case R = 1.
static int load_mesh(pic_ctx c, int32_t R, const int32_t *rno, const int32_t *rto,
                     const double *E0r, int32_t N, const double *xyz, int32_t T,
                     const int32_t *tet, const int32_t *nbr, const int32_t *pnbr,
                     const uint8_t *dir, int32_t F, const int32_t *face_nodes,
                     const int32_t *face_tet, const double *wf)
{
    CK(cudaSetDevice(c->dev));
    if (N < 4 || T < 1 || F < 0 || !xyz || !tet || !nbr || !dir ||
        (F > 0 && (!face_nodes || !face_tet || !wf)))
        return fail(c, PIC_ERR_ARG, "mesh_load: bad sizes or null arrays");
    if ((long long)F * 3 >= (1LL << 24) || T >= (1 << 27))
        return fail(c, PIC_ERR_ARG, "mesh_load: mesh too large for the id / neighbour packing");
    CK(cudaStreamSynchronize(c->s));
    free_mesh(c);

    // ---- validation --------------------------------------------------------
    for (long long i = 0; i < 3LL * N; ++i)
        if (!std::isfinite(xyz[i]))
            return fail(c, PIC_ERR_ARG, "mesh_load: non-finite node coordinate");
    for (long long t = 0; t < T; ++t)
        for (int k = 0; k < 4; ++k) {
            int v = tet[4 * t + k], b = nbr[4 * t + k];
            if (v < 0 || v >= N)
                return fail(c, PIC_ERR_MESH, "mesh_load: tet %lld node out of range", t);
            if (b >= T || b < PIC_BND_SIDE)
                return fail(c, PIC_ERR_MESH, "mesh_load: tet %lld bad neighbour %d", t, b);
            if (b >= 0) {
                int back = 0;
                for (int m = 0; m < 4; ++m)
                    back += nbr[4LL * b + m] == t;
                if (back != 1)
                    return fail(c, PIC_ERR_MESH, "mesh_load: neighbours of %lld not mutual", t);
            }
            if (b == PIC_BND_SIDE && (!pnbr || pnbr[4 * t + k] < 0 || pnbr[4 * t + k] >= T))
                return fail(c, PIC_ERR_MESH, "mesh_load: side face of %lld has no partner", t);
        }
    for (long long f = 0; f < F; ++f) {
        if (face_tet[f] < 0 || face_tet[f] >= T)
            return fail(c, PIC_ERR_MESH, "mesh_load: face %lld bad tetrahedron", f);
        if (!(wf[f] > 0) || !std::isfinite(wf[f]))
            return fail(c, PIC_ERR_ARG, "mesh_load: face %lld bad work function", f);
        for (int k = 0; k < 3; ++k)
            if (face_nodes[3 * f + k] < 0 || face_nodes[3 * f + k] >= N)
                return fail(c, PIC_ERR_MESH, "mesh_load: face %lld node out of range", f);
    }
    // orientation (sign only; the exact geometry is computed on the device)
    for (long long t = 0; t < T; ++t) {
        const double *X[4];
        for (int k = 0; k < 4; ++k)
            X[k] = xyz + 3LL * tet[4 * t + k];
        double a[3], b[3], d[3];
        for (int i = 0; i < 3; ++i) {
            a[i] = X[1][i] - X[0][i];
            b[i] = X[2][i] - X[0][i];
            d[i] = X[3][i] - X[0][i];
        }
        double det = a[0] * (b[1] * d[2] - b[2] * d[1]) - a[1] * (b[0] * d[2] - b[2] * d[0]) +
                     a[2] * (b[0] * d[1] - b[1] * d[0]);
        if (!(det > 0))
            return fail(c, PIC_ERR_MESH, "mesh_load: tet %lld not positively oriented", t);
    }
    // ---- replicas ------------------------------------------------------------
    if (R < 1 || !rno || !rto || !E0r || rno[0] != 0 || rto[0] != 0 || rno[R] != N || rto[R] != T)
        return fail(c, PIC_ERR_ARG, "mesh_load: bad replica offsets");
    for (int r = 0; r < R; ++r)
        if (rno[r + 1] <= rno[r] || rto[r + 1] <= rto[r] || !std::isfinite(E0r[r]))
            return fail(c, PIC_ERR_ARG, "mesh_load: replica %d empty or bad E0", r);
    std::vector<int> tet_rep((size_t)T), face_rep((size_t)F + 1, 0), rep_face_off((size_t)R + 1, 0);
    for (int r = 0; r < R; ++r)
        for (long long t = rto[r]; t < rto[r + 1]; ++t)
            tet_rep[t] = r;
    for (long long t = 0; t < T; ++t) {
        int r = tet_rep[t];
        for (int k = 0; k < 4; ++k) {
            int v = tet[4 * t + k], b = nbr[4 * t + k];
            if (v < rno[r] || v >= rno[r + 1])
                return fail(c, PIC_ERR_MESH, "mesh_load: tet %lld uses a node of another replica", t);
            if ((b >= 0 && tet_rep[b] != r) ||
                (b == PIC_BND_SIDE && tet_rep[pnbr[4 * t + k]] != r))
                return fail(c, PIC_ERR_MESH, "mesh_load: tet %lld neighbours another replica", t);
        }
    }
    for (long long f = 0; f < F; ++f) {
        int r = tet_rep[face_tet[f]];
        if (f > 0 && r < face_rep[f - 1])
            return fail(c, PIC_ERR_MESH, "mesh_load: faces are not grouped by replica");
        face_rep[f] = r;
        for (int k = 0; k < 3; ++k)
            if (face_nodes[3 * f + k] < rno[r] || face_nodes[3 * f + k] >= rno[r + 1])
                return fail(c, PIC_ERR_MESH, "mesh_load: face %lld uses a node of another replica", f);
    }
    for (int r = 0, f = 0; r <= R; ++r) {
        while (f < F && face_rep[f] < r)
            ++f;
        rep_face_off[r] = f;
    }
    // bounding box of each replica (its periodic box) and of everything
    std::vector<double> rlo(3 * (size_t)R), rhi(3 * (size_t)R), rep_L(2 * (size_t)R);
    for (int r = 0; r < R; ++r) {
        for (int i = 0; i < 3; ++i)
            rlo[3 * r + i] = rhi[3 * r + i] = xyz[3LL * rno[r] + i];
        for (long long n = rno[r]; n < rno[r + 1]; ++n)
            for (int i = 0; i < 3; ++i) {
                rlo[3 * r + i] = std::min(rlo[3 * r + i], xyz[3 * n + i]);
                rhi[3 * r + i] = std::max(rhi[3 * r + i], xyz[3 * n + i]);
            }
        rep_L[2 * r + 0] = rhi[3 * r + 0] - rlo[3 * r + 0];
        rep_L[2 * r + 1] = rhi[3 * r + 1] - rlo[3 * r + 1];
    }
    for (int i = 0; i < 3; ++i) {
        c->lo[i] = rlo[i];
        c->hi[i] = rhi[i];
    }
    for (int r = 1; r < R; ++r)
        for (int i = 0; i < 3; ++i) {
            c->lo[i] = std::min(c->lo[i], rlo[3 * r + i]);
            c->hi[i] = std::max(c->hi[i], rhi[3 * r + i]);
        }

    // ---- packed neighbour table --------------------------------------------
    auto face_vertex = [&](long long t, int k, int m) {  // m-th node of face k
        int idx = m + (m >= k ? 1 : 0);
        return tet[4 * t + idx];
    };
    std::vector<signed char> side_code(4 * (size_t)T, -1);
    for (long long t = 0; t < T; ++t)
        for (int k = 0; k < 4; ++k) {
            if (nbr[4 * t + k] != PIC_BND_SIDE)
                continue;
            int code = -1, r = tet_rep[t];
            for (int ax = 0; ax < 2 && code < 0; ++ax) {
                bool at_lo = true, at_hi = true;
                for (int m = 0; m < 3; ++m) {
                    double q = xyz[3LL * face_vertex(t, k, m) + ax];
                    at_lo = at_lo && q == rlo[3 * r + ax];
                    at_hi = at_hi && q == rhi[3 * r + ax];
                }
                if (at_lo)
                    code = 2 * ax;      // +L
                else if (at_hi)
                    code = 2 * ax + 1;  // -L
            }
            if (code < 0)
                return fail(c, PIC_ERR_MESH, "mesh_load: side face of %lld not on a box plane", t);
            side_code[4 * t + k] = (signed char)code;
        }
    std::vector<int4> nb4((size_t)T);
    for (long long t = 0; t < T; ++t) {
        int out[4];
        for (int k = 0; k < 4; ++k) {
            int b = nbr[4 * t + k];
            if (b >= 0) {
                int m = 0;
                while (nbr[4LL * b + m] != t)
                    ++m;
                out[k] = (b << 2) | m;
            } else if (b == PIC_BND_TOP) {
                out[k] = NB_TOP;
            } else if (b == PIC_BND_CATHODE) {
                out[k] = NB_CATHODE;
            } else {
                int p = pnbr[4 * t + k], sc = side_code[4 * t + k], want = sc ^ 1, m = -1;
                for (int q = 0; q < 4 && m < 0; ++q)
                    if (nbr[4LL * p + q] == PIC_BND_SIDE && pnbr[4LL * p + q] == t &&
                        side_code[4LL * p + q] == want)
                        m = q;
                if (m < 0)
                    return fail(c, PIC_ERR_MESH, "mesh_load: periodic partner of %lld does not match", t);
                out[k] = NB_SIDE - ((p << 4) | (sc << 2) | m);
            }
        }
        nb4[t] = make_int4(out[0], out[1], out[2], out[3]);
    }

    // ---- free DOFs and the stiffness pattern --------------------------------
    // each replica's rows start on a 32-row slice, so that no slice (and no
    // solver block) mixes two replicas; rows between replicas are padding
    std::vector<int> dof((size_t)N), rep_slice((size_t)R + 1, 0);
    int nf = 0, nreal = 0;
    for (int r = 0; r < R; ++r) {
        nf = (nf + 31) & ~31;
        rep_slice[r] = nf / 32;
        for (long long n = rno[r]; n < rno[r + 1]; ++n)
            dof[n] = dir[n] ? -1 : (++nreal, nf++);
    }
    nf = (nf + 31) & ~31;
    rep_slice[R] = nf / 32;
    if (nreal == 0)
        return fail(c, PIC_ERR_MESH, "mesh_load: no free nodes");
    std::vector<long long> rs((size_t)nf + 1, 0);
    for (long long t = 0; t < T; ++t)
        for (int i = 0; i < 4; ++i) {
            int di = dof[tet[4 * t + i]];
            if (di < 0)
                continue;
            for (int j = 0; j < 4; ++j)
                if (dof[tet[4 * t + j]] >= 0)
                    rs[di + 1]++;
        }
    for (int i = 0; i < nf; ++i)
        rs[i + 1] += rs[i];
    std::vector<int> raw((size_t)rs[nf]);
    {
        std::vector<long long> fill(rs.begin(), rs.end() - 1);
        for (long long t = 0; t < T; ++t)
            for (int i = 0; i < 4; ++i) {
                int di = dof[tet[4 * t + i]];
                if (di < 0)
                    continue;
                for (int j = 0; j < 4; ++j) {
                    int dj = dof[tet[4 * t + j]];
                    if (dj >= 0)
                        raw[fill[di]++] = dj;
                }
            }
    }
    std::vector<long long> rowptr((size_t)nf + 1, 0);
    std::vector<int> colv;
    colv.reserve((size_t)rs[nf] / 3);
    for (int i = 0; i < nf; ++i) {
        auto b = raw.begin() + rs[i], e = raw.begin() + rs[i + 1];
        std::sort(b, e);
        auto u = std::unique(b, e);
        colv.insert(colv.end(), b, u);
        rowptr[i + 1] = (long long)colv.size();
    }
    std::vector<int>().swap(raw);
    const long long nnz = rowptr[nf];
    auto slot_of = [&](int row, int cl) -> long long {
        auto b = colv.begin() + rowptr[row], e = colv.begin() + rowptr[row + 1];
        return (long long)(std::lower_bound(b, e, cl) - colv.begin());
    };
    // contributions of each nonzero in increasing element order
    std::vector<long long> cptr((size_t)nnz + 1, 0);
    for (long long t = 0; t < T; ++t)
        for (int i = 0; i < 4; ++i) {
            int di = dof[tet[4 * t + i]];
            if (di < 0)
                continue;
            for (int j = 0; j < 4; ++j) {
                int dj = dof[tet[4 * t + j]];
                if (dj >= 0)
                    cptr[slot_of(di, dj) + 1]++;
            }
        }
    for (long long s = 0; s < nnz; ++s)
        cptr[s + 1] += cptr[s];
    std::vector<int> contrib((size_t)cptr[nnz]);
    {
        std::vector<long long> fill(cptr.begin(), cptr.end() - 1);
        for (long long t = 0; t < T; ++t)
            for (int i = 0; i < 4; ++i) {
                int di = dof[tet[4 * t + i]];
                if (di < 0)
                    continue;
                for (int j = 0; j < 4; ++j) {
                    int dj = dof[tet[4 * t + j]];
                    if (dj >= 0)
                        contrib[fill[slot_of(di, dj)]++] = (int)((t << 4) | (i << 2) | j);
                }
            }
    }
    // sliced ELLPACK, 32 rows per slice, padding rows/entries point at their own row
    const int n_pad = (nf + 31) & ~31, n_slices = n_pad / 32;
    std::vector<int> sptr((size_t)n_slices + 1, 0);
    for (int s = 0; s < n_slices; ++s) {
        long long w = 0;
        for (int l = 0; l < 32; ++l) {
            int row = s * 32 + l;
            if (row < nf)
                w = std::max(w, rowptr[row + 1] - rowptr[row]);
        }
        if ((long long)sptr[s] + 32 * w >= (1LL << 31))
            return fail(c, PIC_ERR_ARG, "mesh_load: matrix too large");
        sptr[s + 1] = sptr[s] + (int)(32 * w);
    }
    const long long sell_len = sptr[n_slices];
    std::vector<int> scol((size_t)sell_len);
    std::vector<long long> spos((size_t)nnz);
    std::vector<int> srow((size_t)nnz), scl((size_t)nnz);
    for (int s = 0; s < n_slices; ++s) {
        int w = (sptr[s + 1] - sptr[s]) / 32;
        for (int l = 0; l < 32; ++l) {
            int row = s * 32 + l;
            long long len = row < nf ? rowptr[row + 1] - rowptr[row] : 0;
            for (int k = 0; k < w; ++k) {
                long long pos = sptr[s] + (long long)k * 32 + l;
                if (k < len) {
                    long long slot = rowptr[row] + k;
                    scol[pos] = colv[slot];
                    spos[slot] = pos;
                    srow[slot] = row;
                    scl[slot] = colv[slot];
                } else {
                    scol[pos] = row;
                }
            }
        }
    }
    // Neumann contributions per free DOF in increasing (tet, face) order
    std::vector<int> fptr((size_t)nf + 1, 0), fcon;
    {
        std::vector<std::pair<int, int>> pairs;  // (dof, tet<<2|face)
        for (long long t = 0; t < T; ++t)
            for (int k = 0; k < 4; ++k) {
                if (nbr[4 * t + k] != PIC_BND_TOP)
                    continue;
                for (int m = 0; m < 3; ++m) {
                    int d = dof[face_vertex(t, k, m)];
                    if (d >= 0)
                        pairs.push_back({d, (int)((t << 2) | k)});
                }
            }
        std::stable_sort(pairs.begin(), pairs.end(),
                         [](const std::pair<int, int> &x, const std::pair<int, int> &y) {
                             return x.first < y.first;
                         });
        fcon.resize(pairs.size());
        for (size_t i = 0; i < pairs.size(); ++i) {
            fptr[pairs[i].first + 1]++;
            fcon[i] = pairs[i].second;
        }
        for (int i = 0; i < nf; ++i)
            fptr[i + 1] += fptr[i];
    }
    // couplings of each free row with Dirichlet nodes, in increasing
    // (element, local j) order: the load of prescribed values (pic_set_dirichlet)
    std::vector<int> dptr((size_t)nf + 1, 0), dcon;
    for (long long t = 0; t < T; ++t)
        for (int i = 0; i < 4; ++i) {
            int di = dof[tet[4 * t + i]];
            if (di < 0)
                continue;
            for (int j = 0; j < 4; ++j)
                if (dir[tet[4 * t + j]])
                    dptr[di + 1]++;
        }
    for (int i = 0; i < nf; ++i)
        dptr[i + 1] += dptr[i];
    dcon.resize((size_t)dptr[nf]);
    {
        std::vector<int> fill(dptr.begin(), dptr.end() - 1);
        for (long long t = 0; t < T; ++t)
            for (int i = 0; i < 4; ++i) {
                int di = dof[tet[4 * t + i]];
                if (di < 0)
                    continue;
                for (int j = 0; j < 4; ++j)
                    if (dir[tet[4 * t + j]])
                        dcon[fill[di]++] = (int)((t << 4) | (i << 2) | j);
            }
    }
    std::vector<int> dof_node((size_t)n_pad, -1);
    for (int n = 0; n < N; ++n)
        if (dof[n] >= 0)
            dof_node[dof[n]] = n;

    // ---- device buffers ------------------------------------------------------
    c->N = N;
    c->T = T;
    c->F = F;
    c->NQ = 3 * F;
    c->n_free = nreal;
    c->n_rows = nf;
    c->n_rep = R;
    c->n_pad = n_pad;
    c->n_slices = n_slices;
    c->sell_len = sell_len;
    c->nnz = nnz;
    const bool d64 = fp64(c);
    const size_t cap = (size_t)c->p.capacity;
    const size_t rsz = d64 ? 8 : 4;
    int4 *d_nb = nullptr;
    long long *d_cptr = nullptr, *d_spos = nullptr;
    int *d_contrib = nullptr, *d_srow = nullptr, *d_scl = nullptr, *d_fptr = nullptr, *d_fcon = nullptr;
    std::vector<int4> tet4((size_t)T);
    for (long long t = 0; t < T; ++t)
        tet4[t] = make_int4(tet[4 * t], tet[4 * t + 1], tet[4 * t + 2], tet[4 * t + 3]);

    CK(dalloc(c, &c->xyz, 3 * (size_t)N));
    CK(dalloc(c, &c->tet4, (size_t)T));
    CK(dalloc(c, &c->rec64, (size_t)T));
    if (!d64)
        CK(dalloc(c, &c->rec32, (size_t)T));
    CK(dalloc(c, &c->det, (size_t)T));
    CK(dalloc(c, &c->dir, (size_t)N));
    CK(dalloc(c, &c->face_nodes, 3 * (size_t)F + 3));
    CK(dalloc(c, &c->face_tet, (size_t)F + 1));
    CK(dalloc(c, &c->wf, (size_t)F + 1));
    CK(dalloc(c, &c->fnhat, 3 * (size_t)F + 3));
    CK(dalloc(c, &c->farea, (size_t)F + 1));
    CK(dalloc(c, &c->dof_node, (size_t)n_pad));
    CK(dalloc(c, &c->slice_ptr, (size_t)n_slices + 1));
    CK(dalloc(c, &c->col, (size_t)sell_len));
    CK(dalloc(c, &c->val64, (size_t)sell_len));
    CK(dalloc(c, &c->val32, (size_t)sell_len));
    CK(dalloc(c, &c->dinv64, (size_t)n_pad));
    CK(dalloc(c, &c->dinv32, (size_t)n_pad));
    CK(dalloc(c, &c->fN, (size_t)n_pad));
    CK(dalloc(c, &c->phi, (size_t)N));
    CK(dalloc(c, &c->x, (size_t)n_pad));
    {
        void *e = nullptr;
        CK(cudaMalloc(&e, (size_t)T * (d64 ? sizeof(Vec4d) : sizeof(float4))));
        c->allocs.push_back(e);
        c->E = e;
    }
    CK(dalloc(c, &c->W, (size_t)N));
    for (int b = 0; b < 2; ++b) {
        for (int k = 0; k < 6; ++k) {
            void *q = nullptr;
            CK(cudaMalloc(&q, cap * rsz));
            c->allocs.push_back(q);
            c->pbuf[b][k] = q;
        }
        CK(dalloc(c, &c->cell[b], cap));
        CK(dalloc(c, &c->id[b], cap));
    }
    CK(dalloc(c, &c->st, 1));
    CK(dalloc(c, &c->qcount, (size_t)c->NQ + 1));
    CK(dalloc(c, &c->qoff, (size_t)c->NQ + 1));
    CK(dalloc(c, &c->f, (size_t)n_pad));
    CK(dalloc(c, &c->r, (size_t)n_pad));
    CK(dalloc(c, &c->z, (size_t)n_pad));
    CK(dalloc(c, &c->p0, (size_t)n_pad));
    CK(dalloc(c, &c->p1, (size_t)n_pad));
    CK(dalloc(c, &c->ap, (size_t)n_pad));
    CK(dalloc(c, &c->r32, (size_t)n_pad));
    CK(dalloc(c, &c->z32, (size_t)n_pad));
    CK(dalloc(c, &c->p32_0, (size_t)n_pad));
    CK(dalloc(c, &c->p32_1, (size_t)n_pad));
    CK(dalloc(c, &c->ap32, (size_t)n_pad));
    CK(dalloc(c, &c->dx32, (size_t)n_pad));
    CK(dalloc(c, &c->d0, (size_t)n_pad));
    CK(dalloc(c, &c->d1, (size_t)n_pad));
    CK(dalloc(c, &c->d32_0, (size_t)n_pad));
    CK(dalloc(c, &c->d32_1, (size_t)n_pad));
    CK(dalloc(c, &c->dtag, 2 * (size_t)n_pad));
    CK(dalloc(c, &c->pcg_epoch, 1));
    PcgHalo halo;
    c->lcol = c->halo_ptr = c->halo_idx = nullptr;
    CK(pcg_plan(sptr.data(), scol.data(), n_slices, c->num_sms, c->p.precision, c->p.pcg_variant,
                R, rep_slice.data(), nullptr, c->pcg_bps, &c->plan, &halo));
    c->rep_slice = rep_slice;
    c->rep_sell.assign((size_t)R, 0);
    c->rep_free.assign((size_t)R, 0);
    for (int r = 0; r < R; ++r) {
        c->rep_sell[r] = (long long)sptr[rep_slice[r + 1]] - sptr[rep_slice[r]];
        for (long long n = rno[r]; n < rno[r + 1]; ++n)
            c->rep_free[r] += dir[n] ? 0 : 1;
    }
    CK(dalloc(c, &c->rep_slice_d, rep_slice.size()));
    CK(cudaMemcpyAsync(c->rep_slice_d, rep_slice.data(), sizeof(int) * rep_slice.size(),
                       cudaMemcpyHostToDevice, c->s));
    // a batch solve can be re-planned with more blocks (pic_set_tuning)
    const int max_grid = c->plan.n_groups > 0
                             ? std::max(c->plan.grid, pcg_max_group_blocks(c->p.precision, c->num_sms))
                             : c->plan.grid;
    CK(dalloc(c, &c->partials, (size_t)2 * max_grid * 4));
    CK(dalloc(c, &c->part8, (size_t)2 * max_grid * 8));
    c->grp = c->blk_grp = nullptr;
    c->grp_bar = nullptr;
    if (c->plan.n_groups > 0) {
        CK(dalloc(c, &c->grp, halo.grp.size()));
        CK(dalloc(c, &c->blk_grp, (size_t)max_grid));
        CK(dalloc(c, &c->grp_bar, (size_t)c->plan.n_groups));
        CK(dalloc(c, &c->grp_iters, (size_t)c->plan.n_groups));
        CK(cudaMemsetAsync(c->grp_iters, 0, sizeof(int) * c->plan.n_groups, c->s));
        c->grp_h = halo.grp;
        c->blk_grp_h = halo.blk_grp;
        CK(cudaMemcpyAsync(c->grp, halo.grp.data(), sizeof(int) * halo.grp.size(),
                           cudaMemcpyHostToDevice, c->s));
        CK(cudaMemcpyAsync(c->blk_grp, halo.blk_grp.data(), sizeof(int) * halo.blk_grp.size(),
                           cudaMemcpyHostToDevice, c->s));
    }
    CK(dalloc(c, &c->tet_rep, (size_t)T));
    CK(dalloc(c, &c->face_rep, (size_t)F + 1));
    CK(dalloc(c, &c->rep_face_off, (size_t)R + 1));
    CK(dalloc(c, &c->rep_L, 2 * (size_t)R));
    CK(dalloc(c, &c->E0_rep, (size_t)R));
    CK(dalloc(c, &c->rep_tet_off_d, (size_t)R + 1));
    CK(cudaMemcpyAsync(c->rep_tet_off_d, rto, sizeof(int) * (R + 1), cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync(c->tet_rep, tet_rep.data(), sizeof(int) * T, cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync(c->face_rep, face_rep.data(), sizeof(int) * (F + 1), cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync(c->rep_face_off, rep_face_off.data(), sizeof(int) * (R + 1),
                       cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync(c->rep_L, rep_L.data(), sizeof(double) * 2 * R, cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync(c->E0_rep, E0r, sizeof(double) * R, cudaMemcpyHostToDevice, c->s));
    CK(cudaStreamSynchronize(c->s));
    if (c->plan.resident) {
        CK(dalloc(c, &c->lcol, halo.lcol.size()));
        CK(dalloc(c, &c->halo_ptr, halo.halo_ptr.size()));
        CK(dalloc(c, &c->halo_idx, halo.halo_idx.size() + 1));
        CK(cudaMemcpyAsync(c->lcol, halo.lcol.data(), sizeof(int) * halo.lcol.size(),
                           cudaMemcpyHostToDevice, c->s));
        CK(cudaMemcpyAsync(c->halo_ptr, halo.halo_ptr.data(), sizeof(int) * halo.halo_ptr.size(),
                           cudaMemcpyHostToDevice, c->s));
        if (!halo.halo_idx.empty())
            CK(cudaMemcpyAsync(c->halo_idx, halo.halo_idx.data(),
                               sizeof(int) * halo.halo_idx.size(), cudaMemcpyHostToDevice, c->s));
        CK(cudaStreamSynchronize(c->s));
    }
    CK(dalloc(c, &c->sstats, 1));
    CK(dalloc(c, &c->dptr, dptr.size()));
    CK(dalloc(c, &c->dcon, dcon.size() + 1));
    CK(dalloc(c, &c->gD, (size_t)N));
    CK(dalloc(c, &c->fD, (size_t)n_pad));
    CK(cudaMemcpyAsync(c->dptr, dptr.data(), sizeof(int) * dptr.size(), cudaMemcpyHostToDevice,
                       c->s));
    if (!dcon.empty())
        CK(cudaMemcpyAsync(c->dcon, dcon.data(), sizeof(int) * dcon.size(), cudaMemcpyHostToDevice,
                           c->s));
    CK(cudaMemsetAsync(c->gD, 0, sizeof(double) * N, c->s));
    CK(cudaMemsetAsync(c->fD, 0, sizeof(double) * n_pad, c->s));
    CK(cudaStreamSynchronize(c->s));
    c->dir_h.assign(dir, dir + N);
    CK(dalloc(c, &c->scnt, (size_t)T));
    CK(dalloc(c, &c->soff, (size_t)T + 1));
    CK(dalloc(c, &c->srank, cap));
    CK(dalloc(c, &c->sscan, 2 * (((size_t)T + 1023) / 1024) + 2));
    c->ccnt = c->coff = c->cfill = c->cperm = c->cscan = nullptr;
    c->ckey = nullptr;
    if (c->p.collisions) {
        int rc = alloc_collision_scratch(c);
        if (rc)
            return rc;
    }
    CK(dalloc(c, &c->slot, 1));
    CK(cudaMemsetAsync(c->slot, 0, sizeof(pic_step_stats), c->s));

    auto up = [&](void *dst, const void *src, size_t bytes) {
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->s);
    };
    CK(up(c->xyz, xyz, sizeof(double) * 3 * N));
    CK(up(c->tet4, tet4.data(), sizeof(int4) * T));
    CK(up(c->dir, dir, (size_t)N));
    if (F) {
        CK(up(c->face_nodes, face_nodes, sizeof(int) * 3 * F));
        CK(up(c->face_tet, face_tet, sizeof(int) * F));
        CK(up(c->wf, wf, sizeof(double) * F));
    }
    CK(up(c->dof_node, dof_node.data(), sizeof(int) * n_pad));
    CK(up(c->slice_ptr, sptr.data(), sizeof(int) * (n_slices + 1)));
    CK(up(c->col, scol.data(), sizeof(int) * sell_len));
    CK(cudaMemsetAsync(c->val64, 0, sizeof(double) * sell_len, c->s));
    CK(cudaMemsetAsync(c->val32, 0, sizeof(float) * sell_len, c->s));
    CK(cudaMemsetAsync(c->dinv64, 0, sizeof(double) * n_pad, c->s));
    CK(cudaMemsetAsync(c->dinv32, 0, sizeof(float) * n_pad, c->s));
    CK(cudaMemsetAsync(c->fN, 0, sizeof(double) * n_pad, c->s));
    CK(cudaMemsetAsync(c->phi, 0, sizeof(double) * N, c->s));
    CK(cudaMemsetAsync(c->x, 0, sizeof(double) * n_pad, c->s));
    CK(cudaMemsetAsync(c->W, 0, sizeof(unsigned long long) * N, c->s));
    CK(cudaMemsetAsync(c->st, 0, sizeof(DevState), c->s));
    for (double *v : {c->f, c->r, c->z, c->p0, c->p1, c->ap})
        CK(cudaMemsetAsync(v, 0, sizeof(double) * n_pad, c->s));
    for (double *v : {c->d0, c->d1})
        CK(cudaMemsetAsync(v, 0, sizeof(double) * n_pad, c->s));
    for (float *v : {c->r32, c->z32, c->p32_0, c->p32_1, c->ap32, c->dx32, c->d32_0, c->d32_1})
        CK(cudaMemsetAsync(v, 0, sizeof(float) * n_pad, c->s));
    // all-ones tags: no epoch (< 255) produces them
    CK(cudaMemsetAsync(c->dtag, 0xFF, sizeof(unsigned long long) * 2 * n_pad, c->s));
    CK(cudaMemsetAsync(c->pcg_epoch, 0, sizeof(unsigned), c->s));

    // temporaries of the assembly
    std::vector<void *> tmp;
    auto tmalloc = [&](void **p, size_t bytes) {
        cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
        if (e == cudaSuccess)
            tmp.push_back(*p);
        return e;
    };
    auto free_tmp = [&]() {
        cudaStreamSynchronize(c->s);
        for (void *q : tmp)
            cudaFree(q);
        tmp.clear();
    };
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = tmalloc((void **)&d_nb, sizeof(int4) * T);
    if (e == cudaSuccess) e = tmalloc((void **)&d_cptr, sizeof(long long) * (nnz + 1));
    if (e == cudaSuccess) e = tmalloc((void **)&d_contrib, sizeof(int) * contrib.size());
    if (e == cudaSuccess) e = tmalloc((void **)&d_spos, sizeof(long long) * nnz);
    if (e == cudaSuccess) e = tmalloc((void **)&d_srow, sizeof(int) * nnz);
    if (e == cudaSuccess) e = tmalloc((void **)&d_scl, sizeof(int) * nnz);
    // the Neumann tables stay (pic_set_applied_field rebuilds the load)
    if (e == cudaSuccess) e = dalloc(c, &d_fptr, (size_t)nf + 1);
    if (e == cudaSuccess) e = dalloc(c, &d_fcon, fcon.size() + 1);
    c->nfptr = d_fptr;
    c->nfcon = d_fcon;
    if (e == cudaSuccess) e = up(d_nb, nb4.data(), sizeof(int4) * T);
    if (e == cudaSuccess) e = up(d_cptr, cptr.data(), sizeof(long long) * (nnz + 1));
    if (e == cudaSuccess) e = up(d_contrib, contrib.data(), sizeof(int) * contrib.size());
    if (e == cudaSuccess) e = up(d_spos, spos.data(), sizeof(long long) * nnz);
    if (e == cudaSuccess) e = up(d_srow, srow.data(), sizeof(int) * nnz);
    if (e == cudaSuccess) e = up(d_scl, scl.data(), sizeof(int) * nnz);
    if (e == cudaSuccess) e = up(d_fptr, fptr.data(), sizeof(int) * (nf + 1));
    if (e == cudaSuccess && !fcon.empty()) e = up(d_fcon, fcon.data(), sizeof(int) * fcon.size());
    if (e == cudaSuccess) {
        e = launch_geometry(c->s, T, c->xyz, c->tet4, d_nb, c->rec64, c->rec32, c->det);
        ++c->launches;
    }
    if (e == cudaSuccess) {
        e = launch_matrix_values(c->s, nnz, d_cptr, d_contrib, c->rec64, c->det, d_spos, d_srow,
                                 d_scl, c->val64, c->val32, c->dinv64, c->dinv32);
        ++c->launches;
    }
    if (e == cudaSuccess) {
        e = launch_neumann(c->s, nf, d_fptr, d_fcon, c->tet4, c->xyz, c->tet_rep, c->E0_rep, c->fN);
        ++c->launches;
    }
    if (e == cudaSuccess) {
        e = launch_face_geometry(c->s, F, c->face_nodes, c->xyz, c->fnhat, c->farea);
        ++c->launches;
    }
    free_tmp();
    if (e != cudaSuccess)
        return fail(c, PIC_ERR_CUDA, "mesh_load: %s", cudaGetErrorString(e));
    CK(cudaStreamSynchronize(c->s));
    {
        // Gershgorin bound of the Jacobi-scaled matrix: max_i sum_j |M_ij| / M_ii
        std::vector<double> hv((size_t)sell_len), hd((size_t)n_pad);
        CK(cudaMemcpy(hv.data(), c->val64, sizeof(double) * sell_len, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(hd.data(), c->dinv64, sizeof(double) * n_pad, cudaMemcpyDeviceToHost));
        double bmax = 0.0;
        for (int sl = 0; sl < n_slices; ++sl) {
            int w = (sptr[sl + 1] - sptr[sl]) / 32;
            for (int l = 0; l < 32; ++l) {
                double sum = 0.0;
                for (int k = 0; k < w; ++k)
                    sum += std::fabs(hv[(size_t)sptr[sl] + (size_t)k * 32 + l]);
                bmax = std::max(bmax, sum * hd[(size_t)sl * 32 + l]);
            }
        }
        c->cheb_b = bmax > 0.0 ? bmax : 2.0;
        // coarse matrix of the resident solver's blocks (two-level
        // preconditioner): A0 = R0 M R0^T with R0 summing each block's rows,
        // inverted here in FP64 (Cholesky)
        c->coarse_inv = nullptr;
        c->coarse_r = nullptr;
        if (c->plan.resident) {
            const int G = c->plan.grid;
            std::vector<int> blk_of_slice((size_t)n_slices);
            for (long long b = 0; b < G; ++b)
                for (int sl = (int)((b * n_slices) / G); sl < (int)(((b + 1) * n_slices) / G); ++sl)
                    blk_of_slice[sl] = (int)b;
            std::vector<double> A0((size_t)G * G, 0.0);
            for (int sl = 0; sl < n_slices; ++sl) {
                const int w = (sptr[sl + 1] - sptr[sl]) / 32, bi = blk_of_slice[sl];
                for (int l = 0; l < 32; ++l)
                    for (int k = 0; k < w; ++k) {
                        const size_t e = (size_t)sptr[sl] + (size_t)k * 32 + l;
                        const double v = hv[e];
                        if (v != 0.0)
                            A0[(size_t)bi * G + blk_of_slice[scol[e] / 32]] += v;
                    }
            }
            std::vector<float> inv((size_t)G * G);
            if (spd_inverse(A0, G, inv.data())) {
                float *ci = nullptr;
                CK(dalloc(c, &ci, inv.size()));
                CK(cudaMemcpy(ci, inv.data(), sizeof(float) * inv.size(), cudaMemcpyHostToDevice));
                c->coarse_inv = ci;
                CK(dalloc(c, &c->coarse_r, (size_t)2 * G));   // sums of r, of A p
            }
        }
        // multigrid hierarchy of the resident solver (pcg_cheb_local = 4)
        c->mg = {};
        if (c->plan.resident) {
            MgHost mh;
            bool ok = mg_build(sptr.data(), scol.data(), hv.data(), hd.data(), n_slices,
                               c->plan.grid, MG_PASSES0, MG_PASSES1, MG_MAX_COARSE, &mh);
            if (ok)
                CK(pcg_plan_mg(&c->plan, c->p.precision, c->p.pcg_variant,
                               mg_smem_bytes(mh, fp64(c) ? 8 : 4), &ok));
            if (ok) {
                int rc = upload_mg(c, mh);
                if (rc)
                    return rc;
                // the V-cycle replaces the two-level Chebyshev preconditioner
                // as the default of the polynomial-preconditioned solvers
                if (c->cheb_local == 3)
                    c->cheb_local = 4;
            }
        }
        // general kernels (batches, large systems): aggregates of
        // PCG_AGG_SLICES slices within each group, A0 of each group inverted
        c->agg_inv = nullptr;
        if (!c->plan.resident) {
            const int NG = c->plan.n_groups > 0 ? c->plan.n_groups : 1;
            auto g_s0 = [&](int g) { return c->plan.n_groups > 0 ? rep_slice[g] : 0; };
            auto g_s1 = [&](int g) { return c->plan.n_groups > 0 ? rep_slice[g + 1] : n_slices; };
            std::vector<int> agg_off((size_t)NG + 1, 0);
            std::vector<long long> inv_off((size_t)NG + 1, 0);
            for (int g = 0; g < NG; ++g) {
                const int na = (g_s1(g) - g_s0(g) + PCG_AGG_SLICES - 1) / PCG_AGG_SLICES;
                agg_off[g + 1] = agg_off[g] + na;
                inv_off[g + 1] = inv_off[g] + (long long)na * na;
            }
            std::vector<float> inv((size_t)inv_off[NG]);
            bool ok = true;
            for (int g = 0; g < NG && ok; ++g) {
                const int s0 = g_s0(g), na = agg_off[g + 1] - agg_off[g];
                std::vector<double> A0((size_t)na * na, 0.0);
                for (int sl = s0; sl < g_s1(g); ++sl) {
                    const int w = (sptr[sl + 1] - sptr[sl]) / 32, ai = (sl - s0) / PCG_AGG_SLICES;
                    for (int l = 0; l < 32; ++l)
                        for (int k = 0; k < w; ++k) {
                            const size_t e = (size_t)sptr[sl] + (size_t)k * 32 + l;
                            if (hv[e] != 0.0)
                                A0[(size_t)ai * na + (scol[e] / 32 - s0) / PCG_AGG_SLICES] += hv[e];
                        }
                }
                ok = spd_inverse(A0, na, inv.data() + inv_off[g]);
            }
            if (ok) {
                int *ao = nullptr;
                long long *io = nullptr;
                float *ai = nullptr;
                CK(dalloc(c, &ao, agg_off.size()));
                CK(dalloc(c, &io, inv_off.size()));
                CK(dalloc(c, &ai, inv.size()));
                CK(dalloc(c, &c->slice_r, (size_t)n_slices));
                CK(dalloc(c, &c->agg_r, (size_t)agg_off[NG]));
                CK(dalloc(c, &c->agg_z, (size_t)agg_off[NG]));
                CK(cudaMemcpy(ao, agg_off.data(), sizeof(int) * agg_off.size(), cudaMemcpyHostToDevice));
                CK(cudaMemcpy(io, inv_off.data(), sizeof(long long) * inv_off.size(),
                              cudaMemcpyHostToDevice));
                CK(cudaMemcpy(ai, inv.data(), sizeof(float) * inv.size(), cudaMemcpyHostToDevice));
                c->agg_off = ao;
                c->inv_off = io;
                c->agg_inv = ai;
            }
        }
        // multigrid hierarchy of the general kernels (pcg_cheb_local = 4)
        c->gmg = {};
        if (!c->plan.resident) {
            GmgHost gh;
            if (gmg_build(sptr.data(), scol.data(), hv.data(), hd.data(), n_slices, R,
                          rep_slice.data(), MG_PASSES0, MG_PASSES1, GMG_MAX_COARSE,
                          GMG_MAX_LEVELS, &gh)) {
                int rc = upload_gmg(c, gh);
                if (rc)
                    return rc;
                if (c->cheb_local == 3)
                    c->cheb_local = 4;
            }
        }
    }
    c->loaded = true;
    c->a = 0;
    c->step = 0;
    int rc = refresh_field(c);
    if (rc)
        return rc;
    CK(cudaStreamSynchronize(c->s));
    return PIC_OK;
}

extern "C" int mesh_load(pic_ctx c, int32_t N, const double *xyz, int32_t T, const int32_t *tet,
                         const int32_t *nbr, const int32_t *pnbr, const uint8_t *dir,
                         int32_t F, const int32_t *face_nodes, const int32_t *face_tet,
                         const double *wf)
{
    if (!c)
        return fail(nullptr, PIC_ERR_ARG, "null context");
    int32_t rno[2] = {0, N}, rto[2] = {0, T};
    double e0 = c->p.E0;
    return load_mesh(c, 1, rno, rto, &e0, N, xyz, T, tet, nbr, pnbr, dir, F, face_nodes,
                     face_tet, wf);
}

extern "C" int mesh_load_batch(pic_ctx c, int32_t n_rep, const int32_t *rep_node_off,
                               const int32_t *rep_tet_off, const double *E0_rep, int32_t N,
                               const double *xyz, int32_t T, const int32_t *tet,
                               const int32_t *nbr, const int32_t *pnbr, const uint8_t *dir,
                               int32_t F, const int32_t *face_nodes, const int32_t *face_tet,
                               const double *wf)
{
    if (!c)
        return fail(nullptr, PIC_ERR_ARG, "null context");
    if (n_rep < 1 || n_rep > (1 << 16))
        return fail(c, PIC_ERR_ARG, "mesh_load_batch: bad replica count");
    return load_mesh(c, n_rep, rep_node_off, rep_tet_off, E0_rep, N, xyz, T, tet, nbr, pnbr, dir,
                     F, face_nodes, face_tet, wf);
}

// Re-plan the batch solve's block groups (same kernels, new group tables);
// work = per-replica weights or null (slices).  The tables live in device
// memory, so captured graphs stay valid unless the grid size changes.
static int replan_batch(pic_ctx c, const double *work)
{
    PcgLaunch plan;
    PcgHalo halo;
    CK(pcg_plan(nullptr, nullptr, c->n_slices, c->num_sms, c->p.precision, c->p.pcg_variant,
                c->n_rep, c->rep_slice.data(), work, c->pcg_bps, &plan, &halo));
    if (halo.grp == c->grp_h && halo.blk_grp == c->blk_grp_h)
        return PIC_OK;
    c->grp_h = halo.grp;
    c->blk_grp_h = halo.blk_grp;
    CK(cudaMemcpyAsync(c->grp, c->grp_h.data(), sizeof(int) * c->grp_h.size(),
                       cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync(c->blk_grp, c->blk_grp_h.data(), sizeof(int) * c->blk_grp_h.size(),
                       cudaMemcpyHostToDevice, c->s));
    if (plan.grid != c->plan.grid)
        free_graphs(c);
    c->plan = plan;
    return PIC_OK;
}

// Balance the batch solve on the iteration counts of the last solve of each
// replica (stable from step to step: every solve is warm-started).
static int balance_batch(pic_ctx c)
{
    if (c->plan.n_groups <= 0 || !c->pcg_balance)
        return PIC_OK;
    const int G = c->plan.n_groups;
    std::vector<int> it((size_t)G);
    CK(cudaMemcpyAsync(it.data(), c->grp_iters, sizeof(int) * G, cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    std::vector<double> w((size_t)G);
    bool any = false;
    for (int g = 0; g < G; ++g) {
        any = any || it[g] > 0;
        w[g] = (double)(c->rep_slice[g + 1] - c->rep_slice[g]) * (double)std::max(it[g], 1);
    }
    return replan_batch(c, any ? w.data() : nullptr);
}

extern "C" int pic_replica_info(pic_ctx c, int32_t *pcg_iters, int64_t *stored, int32_t *rows,
                                int32_t *free_dofs)
{
    REQUIRE_MESH();
    const int R = c->n_rep;
    if (pcg_iters) {
        if (c->plan.n_groups > 0) {
            CK(cudaMemcpyAsync(pcg_iters, c->grp_iters, sizeof(int) * R, cudaMemcpyDeviceToHost,
                               c->s));
            CK(cudaStreamSynchronize(c->s));
        } else {
            for (int r = 0; r < R; ++r)
                pcg_iters[r] = 0;
        }
    }
    for (int r = 0; r < R; ++r) {
        if (stored)
            stored[r] = c->rep_sell[r];
        if (rows)
            rows[r] = 32 * (c->rep_slice[r + 1] - c->rep_slice[r]);
        if (free_dofs)
            free_dofs[r] = c->rep_free[r];
    }
    return PIC_OK;
}

extern "C" int pic_get_tuning(pic_ctx c, pic_tuning *t)
{
    if (!c || !t)
        return fail(c, PIC_ERR_ARG, "null argument");
    t->particle_blocks_per_sm = c->pgrid / c->num_sms;
    t->walk_form = c->walk_form;
    t->pcg_blocks_per_sm = c->pcg_bps;
    t->pcg_cheb_degree = c->p.pcg_cheb_degree;
    t->pcg_balance = c->pcg_balance;
    t->pcg_cheb_local = c->cheb_local;
    t->sort_cells = c->sort_cells;
    t->pcg_halo_sync = c->halo_sync;
    t->wait_limit = c->wait_limit;
    t->pcg_mg_degree0 = mg_degree(c, 0);
    t->pcg_mg_degree1 = mg_degree(c, 1);
    return PIC_OK;
}

extern "C" int pic_set_tuning(pic_ctx c, const pic_tuning *t)
{
    if (!c || !t)
        return fail(c, PIC_ERR_ARG, "null argument");
    if (t->particle_blocks_per_sm < 1 || t->particle_blocks_per_sm > 64 || t->walk_form < 0 ||
        t->walk_form > 3 || t->pcg_blocks_per_sm < 0 || t->pcg_blocks_per_sm > 64 ||
        t->pcg_cheb_degree < 0 || t->pcg_cheb_degree > 32 || t->pcg_balance < 0 ||
        t->pcg_balance > 1 || t->pcg_cheb_local < 0 || t->pcg_cheb_local > 4 ||
        (t->pcg_cheb_local == 4 && c->mg.n1 == 0 && c->gmg.nlev == 0) ||
        t->sort_cells < 0 || t->sort_cells > 1 || t->pcg_halo_sync < 0 || t->pcg_halo_sync > 1 ||
        t->wait_limit < 0 || t->wait_limit > (1 << 30) || t->pcg_mg_degree0 < 0 ||
        t->pcg_mg_degree0 > 8 || t->pcg_mg_degree1 < 0 || t->pcg_mg_degree1 > 8 ||
        (t->pcg_cheb_degree >= 2 && !(c->p.pcg_cheb_ratio > 1.0)))
        return fail(c, PIC_ERR_ARG, "pic_set_tuning: value out of range");
    CK(cudaSetDevice(c->dev));
    CK(cudaStreamSynchronize(c->s));
    free_graphs(c);
    c->pgrid = t->particle_blocks_per_sm * c->num_sms;
    c->walk_form = t->walk_form;
    c->pcg_bps = t->pcg_blocks_per_sm;
    c->pcg_balance = t->pcg_balance;
    c->cheb_local = t->pcg_cheb_local;
    c->sort_cells = t->sort_cells;
    c->halo_sync = t->pcg_halo_sync;
    c->wait_limit = t->wait_limit;
    c->mg_deg0 = t->pcg_mg_degree0;
    c->mg_deg1 = t->pcg_mg_degree1;
    c->p.pcg_cheb_degree = t->pcg_cheb_degree;
    // the one-system general solver: its grid follows pcg_blocks_per_sm
    if (c->loaded && !c->plan.resident && c->plan.n_groups <= 0) {
        const int grid = pcg_general_grid(c->p.precision, c->n_slices, c->num_sms, c->pcg_bps);
        if (grid < 1)
            return fail(c, PIC_ERR_CUDA, "pic_set_tuning: no solver grid");
        c->plan.grid = grid;
    }
    // the iteration counts of the last solves stay valid weights
    if (c->loaded && c->plan.n_groups > 0)
        return c->pcg_balance ? balance_batch(c) : replan_batch(c, nullptr);
    return PIC_OK;
}

extern "C" int pic_mesh_info(pic_ctx c, pic_info *info)
{
    REQUIRE_MESH();
    if (!info)
        return fail(c, PIC_ERR_ARG, "null info");
    info->n_nodes = c->N;
    info->n_tets = c->T;
    info->n_faces = c->F;
    info->n_free = c->n_free;
    info->nnz = c->nnz;
    info->sell_len = c->sell_len;
    info->pcg_grid = c->plan.grid;
    info->particle_grid = c->pgrid;
    for (int i = 0; i < 3; ++i) {
        info->box_lo[i] = c->lo[i];
        info->box_hi[i] = c->hi[i];
    }
    info->n_rep = c->n_rep;
    info->n_rows = c->n_rows;
    info->pcg_resident = c->plan.resident ? 1 : 0;
    info->graph = c->graph_state;
    info->mg_levels = c->plan.resident ? (c->mg.n1 > 0 ? 2 : 0) : c->gmg.nlev;
    info->mg_coarse_rows = c->plan.resident ? c->mg.n2 : c->gmg.coarse_max;
    return PIC_OK;
}

// ===========================================================================
// the steps
// ===========================================================================
extern "C" int pic_init_potential(pic_ctx c, int32_t *iters, double *rel_res)
{
    REQUIRE_MESH();
    CK(cudaMemsetAsync(c->W, 0, sizeof(unsigned long long) * c->N, c->s));
    CK(cudaMemsetAsync(c->x, 0, sizeof(double) * c->n_pad, c->s));
    CK(cudaMemsetAsync(c->sstats, 0, sizeof(pic_step_stats), c->s));
    int rc = run_pcg(c, c->sstats, nullptr);
    if (rc)
        return rc;
    rc = refresh_field(c);
    if (rc)
        return rc;
    if (iters || rel_res) {
        pic_step_stats h;
        CK(cudaMemcpyAsync(&h, c->sstats, sizeof h, cudaMemcpyDeviceToHost, c->s));
        CK(cudaStreamSynchronize(c->s));
        if (iters)
            *iters = h.pcg_iters;
        if (rel_res)
            *rel_res = h.pcg_relres;
    }
    return check_device_error(c);
}

template <typename R> static int do_inject(pic_ctx c, int64_t step)
{
    RunConst k = run_const(c);
    MeshView<R> m = view<R>(c);
    const long long step_h = step;   // pageable source: staged before the call returns
    CK(cudaMemcpyAsync(&c->st->hdr.step, &step_h, sizeof step_h, cudaMemcpyHostToDevice, c->s));
    const long long *stepp = &c->st->hdr.step;
    LAUNCH(K_INJECT_COUNT, launch_inject_count<R>(c->s, c->NQ, m, k, stepp, c->qcount, &c->st->err));
    LAUNCH(K_INJECT_SCAN, launch_inject_scan(c->s, c->NQ, c->qcount, c->qoff, c->st, c->a,
                                             c->p.capacity, 1, c->sstats));
    LAUNCH(K_INJECT_EMIT, launch_inject_emit<R>(c->s, c->pgrid, m, k, stepp, c->NQ, c->qoff,
                                                parts<R>(c, c->a), c->st));
    return PIC_OK;
}

extern "C" int inject(pic_ctx c, int64_t step, int64_t *n_injected)
{
    REQUIRE_MESH();
    if (step < 0 || step >= (1LL << 21))
        return fail(c, PIC_ERR_ARG, "inject: step out of range");
    int rc = fp64(c) ? do_inject<double>(c, step) : do_inject<float>(c, step);
    if (rc)
        return rc;
    if (n_injected) {
        DevState h;
        CK(cudaMemcpyAsync(&h, c->st, sizeof h, cudaMemcpyDeviceToHost, c->s));
        CK(cudaStreamSynchronize(c->s));
        *n_injected = h.n_new;
        return check_device_error(c);
    }
    return PIC_OK;
}

template <typename R> static int do_push(pic_ctx c)
{
    RunConst k = run_const(c);
    LAUNCH(K_PUSH_RELOCATE, launch_push_relocate<R>(c->s, c->pgrid, view<R>(c), k, parts<R>(c, c->a),
                                                    parts<R>(c, 1 - c->a), c->a, c->st, c->sstats));
    return PIC_OK;
}

extern "C" int push_relocate(pic_ctx c, int64_t step, pic_step_stats *out)
{
    REQUIRE_MESH();
    (void)step;
    CK(cudaMemsetAsync(&c->st->cnt[1 - c->a], 0, sizeof(unsigned long long), c->s));
    CK(cudaMemsetAsync(c->sstats, 0, sizeof(pic_step_stats), c->s));
    int rc = fp64(c) ? do_push<double>(c) : do_push<float>(c);
    if (rc)
        return rc;
    c->a = 1 - c->a;
    CK(cudaMemsetAsync(&c->st->n_fresh, 0, sizeof(long long), c->s));
    if (out) {
        pic_step_stats h;
        DevState d;
        CK(cudaMemcpyAsync(&h, c->sstats, sizeof h, cudaMemcpyDeviceToHost, c->s));
        CK(cudaMemcpyAsync(&d, c->st, sizeof d, cudaMemcpyDeviceToHost, c->s));
        CK(cudaStreamSynchronize(c->s));
        h.alive = (int64_t)d.cnt[c->a];
        h.injected = 0;
        h.collected_charge = (c->p.q * c->p.w_sp) * (double)h.collected;
        *out = h;
        return check_device_error(c);
    }
    return PIC_OK;
}

extern "C" int deposit(pic_ctx c, int64_t *W_out)
{
    REQUIRE_MESH();
    CK(cudaMemsetAsync(c->W, 0, sizeof(unsigned long long) * c->N, c->s));
    RunConst k = run_const(c);
    if (fp64(c))
        LAUNCH(K_DEPOSIT, launch_deposit<double>(c->s, c->pgrid, view<double>(c), k,
                                                 parts<double>(c, c->a), c->a, c->st, c->W));
    else
        LAUNCH(K_DEPOSIT, launch_deposit<float>(c->s, c->pgrid, view<float>(c), k,
                                                parts<float>(c, c->a), c->a, c->st, c->W));
    if (W_out) {
        CK(cudaMemcpyAsync(W_out, c->W, sizeof(int64_t) * c->N, cudaMemcpyDefault, c->s));
        CK(cudaStreamSynchronize(c->s));
    }
    return PIC_OK;
}

extern "C" int poisson_solve(pic_ctx c, double *phi, int32_t *iters, double *rel_res)
{
    REQUIRE_MESH();
    CK(cudaMemsetAsync(c->sstats, 0, sizeof(pic_step_stats), c->s));
    int rc = run_pcg(c, c->sstats, nullptr);
    if (rc)
        return rc;
    rc = refresh_field(c);
    if (rc)
        return rc;
    if (phi)
        CK(cudaMemcpyAsync(phi, c->phi, sizeof(double) * c->N, cudaMemcpyDefault, c->s));
    if (iters || rel_res || phi) {
        pic_step_stats h;
        CK(cudaMemcpyAsync(&h, c->sstats, sizeof h, cudaMemcpyDeviceToHost, c->s));
        CK(cudaStreamSynchronize(c->s));
        if (iters)
            *iters = h.pcg_iters;
        if (rel_res)
            *rel_res = h.pcg_relres;
        return check_device_error(c);
    }
    return PIC_OK;
}

// One PIC cycle, all on the device: the step index comes from st->hdr and
// the statistics go to c->slot, so the same launches can be captured once in
// a CUDA graph and replayed every step of the same buffer parity.
template <typename R> static int step_once(pic_ctx c)
{
    RunConst k = run_const(c);
    MeshView<R> m = view<R>(c);
    const long long *stepp = &c->st->hdr.step;
    pic_step_stats *ds = c->slot;
    CK(cudaMemsetAsync(c->W, 0, sizeof(unsigned long long) * c->N, c->s));
    CK(cudaMemsetAsync(&c->st->cnt[1 - c->a], 0, sizeof(unsigned long long), c->s));
    CK(cudaMemsetAsync(&c->st->work, 0, sizeof(unsigned long long), c->s));
    LAUNCH(K_INJECT_COUNT, launch_inject_count<R>(c->s, c->NQ, m, k, stepp, c->qcount, &c->st->err));
    LAUNCH(K_INJECT_SCAN, launch_inject_scan(c->s, c->NQ, c->qcount, c->qoff, c->st, c->a,
                                             c->p.capacity, 0, ds));
    LAUNCH(K_STEP_FUSED, launch_step_fused<R>(c->s, c->pgrid, c->walk_form, m, k, stepp, c->NQ,
                                              c->qoff,
                                              parts<R>(c, c->a), parts<R>(c, 1 - c->a), c->a,
                                              c->st, c->W, ds));
    if (c->sort_cells) {
        // survivors back into this buffer, ordered by cell
        LAUNCH(K_SORT, launch_sort_by_cell<R>(c->s, c->pgrid, c->T, parts<R>(c, 1 - c->a),
                                              parts<R>(c, c->a), &c->st->cnt[1 - c->a],
                                              &c->st->cnt[c->a], c->scnt, c->soff, c->srank,
                                              c->sscan));
    } else {
        c->a = 1 - c->a;
    }
    if (c->p.collisions)
        LAUNCH(K_COLLIDE, launch_collide<R>(c->s, coll_args<R>(c)));
    int rc = run_pcg(c, ds, &c->st->cnt[c->a]);
    if (rc)
        return rc;
    rc = refresh_field(c, true);
    if (rc)
        return rc;
    c->step = c->step + 1;
    return PIC_OK;
}

static int step_direct(pic_ctx c)
{
    return fp64(c) ? step_once<double>(c) : step_once<float>(c);
}

// Capture the step of the current parity into a graph.  Capture runs on a
// stream of the context's own (the caller's stream may be the legacy default
// stream, which cannot be captured); the graph is replayed on the caller's
// stream.  Capturing launches nothing, so the host-side step state is put
// back afterwards.  If the driver refuses any part of the capture the
// context keeps launching the kernels directly (graph_state = -1).
static void capture_step(pic_ctx c)
{
    const int a = c->a;
    const int64_t step = c->step;
    const long long launches = c->launches;
    cudaStream_t user = c->s;
    if (!c->cap_s && cudaStreamCreateWithFlags(&c->cap_s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        c->cap_s = nullptr;
        c->graph_state = -1;
        return;
    }
    if (cudaStreamSynchronize(user) != cudaSuccess) {
        cudaGetLastError();
        c->graph_state = -1;
        return;
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(c->cap_s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        c->graph_state = -1;
        return;
    }
    c->s = c->cap_s;
    const std::string err = c->err;
    int rc = step_direct(c);
    const int a_after = c->a;
    cudaError_t e = cudaStreamEndCapture(c->cap_s, &g);
    c->s = user;
    const long long per_step = c->launches - launches;
    c->launches = launches;
    c->a = a;
    c->step = step;
    cudaGraphExec_t x = nullptr;
    if (rc == PIC_OK && e == cudaSuccess && g &&
        cudaGraphInstantiate(&x, g, 0) == cudaSuccess) {
        c->gexec[a] = x;
        c->glaunch[a] = per_step;
        c->gnext[a] = a_after;
        c->graph_state = 1;
    } else {
        cudaGetLastError();
        c->err = err;
        c->graph_state = -1;
    }
    if (g)
        cudaGraphDestroy(g);
}

static int run_step(pic_ctx c)
{
    if (c->p.graph && !c->prof && c->graph_state >= 0) {
        const int a = c->a;
        if (!c->gexec[a])
            capture_step(c);
        if (c->gexec[a]) {
            CK(cudaGraphLaunch(c->gexec[a], c->s));
            c->launches += c->glaunch[a];
            c->a = c->gnext[a];
            c->step = c->step + 1;
            return PIC_OK;
        }
    }
    return step_direct(c);
}

extern "C" int pic_step(pic_ctx c, int64_t n, pic_step_stats *stats)
{
    REQUIRE_MESH();
    if (n < 0 || c->step + n >= (1LL << 21))
        return fail(c, PIC_ERR_ARG, "pic_step: bad step count");
    if (n == 0)
        return PIC_OK;
    int rc = ensure_dstats(c, n);
    if (rc)
        return rc;
    rc = balance_batch(c);
    if (rc)
        return rc;
    CK(cudaMemsetAsync(c->dstats, 0, sizeof(pic_step_stats) * (size_t)n, c->s));
    const StepHdr hdr{c->step, c->step, c->dstats, c->dstats_cap};   // staged before return
    CK(cudaMemcpyAsync(&c->st->hdr, &hdr, sizeof hdr, cudaMemcpyHostToDevice, c->s));
    CK(cudaMemsetAsync(c->slot, 0, sizeof(pic_step_stats), c->s));
    for (int64_t s = 0; s < n; ++s) {
        rc = run_step(c);
        if (rc)
            return rc;
    }
    if (stats && is_device_ptr(stats)) {
        CK(cudaMemcpyAsync(stats, c->dstats, sizeof(pic_step_stats) * (size_t)n,
                           cudaMemcpyDeviceToDevice, c->s));
        return PIC_OK;
    }
    if (stats) {
        CK(cudaMemcpyAsync(stats, c->dstats, sizeof(pic_step_stats) * (size_t)n,
                           cudaMemcpyDeviceToHost, c->s));
        CK(cudaStreamSynchronize(c->s));
        for (int64_t s = 0; s < n; ++s)
            stats[s].collected_charge = (c->p.q * c->p.w_sp) * (double)stats[s].collected;
        return check_device_error(c);
    }
    return PIC_OK;
}

// ===========================================================================
// adjoint: reverse mode over the steps (see pic_adjoint in picfem.h)
// ===========================================================================
namespace {

// device memory owned by one pic_adjoint call, freed on every exit
struct Scratch {
    std::vector<void *> mem;
    ~Scratch()
    {
        for (void *p : mem)
            cudaFree(p);
    }
    template <typename T> cudaError_t get(T **p, size_t n)
    {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, (n ? n : 1) * sizeof(T));
        if (e == cudaSuccess) {
            mem.push_back(q);
            *p = (T *)q;
        }
        return e;
    }
};

template <typename R> cudaError_t alloc_parts(Scratch &m, Particles<R> &P, long long n)
{
    cudaError_t e = cudaSuccess;
    R **f[6] = {&P.x, &P.y, &P.z, &P.vx, &P.vy, &P.vz};
    for (R **q : f)
        if (e == cudaSuccess)
            e = m.get(q, (size_t)n);
    if (e == cudaSuccess)
        e = m.get(&P.cell, (size_t)n);
    if (e == cudaSuccess)
        e = m.get(&P.id, (size_t)n);
    return e;
}

template <typename R>
cudaError_t copy_parts(cudaStream_t s, Particles<R> dst, Particles<R> src, long long n)
{
    if (n <= 0)
        return cudaSuccess;
    const size_t b = sizeof(R) * (size_t)n;
    R *d[6] = {dst.x, dst.y, dst.z, dst.vx, dst.vy, dst.vz};
    R *o[6] = {src.x, src.y, src.z, src.vx, src.vy, src.vz};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 6 && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(d[k], o[k], b, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dst.cell, src.cell, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dst.id, src.id, sizeof(long long) * (size_t)n, cudaMemcpyDeviceToDevice,
                            s);
    return e;
}

template <typename R> struct Ckpt {      // the state at the start of a step
    Particles<R> sp{};
    long long n = 0;
    double *phi = nullptr;
    int64_t step = 0;
};

template <typename R> struct TapeStep {  // what the reverse pass needs of one step
    Particles<R> pre{};                  // SPs before the push (old, then injected)
    long long n = 0, n_old = 0;
    int *dest = nullptr;                 // slot after the push, or DEST_*
    double *phi = nullptr;               // Phi_k
};

struct AdjBuffers {
    AdjSP a[2];
    double *Ebar[2];
    double *phibar, *rhs, *x, *fbar, *gE0, *gwf;
    Vec4d *E64;
    int *dest, *scan;
};

}  // namespace

template <typename R> static int save_ckpt(pic_ctx c, Scratch &m, Ckpt<R> &k)
{
    DevState h;
    CK(cudaMemcpyAsync(&h, c->st, sizeof h, cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    k.n = (long long)h.cnt[c->a];
    CK(alloc_parts(m, k.sp, k.n));
    CK(copy_parts(c->s, k.sp, parts<R>(c, c->a), k.n));
    CK(m.get(&k.phi, (size_t)c->N));
    CK(cudaMemcpyAsync(k.phi, c->phi, sizeof(double) * c->N, cudaMemcpyDeviceToDevice, c->s));
    k.step = c->step;
    return PIC_OK;
}

template <typename R> static int restore_ckpt(pic_ctx c, const Ckpt<R> &k)
{
    CK(copy_parts(c->s, parts<R>(c, c->a), k.sp, k.n));
    const unsigned long long n = (unsigned long long)k.n;   // staged before return
    const long long zero = 0;
    CK(cudaMemcpyAsync(&c->st->cnt[c->a], &n, sizeof n, cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync(&c->st->n_fresh, &zero, sizeof zero, cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync(c->phi, k.phi, sizeof(double) * c->N, cudaMemcpyDeviceToDevice, c->s));
    k_phi_to_x<<<(c->n_rows + 255) / 256, 256, 0, c->s>>>(c->n_rows, c->dof_node, c->phi, c->x);
    ++c->launches;
    CK(cudaGetLastError());
    c->step = k.step;
    return refresh_field(c);
}

// One step with the same arithmetic as pic_step, but with survivors kept in
// index order (ordered push + stable compaction back into the same buffer),
// so that a recomputed segment reproduces the forward run SP for SP.  With a
// tape, the step's SPs before the push, their destinations and Phi_k are kept.
template <typename R>
static int ordered_step(pic_ctx c, Scratch &m, const AdjBuffers &B, TapeStep<R> *tp,
                        long long *collected)
{
    const int64_t step = c->step;
    RunConst k = run_const(c);
    if (tp) {
        CK(m.get(&tp->phi, (size_t)c->N));
        CK(cudaMemcpyAsync(tp->phi, c->phi, sizeof(double) * c->N, cudaMemcpyDeviceToDevice, c->s));
    }
    int rc = do_inject<R>(c, step);
    if (rc)
        return rc;
    DevState h;
    CK(cudaMemcpyAsync(&h, c->st, sizeof h, cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    if (h.err)
        return check_device_error(c);
    const long long n = (long long)h.cnt[c->a];
    int *dest = B.dest;
    if (tp) {
        tp->n = n;
        tp->n_old = n - h.n_fresh;
        CK(alloc_parts(m, tp->pre, n));
        CK(copy_parts(c->s, tp->pre, parts<R>(c, c->a), n));
        CK(m.get(&tp->dest, (size_t)n));
        dest = tp->dest;
    }
    CK(cudaMemsetAsync(c->sstats, 0, sizeof(pic_step_stats), c->s));
    LAUNCH(K_PUSH_RELOCATE, launch_push_relocate<R>(c->s, c->pgrid, view<R>(c), k, parts<R>(c, c->a),
                                                    parts<R>(c, 1 - c->a), c->a, c->st, c->sstats,
                                                    dest));
    LAUNCH(K_COMPACT, launch_compact<R>(c->s, n, dest, parts<R>(c, 1 - c->a), parts<R>(c, c->a),
                                        c->st, c->a, B.scan));
    CK(cudaMemsetAsync(c->W, 0, sizeof(unsigned long long) * c->N, c->s));
    LAUNCH(K_DEPOSIT, launch_deposit<R>(c->s, c->pgrid, view<R>(c), k, parts<R>(c, c->a), c->a,
                                        c->st, c->W));
    rc = run_pcg(c, c->sstats, nullptr);
    if (rc)
        return rc;
    rc = refresh_field(c);
    if (rc)
        return rc;
    pic_step_stats st;
    CK(cudaMemcpyAsync(&st, c->sstats, sizeof st, cudaMemcpyDeviceToHost, c->s));
    rc = check_device_error(c);
    if (rc)
        return rc;
    *collected += st.collected;
    c->step = step + 1;
    return PIC_OK;
}

// Reverse of recorded step k.  On entry B.a[in] is the adjoint of the state
// after the step (by slot of `post`) and Ebar_next that of E_{k+1}; on exit
// B.a[1 - in] holds the adjoint of the old SPs before the step and
// Ebar_cur that of E_k.
template <typename R>
static int adjoint_step(pic_ctx c, const AdjBuffers &B, const TapeStep<R> &tp, Particles<R> post,
                        int in, const double *Ebar_next, double *Ebar_cur)
{
    // E_{k+1} = field(Phi_{k+1}), M Phi_{k+1} = f(W_{k+1}, E0): adjoint solve
    CK(cudaMemsetAsync(B.phibar, 0, sizeof(double) * c->N, c->s));
    LAUNCH(K_ADJ_FIELD, launch_field_adjoint(c->s, c->T, c->rec64, c->tet4, Ebar_next, B.phibar));
    LAUNCH(K_ADJ_ROWS, launch_gather_rows(c->s, c->n_rows, c->dof_node, B.phibar, B.rhs));
    CK(cudaMemsetAsync(B.fbar, 0, sizeof(double) * c->N, c->s));
    CK(cudaMemsetAsync(c->sstats, 0, sizeof(pic_step_stats), c->s));
    const SolveOverride ov{B.rhs, B.x, B.fbar, 1e-10};
    int rc = run_pcg(c, c->sstats, nullptr, &ov);
    if (rc)
        return rc;
    LAUNCH(K_ADJ_ROWS, launch_dE0(c->s, c->n_rows, B.x, c->fN, c->rep_slice_d, c->n_rep, c->E0_rep,
                                  B.gE0));
    if (!Ebar_cur)
        return PIC_OK;
    // E_k in FP64 from the recorded Phi_k
    LAUNCH(K_FIELD, launch_field<double>(c->s, c->T, c->rec64, c->tet4, tp.phi, B.E64, nullptr,
                                         nullptr));
    CK(cudaMemsetAsync(Ebar_cur, 0, sizeof(double) * 3 * (size_t)c->T, c->s));
    AdjStep<R> g;
    g.n = tp.n;
    g.n_old = tp.n_old;
    g.pre = tp.pre;
    g.post = post;
    g.dest = tp.dest;
    g.in = B.a[in];
    g.out = B.a[1 - in];
    g.rec64 = c->rec64;
    g.tet = c->tet4;
    g.E = B.E64;
    g.fbar = B.fbar;
    g.coef = (c->p.q * c->p.w_sp) / c->p.eps0;
    g.Ebar = Ebar_cur;
    g.gwf = B.gwf;
    g.face_tet = c->face_tet;
    g.face_rep = c->face_rep;
    g.rep_face_off = c->rep_face_off;
    g.fnhat = c->fnhat;
    g.wf = c->wf;
    g.seed = c->p.seed;
    g.fn_model = c->p.fn_model;
    g.qmdt = c->p.q_over_m * c->p.dt;
    g.dt = c->p.dt;
    g.qw = c->p.q * c->p.w_sp;
    LAUNCH(K_ADJ_SP, launch_adjoint_sp<R>(c->s, g));
    return PIC_OK;
}

template <typename R>
static int run_adjoint(pic_ctx c, int64_t n_steps, int32_t ckpt_every, double *Q, double *dE0,
                       double *dwf)
{
    Scratch m;
    AdjBuffers B{};
    const size_t cap = (size_t)c->p.capacity;
    for (int s = 0; s < 2; ++s) {
        double **f[7] = {&B.a[s].rx, &B.a[s].ry, &B.a[s].rz, &B.a[s].vx,
                         &B.a[s].vy, &B.a[s].vz, &B.a[s].w};
        for (double **q : f)
            CK(m.get(q, cap));
        CK(m.get(&B.Ebar[s], 3 * (size_t)c->T));
    }
    CK(m.get(&B.phibar, (size_t)c->N));
    CK(m.get(&B.fbar, (size_t)c->N));
    CK(m.get(&B.rhs, (size_t)c->n_pad));
    CK(m.get(&B.x, (size_t)c->n_pad));
    CK(m.get(&B.gE0, (size_t)c->n_rep));
    CK(m.get(&B.gwf, (size_t)c->F));
    CK(m.get(&B.E64, (size_t)c->T));
    CK(m.get(&B.dest, cap));
    CK(m.get(&B.scan, 2 * ((cap + 1023) / 1024) + 2));
    CK(cudaMemsetAsync(B.x, 0, sizeof(double) * c->n_pad, c->s));
    CK(cudaMemsetAsync(B.gE0, 0, sizeof(double) * c->n_rep, c->s));
    CK(cudaMemsetAsync(B.gwf, 0, sizeof(double) * (c->F ? c->F : 1), c->s));

    // forward: Phi_0 of the SPs present, then the steps, with checkpoints
    CK(cudaMemsetAsync(c->W, 0, sizeof(unsigned long long) * c->N, c->s));
    RunConst k = run_const(c);
    LAUNCH(K_DEPOSIT, launch_deposit<R>(c->s, c->pgrid, view<R>(c), k, parts<R>(c, c->a), c->a,
                                        c->st, c->W));
    CK(cudaMemsetAsync(c->sstats, 0, sizeof(pic_step_stats), c->s));
    int rc = run_pcg(c, c->sstats, nullptr);
    if (!rc)
        rc = refresh_field(c);
    if (!rc)
        rc = check_device_error(c);
    if (rc)
        return rc;
    const int64_t n_seg = (n_steps + ckpt_every - 1) / ckpt_every;
    std::vector<Ckpt<R>> ck((size_t)n_seg + 1);
    long long collected = 0;
    for (int64_t s = 0; s < n_seg; ++s) {
        if ((rc = save_ckpt(c, m, ck[s])))
            return rc;
        const int64_t len = std::min<int64_t>(ckpt_every, n_steps - s * ckpt_every);
        for (int64_t j = 0; j < len; ++j)
            if ((rc = ordered_step<R>(c, m, B, nullptr, &collected)))
                return rc;
    }
    if ((rc = save_ckpt(c, m, ck[n_seg])))
        return rc;

    // reverse, one recomputed segment at a time
    CK(cudaMemsetAsync(B.Ebar[0], 0, sizeof(double) * 3 * (size_t)c->T, c->s));
    int in = 0, eb = 0;   // B.a[in]: adjoint of the current state; B.Ebar[eb]: of its E
    CK(cudaMemsetAsync(B.a[0].rx, 0, sizeof(double) * cap, c->s));
    {
        double *z[7] = {B.a[0].rx, B.a[0].ry, B.a[0].rz, B.a[0].vx, B.a[0].vy, B.a[0].vz, B.a[0].w};
        for (double *q : z)
            CK(cudaMemsetAsync(q, 0, sizeof(double) * cap, c->s));
    }
    for (int64_t s = n_seg - 1; s >= 0; --s) {
        Scratch seg;
        if ((rc = restore_ckpt(c, ck[s])))
            return rc;
        const int64_t len = std::min<int64_t>(ckpt_every, n_steps - s * ckpt_every);
        std::vector<TapeStep<R>> tape((size_t)len);
        long long dummy = 0;
        for (int64_t j = 0; j < len; ++j)
            if ((rc = ordered_step<R>(c, seg, B, &tape[j], &dummy)))
                return rc;
        for (int64_t j = len - 1; j >= 0; --j) {
            Particles<R> post = j + 1 < len ? tape[j + 1].pre : ck[s + 1].sp;
            if ((rc = adjoint_step<R>(c, B, tape[j], post, in, B.Ebar[eb], B.Ebar[1 - eb])))
                return rc;
            in = 1 - in;
            eb = 1 - eb;
        }
        CK(cudaStreamSynchronize(c->s));   // before the segment's tape is freed
    }
    // Phi_0 = M^-1 f(W_0, E0)
    TapeStep<R> none;
    if ((rc = adjoint_step<R>(c, B, none, Particles<R>{}, in, B.Ebar[eb], nullptr)))
        return rc;
    if ((rc = restore_ckpt(c, ck[n_seg])))
        return rc;
    if (dE0)
        CK(cudaMemcpyAsync(dE0, B.gE0, sizeof(double) * c->n_rep, cudaMemcpyDeviceToHost, c->s));
    if (dwf && c->F)
        CK(cudaMemcpyAsync(dwf, B.gwf, sizeof(double) * c->F, cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    if (Q)
        *Q = (c->p.q * c->p.w_sp) * (double)collected;
    return check_device_error(c);
}

extern "C" int pic_adjoint(pic_ctx c, int64_t n_steps, int32_t ckpt_every, double *Q,
                           double *dQ_dE0, double *dQ_dphi)
{
    REQUIRE_MESH();
    if (c->p.collisions)
        return fail(c, PIC_ERR_NOT_IMPLEMENTED, "pic_adjoint: collisions are not differentiated");
    if (n_steps < 1 || ckpt_every < 1 || c->step + n_steps >= (1LL << 21))
        return fail(c, PIC_ERR_ARG, "pic_adjoint: bad step counts");
    free_graphs(c);
    return fp64(c) ? run_adjoint<double>(c, n_steps, ckpt_every, Q, dQ_dE0, dQ_dphi)
                   : run_adjoint<float>(c, n_steps, ckpt_every, Q, dQ_dE0, dQ_dphi);
}

extern "C" int pic_collide(pic_ctx c, int64_t step)
{
    REQUIRE_MESH();
    if (step < 0 || step >= (1LL << 21))
        return fail(c, PIC_ERR_ARG, "pic_collide: step out of range");
    if (!c->ccnt) {
        int rc = alloc_collision_scratch(c);
        if (rc)
            return rc;
    }
    const long long step_h = step;
    CK(cudaMemcpyAsync(&c->st->hdr.step, &step_h, sizeof step_h, cudaMemcpyHostToDevice, c->s));
    if (fp64(c))
        LAUNCH(K_COLLIDE, launch_collide<double>(c->s, coll_args<double>(c)));
    else
        LAUNCH(K_COLLIDE, launch_collide<float>(c->s, coll_args<float>(c)));
    return check_device_error(c);
}

extern "C" int pic_set_dirichlet(pic_ctx c, const double *g)
{
    REQUIRE_MESH();
    if (!g)
        return fail(c, PIC_ERR_ARG, "null values");
    std::vector<double> h((size_t)c->N);
    for (int n = 0; n < c->N; ++n) {
        if (c->dir_h[n] && !std::isfinite(g[n]))
            return fail(c, PIC_ERR_ARG, "pic_set_dirichlet: non-finite value at node %d", n);
        h[n] = c->dir_h[n] ? g[n] : 0.0;
    }
    CK(cudaMemcpyAsync(c->gD, h.data(), sizeof(double) * c->N, cudaMemcpyHostToDevice, c->s));
    LAUNCH(K_UTIL, launch_dirichlet_load(c->s, c->n_rows, c->dptr, c->dcon, c->rec64, c->det,
                                         c->tet4, c->gD, c->fD));
    k_set_dirichlet<<<(c->N + 255) / 256, 256, 0, c->s>>>(c->N, c->dir, c->gD, c->phi);
    ++c->launches;
    CK(cudaGetLastError());
    int rc = refresh_field(c);
    if (rc)
        return rc;
    CK(cudaStreamSynchronize(c->s));
    return PIC_OK;
}

extern "C" int pic_set_applied_field(pic_ctx c, const double *E0)
{
    REQUIRE_MESH();
    if (!E0)
        return fail(c, PIC_ERR_ARG, "null E0");
    for (int r = 0; r < c->n_rep; ++r)
        if (!std::isfinite(E0[r]))
            return fail(c, PIC_ERR_ARG, "pic_set_applied_field: non-finite E0");
    CK(cudaMemcpyAsync(c->E0_rep, E0, sizeof(double) * c->n_rep, cudaMemcpyHostToDevice, c->s));
    CK(cudaMemsetAsync(c->fN, 0, sizeof(double) * c->n_pad, c->s));
    LAUNCH(K_UTIL, launch_neumann(c->s, c->n_rows, c->nfptr, c->nfcon, c->tet4, c->xyz, c->tet_rep,
                                  c->E0_rep, c->fN));
    CK(cudaStreamSynchronize(c->s));
    if (c->n_rep == 1)
        c->p.E0 = E0[0];
    return PIC_OK;
}

// ===========================================================================
// state
// ===========================================================================
extern "C" int pic_get_step(pic_ctx c, int64_t *step)
{
    if (!c || !step)
        return fail(c, PIC_ERR_ARG, "null argument");
    *step = c->step;
    return PIC_OK;
}
extern "C" int pic_set_step(pic_ctx c, int64_t step)
{
    if (!c || step < 0 || step >= (1LL << 21))
        return fail(c, PIC_ERR_ARG, "bad step");
    c->step = step;
    return PIC_OK;
}

extern "C" int pic_get_potential(pic_ctx c, double *phi)
{
    REQUIRE_MESH();
    if (!phi)
        return fail(c, PIC_ERR_ARG, "null phi");
    CK(cudaMemcpyAsync(phi, c->phi, sizeof(double) * c->N, cudaMemcpyDefault, c->s));
    CK(cudaStreamSynchronize(c->s));
    return PIC_OK;
}

extern "C" int pic_get_potential_async(pic_ctx c, double *phi)
{
    REQUIRE_MESH();
    if (!phi)
        return fail(c, PIC_ERR_ARG, "null phi");
    CK(cudaMemcpyAsync(phi, c->phi, sizeof(double) * c->N, cudaMemcpyDefault, c->s));
    return PIC_OK;
}

extern "C" int pic_set_potential(pic_ctx c, const double *phi)
{
    REQUIRE_MESH();
    if (!phi)
        return fail(c, PIC_ERR_ARG, "null phi");
    CK(cudaMemcpyAsync(c->phi, phi, sizeof(double) * c->N, cudaMemcpyDefault, c->s));
    k_set_dirichlet<<<(c->N + 255) / 256, 256, 0, c->s>>>(c->N, c->dir, c->gD, c->phi);
    ++c->launches;
    k_phi_to_x<<<(c->n_rows + 255) / 256, 256, 0, c->s>>>(c->n_rows, c->dof_node, c->phi, c->x);
    ++c->launches;
    CK(cudaGetLastError());
    int rc = refresh_field(c);
    if (rc)
        return rc;
    CK(cudaStreamSynchronize(c->s));
    return PIC_OK;
}

extern "C" int pic_get_field(pic_ctx c, double *E)
{
    REQUIRE_MESH();
    if (!E)
        return fail(c, PIC_ERR_ARG, "null E");
    void *tmp = nullptr;
    CK(stage(c, 0, sizeof(double) * 3 * c->T, &tmp));
    if (fp64(c))
        LAUNCH(K_UTIL, launch_field_unpack<double>(c->s, c->T, (const Vec4d *)c->E, (double *)tmp));
    else
        LAUNCH(K_UTIL, launch_field_unpack<float>(c->s, c->T, (const float4 *)c->E, (double *)tmp));
    CK(cudaMemcpyAsync(E, tmp, sizeof(double) * 3 * c->T, cudaMemcpyDefault, c->s));
    CK(cudaStreamSynchronize(c->s));
    return PIC_OK;
}

extern "C" int pic_get_charge(pic_ctx c, int64_t *W)
{
    REQUIRE_MESH();
    if (!W)
        return fail(c, PIC_ERR_ARG, "null W");
    CK(cudaMemcpyAsync(W, c->W, sizeof(int64_t) * c->N, cudaMemcpyDefault, c->s));
    CK(cudaStreamSynchronize(c->s));
    return PIC_OK;
}

extern "C" int pic_num_particles(pic_ctx c, int64_t *n)
{
    REQUIRE_MESH();
    if (!n)
        return fail(c, PIC_ERR_ARG, "null n");
    DevState h;
    CK(cudaMemcpyAsync(&h, c->st, sizeof h, cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    *n = (int64_t)h.cnt[c->a];
    return PIC_OK;
}

extern "C" int pic_get_particles(pic_ctx c, double *r, double *v, int32_t *cell, int64_t *id)
{
    REQUIRE_MESH();
    int64_t n = 0;
    int rc = pic_num_particles(c, &n);
    if (rc)
        return rc;
    if (n == 0)
        return PIC_OK;
    void *buf[4] = {r, v, cell, id};
    size_t sz[4] = {sizeof(double) * 3 * n, sizeof(double) * 3 * n, sizeof(int) * n,
                    sizeof(long long) * n};
    void *dev[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int i = 0; i < 4; ++i) {
        if (!buf[i])
            continue;
        if (is_device_ptr(buf[i]))
            dev[i] = buf[i];
        else
            CK(stage(c, i, sz[i], &dev[i]));
    }
    if (fp64(c))
        LAUNCH(K_UTIL, launch_pack<double>(c->s, n, parts<double>(c, c->a), (double *)dev[0],
                                           (double *)dev[1], (int *)dev[2], (long long *)dev[3]));
    else
        LAUNCH(K_UTIL, launch_pack<float>(c->s, n, parts<float>(c, c->a), (double *)dev[0],
                                          (double *)dev[1], (int *)dev[2], (long long *)dev[3]));
    for (int i = 0; i < 4; ++i)
        if (buf[i] && dev[i] != buf[i])
            CK(cudaMemcpyAsync(buf[i], dev[i], sz[i], cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    return PIC_OK;
}

extern "C" int pic_set_particles(pic_ctx c, int64_t n, const double *r, const double *v,
                                 const int32_t *cell, const int64_t *id)
{
    REQUIRE_MESH();
    if (n < 0 || n > c->p.capacity)
        return fail(c, PIC_ERR_CAPACITY, "pic_set_particles: %lld SPs exceed the capacity",
                    (long long)n);
    if (n > 0 && (!r || !v || !cell || !id))
        return fail(c, PIC_ERR_ARG, "pic_set_particles: null array");
    const void *buf[4] = {r, v, cell, id};
    size_t sz[4] = {sizeof(double) * 3 * n, sizeof(double) * 3 * n, sizeof(int) * n,
                    sizeof(long long) * n};
    const void *dev[4] = {nullptr, nullptr, nullptr, nullptr};
    if (n > 0) {
        for (int i = 0; i < 4; ++i) {
            if (is_device_ptr(buf[i])) {
                dev[i] = buf[i];
            } else {
                void *d = nullptr;
                CK(stage(c, i, sz[i], &d));
                CK(cudaMemcpyAsync(d, buf[i], sz[i], cudaMemcpyHostToDevice, c->s));
                dev[i] = d;
            }
        }
        if (!is_device_ptr(cell)) {
            for (int64_t i = 0; i < n; ++i)
                if (cell[i] < 0 || cell[i] >= c->T)
                    return fail(c, PIC_ERR_ARG, "pic_set_particles: cell out of range");
        }
        if (fp64(c))
            LAUNCH(K_UTIL, launch_unpack<double>(c->s, n, (const double *)dev[0], (const double *)dev[1],
                                                 (const int *)dev[2], (const long long *)dev[3],
                                                 parts<double>(c, c->a)));
        else
            LAUNCH(K_UTIL, launch_unpack<float>(c->s, n, (const double *)dev[0], (const double *)dev[1],
                                                (const int *)dev[2], (const long long *)dev[3],
                                                parts<float>(c, c->a)));
    }
    DevState h;
    CK(cudaMemcpyAsync(&h, c->st, sizeof h, cudaMemcpyDeviceToHost, c->s));
    CK(cudaStreamSynchronize(c->s));
    h.cnt[c->a] = (unsigned long long)n;
    h.cnt[1 - c->a] = 0;
    h.n_fresh = 0;
    h.n_new = 0;
    CK(cudaMemcpyAsync(c->st, &h, sizeof h, cudaMemcpyHostToDevice, c->s));
    CK(cudaStreamSynchronize(c->s));
    return PIC_OK;
}

extern "C" int pic_set_work_function(pic_ctx c, const double *wf)
{
    REQUIRE_MESH();
    if (!wf)
        return fail(c, PIC_ERR_ARG, "null work function");
    if (!is_device_ptr(wf))
        for (int f = 0; f < c->F; ++f)
            if (!(wf[f] > 0) || !std::isfinite(wf[f]))
                return fail(c, PIC_ERR_ARG, "pic_set_work_function: face %d invalid", f);
    if (c->F)
        CK(cudaMemcpyAsync(c->wf, wf, sizeof(double) * c->F, cudaMemcpyDefault, c->s));
    return PIC_OK;
}

// ===========================================================================
// counters and profiling
// ===========================================================================
extern "C" int pic_launch_count(pic_ctx c, int64_t *launches)
{
    if (!c || !launches)
        return fail(c, PIC_ERR_ARG, "null argument");
    *launches = c->launches;
    return PIC_OK;
}

extern "C" int pic_profile_enable(pic_ctx c, int32_t enable)
{
    if (!c)
        return fail(nullptr, PIC_ERR_ARG, "null context");
    CK(cudaStreamSynchronize(c->s));
    for (auto &r : c->prof_recs) {
        c->ev_pool.push_back(r.a);
        c->ev_pool.push_back(r.b);
    }
    c->prof_recs.clear();
    for (int k = 0; k < K_NUM; ++k) {
        c->prof_ms[k] = 0;
        c->prof_n[k] = 0;
    }
    c->prof = enable != 0;
    return PIC_OK;
}

extern "C" int pic_profile_read(pic_ctx c, pic_profile_report *out)
{
    if (!c || !out)
        return fail(c, PIC_ERR_ARG, "null argument");
    CK(cudaStreamSynchronize(c->s));
    for (auto &r : c->prof_recs) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, r.a, r.b));
        c->prof_ms[r.kid] += ms;
        c->prof_n[r.kid] += 1;
        c->ev_pool.push_back(r.a);
        c->ev_pool.push_back(r.b);
    }
    c->prof_recs.clear();
    out->n = 0;
    for (int k = 0; k < K_NUM && out->n < PIC_PROF_MAX; ++k) {
        if (!c->prof_n[k])
            continue;
        out->name[out->n] = kKernelNames[k];
        out->launches[out->n] = c->prof_n[k];
        out->ms[out->n] = c->prof_ms[k];
        out->n++;
    }
    return PIC_OK;
}

extern "C" int pic_sync(pic_ctx c)
{
    if (!c)
        return fail(nullptr, PIC_ERR_ARG, "null context");
    CK(cudaSetDevice(c->dev));
    CK(cudaStreamSynchronize(c->s));
    if (!c->loaded)
        return PIC_OK;
    return check_device_error(c);
}
