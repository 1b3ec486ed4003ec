// mg.cu -- set-up of the multigrid preconditioners of the solver: a
// three-level V-cycle for the resident kernels (mg_build) and a V-cycle of
// as many levels as needed for the general kernels (gmg_build), both for
// M Phi = f (App. B, eq. poisson_mat) and built from the matrix alone, at
// mesh_load.
//
// Coarse spaces by aggregation.  A pass of pairwise matching (Notay,
// "An aggregation-based algebraic multigrid method", ETNA 37, 2010) takes the
// rows in order and pairs each row not yet matched with the unmatched row of
// its most negative coupling; several passes on the successive Galerkin
// matrices give aggregates of up to 2^passes rows that follow the strong
// couplings (on a graded grid, the short edges).  Level 1 aggregates the fine
// rows, level 2 the level-1 rows; the prolongations are piecewise constant
// (P has one 1 per row), the coarse matrices are the Galerkin products
// A_l+1 = P^T A_l P, so they stay symmetric positive definite.
//
// Every aggregate stays inside one solver block (the matching never pairs
// rows of different blocks), so restriction and prolongation never cross
// blocks; the level-1 rows of a block are numbered contiguously and their
// matrix rows carry block-local columns [own rows | halo], like the fine
// level.  Level 2 is solved exactly: its dense inverse (FP64 Cholesky,
// stored in FP32) is applied row by row by the block that owns the row.
#include <algorithm>
#include <cmath>
#include <thread>
#include <utility>
#include <vector>

#include "common.cuh"

namespace pf {

namespace {

// CSR matrix over rows 0..n-1 (columns sorted, no duplicates)
struct Csr {
    int n = 0;
    std::vector<int> ptr, col;
    std::vector<double> val;
};

// One pass of pairwise matching within blocks (part[i] = block of row i):
// agg[i] = the aggregate of row i, numbered in the order of their first row
// (so each block's aggregates are contiguous).  Zero couplings never pair.
static int pairwise_pass(const Csr &A, const std::vector<int> &part, std::vector<int> &agg)
{
    agg.assign((size_t)A.n, -1);
    int na = 0;
    for (int i = 0; i < A.n; ++i) {
        if (agg[i] >= 0)
            continue;
        int best_j = -1;
        double best = 0.0;
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
            const int j = A.col[k];
            if (j == i || agg[j] >= 0 || part[j] != part[i])
                continue;
            if (A.val[k] < best) {
                best = A.val[k];
                best_j = j;
            }
        }
        agg[i] = na;
        if (best_j >= 0)
            agg[best_j] = na;
        ++na;
    }
    return na;
}

// Galerkin product P^T A P for the piecewise-constant P of `agg`; an entry
// exists where some A_ij is stored with a nonzero value (the pattern stays
// symmetric whatever the rounding of the sums).  Each coarse row gathers the
// rows of its aggregate in increasing order and their entries in column
// order, so every coarse entry is the sum of its fine entries in row-major
// order; O(nnz) with a marker per coarse column.
static Csr galerkin(const Csr &A, const std::vector<int> &agg, int na)
{
    std::vector<int> mp((size_t)na + 1, 0), mi((size_t)A.n);
    for (int i = 0; i < A.n; ++i)
        mp[agg[i] + 1] += 1;
    for (int a = 0; a < na; ++a)
        mp[a + 1] += mp[a];
    {
        std::vector<int> fill(mp.begin(), mp.end() - 1);
        for (int i = 0; i < A.n; ++i)
            mi[fill[agg[i]]++] = i;
    }
    Csr C;
    C.n = na;
    C.ptr.assign((size_t)na + 1, 0);
    C.col.reserve(A.col.size() / 2);
    C.val.reserve(A.col.size() / 2);
    std::vector<int> mark((size_t)na, -1), cols;
    std::vector<double> acc((size_t)na, 0.0);
    for (int a = 0; a < na; ++a) {
        cols.clear();
        for (int m = mp[a]; m < mp[a + 1]; ++m) {
            const int i = mi[m];
            for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
                if (A.val[k] == 0.0)
                    continue;
                const int b = agg[A.col[k]];
                if (mark[b] != a) {
                    mark[b] = a;
                    acc[b] = 0.0;
                    cols.push_back(b);
                }
                acc[b] += A.val[k];
            }
        }
        std::sort(cols.begin(), cols.end());
        for (int b : cols) {
            C.col.push_back(b);
            C.val.push_back(acc[b]);
        }
        C.ptr[a + 1] = (int)C.col.size();
    }
    return C;
}

// passes of pairwise matching: agg (rows of A -> aggregates), the coarse
// matrix and the block of every aggregate
static Csr coarsen(const Csr &A, const std::vector<int> &part, int passes, std::vector<int> &agg,
                   std::vector<int> &cpart)
{
    agg.resize((size_t)A.n);
    for (int i = 0; i < A.n; ++i)
        agg[i] = i;
    Csr cur = A;
    std::vector<int> p = part, a;
    for (int s = 0; s < passes; ++s) {
        const int na = pairwise_pass(cur, p, a);
        if (na == cur.n)
            break;                               // nothing left to pair
        Csr next = galerkin(cur, a, na);
        std::vector<int> np((size_t)na);
        for (int i = 0; i < cur.n; ++i)
            np[a[i]] = p[i];
        for (int i = 0; i < A.n; ++i)
            agg[i] = a[agg[i]];
        cur = std::move(next);
        p = std::move(np);
    }
    cpart = p;
    return cur;
}

// Block-local columns [own | sorted halo] of the rows of each block, and the
// halo lists; false when block b reads block o's rows but o not b's.
static bool local_columns(const Csr &A, const std::vector<int> &off, int G, std::vector<int> &lcol,
                          std::vector<int> &hptr, std::vector<int> &hidx, int &max_local,
                          int &max_own)
{
    auto owner = [&](int j) {
        return (int)(std::upper_bound(off.begin(), off.end(), j) - off.begin()) - 1;
    };
    lcol.assign(A.col.size(), 0);
    hptr.assign((size_t)G + 1, 0);
    hidx.clear();
    max_local = max_own = 0;
    std::vector<char> reads((size_t)G * G, 0);
    std::vector<int> ext;
    for (int b = 0; b < G; ++b) {
        const int r0 = off[b], r1 = off[b + 1], own = r1 - r0;
        ext.clear();
        for (int i = r0; i < r1; ++i)
            for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k)
                if (A.col[k] < r0 || A.col[k] >= r1)
                    ext.push_back(A.col[k]);
        std::sort(ext.begin(), ext.end());
        ext.erase(std::unique(ext.begin(), ext.end()), ext.end());
        for (int i = r0; i < r1; ++i)
            for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
                const int j = A.col[k];
                lcol[k] = (j >= r0 && j < r1)
                              ? j - r0
                              : own + (int)(std::lower_bound(ext.begin(), ext.end(), j) - ext.begin());
            }
        for (int j : ext)
            reads[(size_t)b * G + owner(j)] = 1;
        hidx.insert(hidx.end(), ext.begin(), ext.end());
        hptr[b + 1] = (int)hidx.size();
        max_local = std::max(max_local, own + (int)ext.size());
        max_own = std::max(max_own, own);
    }
    for (int b = 0; b < G; ++b)
        for (int o = 0; o < G; ++o)
            if (reads[(size_t)b * G + o] != reads[(size_t)o * G + b])
                return false;
    return true;
}

// members of each aggregate, as indices local to its block
static void members(const std::vector<int> &agg, int na, const std::vector<int> &row_off_of,
                    std::vector<int> &ptr, std::vector<int> &idx)
{
    ptr.assign((size_t)na + 1, 0);
    for (size_t i = 0; i < agg.size(); ++i)
        if (agg[i] >= 0)
            ptr[agg[i] + 1] += 1;
    for (int a = 0; a < na; ++a)
        ptr[a + 1] += ptr[a];
    idx.assign((size_t)ptr[na], 0);
    std::vector<int> fill(ptr.begin(), ptr.end() - 1);
    for (size_t i = 0; i < agg.size(); ++i)
        if (agg[i] >= 0)
            idx[fill[agg[i]]++] = (int)i - row_off_of[i];
}

// Gershgorin bound of D^-1 A
static double gershgorin(const Csr &A)
{
    double b = 0.0;
    for (int i = 0; i < A.n; ++i) {
        double s = 0.0, d = 0.0;
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
            s += std::fabs(A.val[k]);
            if (A.col[k] == i)
                d = A.val[k];
        }
        if (d > 0.0)
            b = std::max(b, s / d);
    }
    return b > 0.0 ? b : 2.0;
}

// Inverse of a dense SPD matrix (row-major): Cholesky A = L L^T, then
// L^-1 by forward substitution and A^-1 = L^-T L^-1, stored in FP32.
static bool dense_spd_inverse(std::vector<double> A, int n, std::vector<float> &inv)
{
    for (int j = 0; j < n; ++j) {
        double *Lj = A.data() + (size_t)j * n;
        double d = Lj[j];
        for (int k = 0; k < j; ++k)
            d -= Lj[k] * Lj[k];
        if (!(d > 0.0))
            return false;
        d = std::sqrt(d);
        Lj[j] = d;
        for (int i = j + 1; i < n; ++i) {
            double *Li = A.data() + (size_t)i * n;
            double v = Li[j];
            for (int k = 0; k < j; ++k)
                v -= Li[k] * Lj[k];
            Li[j] = v / d;
        }
    }
    // W = L^-1 (lower triangular), row by row: W_i. = (e_i - sum_{k<i} L_ik W_k.) / L_ii
    std::vector<double> W((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) {
        double *Wi = W.data() + (size_t)i * n;
        const double *Li = A.data() + (size_t)i * n;
        Wi[i] = 1.0;
        for (int k = 0; k < i; ++k) {
            const double l = Li[k];
            const double *Wk = W.data() + (size_t)k * n;
            for (int c = 0; c <= k; ++c)
                Wi[c] -= l * Wk[c];
        }
        const double inv_d = 1.0 / Li[i];
        for (int c = 0; c <= i; ++c)
            Wi[c] *= inv_d;
    }
    // A^-1 = W^T W: (A^-1)_rc = sum_{k >= max(r, c)} W_kr W_kc
    std::vector<double> S((size_t)n * n, 0.0);
    for (int k = 0; k < n; ++k) {
        const double *Wk = W.data() + (size_t)k * n;
        for (int r = 0; r <= k; ++r) {
            const double w = Wk[r];
            if (w == 0.0)
                continue;
            double *Sr = S.data() + (size_t)r * n;
            for (int c = 0; c <= k; ++c)
                Sr[c] += w * Wk[c];
        }
    }
    inv.resize((size_t)n * n);
    for (size_t i = 0; i < inv.size(); ++i)
        inv[i] = (float)S[i];
    return true;
}

}  // namespace

// The fine matrix in CSR from its sliced ELLPACK (rows without a diagonal --
// padding -- are left empty; zero entries are dropped).
static Csr sell_to_csr(const int *sptr, const int *scol, const double *sval, const double *dinv,
                       int n_slices)
{
    const int n = 32 * n_slices;
    Csr A;
    A.n = n;
    A.ptr.assign((size_t)n + 1, 0);
    A.col.reserve((size_t)sptr[n_slices]);
    A.val.reserve((size_t)sptr[n_slices]);
    std::vector<std::pair<int, double>> row;
    for (int s = 0; s < n_slices; ++s) {
        const int w = (sptr[s + 1] - sptr[s]) / 32;
        for (int l = 0; l < 32; ++l) {
            const int i = 32 * s + l;
            row.clear();
            if (dinv[i] != 0.0)
                for (int k = 0; k < w; ++k) {
                    const size_t e = (size_t)sptr[s] + (size_t)k * 32 + l;
                    if (sval[e] != 0.0)
                        row.emplace_back(scol[e], sval[e]);
                }
            std::sort(row.begin(), row.end());
            for (auto &x : row) {
                A.col.push_back(x.first);
                A.val.push_back(x.second);
            }
            A.ptr[i + 1] = (int)A.col.size();
        }
    }
    return A;
}

bool mg_build(const int *sptr, const int *scol, const double *sval, const double *dinv,
              int n_slices, int G, int passes0, int passes1, int max_coarse, MgHost *out)
{
    *out = MgHost{};
    const int n = 32 * n_slices;
    Csr A = sell_to_csr(sptr, scol, sval, dinv, n_slices);
    std::vector<int> part((size_t)n), row0_of((size_t)n);
    for (long long b = 0; b < G; ++b) {
        const int s0 = (int)((b * n_slices) / G), s1 = (int)(((b + 1) * n_slices) / G);
        for (int i = 32 * s0; i < 32 * s1; ++i) {
            part[i] = (int)b;
            row0_of[i] = 32 * s0;
        }
    }
    // level 1
    std::vector<int> agg0, part1;
    Csr A1 = coarsen(A, part, passes0, agg0, part1);
    // padding rows (no diagonal) belong to no aggregate: drop the singletons
    // they formed and renumber
    {
        std::vector<int> keep((size_t)A1.n, 0), renum((size_t)A1.n, -1);
        for (int i = 0; i < n; ++i)
            if (A.ptr[i + 1] > A.ptr[i])
                keep[agg0[i]] = 1;
        int m = 0;
        for (int a = 0; a < A1.n; ++a)
            if (keep[a])
                renum[a] = m++;
        if (m < A1.n) {
            Csr B;
            B.n = m;
            B.ptr.assign((size_t)m + 1, 0);
            std::vector<int> bp((size_t)m);
            for (int a = 0; a < A1.n; ++a) {
                if (renum[a] < 0)
                    continue;
                bp[renum[a]] = part1[a];
                for (int k = A1.ptr[a]; k < A1.ptr[a + 1]; ++k) {
                    B.col.push_back(renum[A1.col[k]]);
                    B.val.push_back(A1.val[k]);
                }
                B.ptr[renum[a] + 1] = (int)B.col.size();
            }
            for (int i = 0; i < n; ++i)
                agg0[i] = renum[agg0[i]];
            A1 = std::move(B);
            part1 = std::move(bp);
        }
    }
    for (int i = 0; i < n; ++i)
        if (A.ptr[i + 1] == A.ptr[i])
            agg0[i] = -1;
    const int n1 = A1.n;
    if (n1 < 2)
        return false;
    std::vector<int> l1_off((size_t)G + 1, 0);
    for (int a = 0; a < n1; ++a)
        l1_off[part1[a] + 1] += 1;
    for (int b = 0; b < G; ++b)
        l1_off[b + 1] += l1_off[b];
    for (int a = 1; a < n1; ++a)
        if (part1[a] < part1[a - 1])
            return false;                         // aggregates are numbered block by block
    // level 2: more passes on the level-1 matrix until it is small enough
    std::vector<int> agg1, part2;
    Csr A2 = coarsen(A1, part1, passes1, agg1, part2);
    for (int extra = 0; A2.n > max_coarse && extra < 4; ++extra) {
        std::vector<int> a, p;
        Csr B = coarsen(A2, part2, 1, a, p);
        if (B.n == A2.n)
            break;
        for (int l = 0; l < n1; ++l)
            agg1[l] = a[agg1[l]];
        A2 = std::move(B);
        part2 = std::move(p);
    }
    const int n2 = A2.n;
    if (n2 > max_coarse || n2 < 1)
        return false;
    std::vector<int> l2_off((size_t)G + 1, 0);
    for (int q = 0; q < n2; ++q)
        l2_off[part2[q] + 1] += 1;
    for (int b = 0; b < G; ++b)
        l2_off[b + 1] += l2_off[b];
    // level-1 local columns, halos, members and the level-2 aggregates
    MgHost &m = *out;
    m.n1 = n1;
    m.n2 = n2;
    if (!local_columns(A1, l1_off, G, m.a1_col, m.h1_ptr, m.h1_idx, m.max_l1_local, m.max_l1_own))
        return false;
    m.a1_ptr = A1.ptr;
    m.a1_val = A1.val;
    m.dinv1.resize((size_t)n1);
    for (int a = 0; a < n1; ++a) {
        double d = 0.0;
        for (int k = A1.ptr[a]; k < A1.ptr[a + 1]; ++k)
            if (A1.col[k] == a)
                d = A1.val[k];
        if (!(d > 0.0))
            return false;
        m.dinv1[a] = 1.0 / d;
    }
    m.lmax1 = gershgorin(A1);
    m.agg0.assign((size_t)n, -1);
    for (int i = 0; i < n; ++i)
        if (agg0[i] >= 0)
            m.agg0[i] = agg0[i] - l1_off[part[i]];
    members(agg0, n1, row0_of, m.m0_ptr, m.m0_idx);
    std::vector<int> l1_row0((size_t)n1);
    for (int a = 0; a < n1; ++a)
        l1_row0[a] = l1_off[part1[a]];
    members(agg1, n2, l1_row0, m.m1_ptr, m.m1_idx);
    m.agg1.resize((size_t)n1);
    for (int a = 0; a < n1; ++a)
        m.agg1[a] = agg1[a] - l2_off[part2[agg1[a]]];
    m.l1_off = l1_off;
    m.l2_off = l2_off;
    m.max_l2_own = 0;
    for (int b = 0; b < G; ++b)
        m.max_l2_own = std::max(m.max_l2_own, l2_off[b + 1] - l2_off[b]);
    std::vector<double> D((size_t)n2 * n2, 0.0);
    for (int q = 0; q < n2; ++q)
        for (int k = A2.ptr[q]; k < A2.ptr[q + 1]; ++k)
            D[(size_t)q * n2 + A2.col[k]] = A2.val[k];
    // symmetrise the sums (their rounding may differ between (q, r) and (r, q))
    for (int q = 0; q < n2; ++q)
        for (int r = 0; r < q; ++r) {
            const double s = 0.5 * (D[(size_t)q * n2 + r] + D[(size_t)r * n2 + q]);
            D[(size_t)q * n2 + r] = D[(size_t)r * n2 + q] = s;
        }
    return dense_spd_inverse(std::move(D), n2, m.a2inv);
}

// ---------------------------------------------------------------------------
// Hierarchy of the general kernels.  The same matching passes and Galerkin
// products, applied to the whole matrix (the general kernels have no block
// ownership: a level's vectors live in global memory), within each system of
// a batch; as many levels as it takes to bring every system down to
// max_coarse rows.  Each level is stored like the fine one: 32-row slices,
// each system's rows padded to whole slices, the matrix in sliced ELLPACK.
// ---------------------------------------------------------------------------
bool gmg_build(const int *sptr, const int *scol, const double *sval, const double *dinv,
               int n_slices, int n_sys, const int *sys_slices, int passes0, int passes1,
               int max_coarse, int max_levels, GmgHost *out)
{
    *out = GmgHost{};
    if (n_sys < 1 || n_slices < 1)
        return false;
    const int n = 32 * n_slices;
    Csr cur = sell_to_csr(sptr, scol, sval, dinv, n_slices);
    std::vector<int> part((size_t)n, 0);
    for (int g = 0; g < n_sys; ++g)
        for (int i = 32 * sys_slices[g]; i < 32 * sys_slices[g + 1]; ++i)
            part[i] = g;
    // row of `cur` -> its row in the stored (padded) layout of its level
    std::vector<int> pad_of((size_t)n);
    for (int i = 0; i < n; ++i)
        pad_of[i] = i;
    int finer_rows = n;
    out->lev.resize(1);
    for (int l = 1; l <= max_levels; ++l) {
        std::vector<int> agg, cpart;
        Csr C = coarsen(cur, part, l == 1 ? passes0 : passes1, agg, cpart);
        // rows without entries (the fine level's padding) are aggregates of
        // their own: they belong to no aggregate, and are dropped
        std::vector<int> renum((size_t)C.n, -1);
        {
            std::vector<char> keep((size_t)C.n, 0);
            int live = 0;
            for (int i = 0; i < cur.n; ++i)
                if (cur.ptr[i + 1] > cur.ptr[i]) {
                    keep[agg[i]] = 1;
                    ++live;
                }
            int m = 0;
            for (int a = 0; a < C.n; ++a)
                if (keep[a])
                    renum[a] = m++;
            if (m < 1 || m >= live)
                return false;                       // nothing was aggregated
            if (m < C.n) {
                Csr B;
                B.n = m;
                B.ptr.assign((size_t)m + 1, 0);
                std::vector<int> bp((size_t)m);
                for (int a = 0; a < C.n; ++a) {
                    if (renum[a] < 0)
                        continue;
                    bp[renum[a]] = cpart[a];
                    for (int k = C.ptr[a]; k < C.ptr[a + 1]; ++k) {
                        B.col.push_back(renum[C.col[k]]);
                        B.val.push_back(C.val[k]);
                    }
                    B.ptr[renum[a] + 1] = (int)B.col.size();
                }
                C = std::move(B);
                cpart = std::move(bp);
            }
        }
        for (int a = 1; a < C.n; ++a)
            if (cpart[a] < cpart[a - 1])
                return false;                       // aggregates are numbered system by system
        GmgLevelHost L;
        std::vector<int> cnt((size_t)n_sys, 0), first((size_t)n_sys + 1, 0);
        for (int a = 0; a < C.n; ++a)
            cnt[cpart[a]] += 1;
        L.gsl.assign((size_t)n_sys + 1, 0);
        for (int g = 0; g < n_sys; ++g) {
            L.gsl[g + 1] = L.gsl[g] + (cnt[g] + 31) / 32;
            first[g + 1] = first[g] + cnt[g];
        }
        L.n_slices = L.gsl[n_sys];
        const int rows = 32 * L.n_slices;
        std::vector<int> pidx((size_t)C.n);
        for (int a = 0; a < C.n; ++a)
            pidx[a] = 32 * L.gsl[cpart[a]] + (a - first[cpart[a]]);
        // finer rows -> this level's rows, and the members of each row
        L.agg.assign((size_t)finer_rows, -1);
        for (int i = 0; i < cur.n; ++i)
            if (agg[i] >= 0 && renum[agg[i]] >= 0 && cur.ptr[i + 1] > cur.ptr[i])
                L.agg[pad_of[i]] = pidx[renum[agg[i]]];
        L.mptr.assign((size_t)rows + 1, 0);
        for (int p = 0; p < finer_rows; ++p)
            if (L.agg[p] >= 0)
                L.mptr[L.agg[p] + 1] += 1;
        for (int q = 0; q < rows; ++q)
            L.mptr[q + 1] += L.mptr[q];
        L.midx.assign((size_t)L.mptr[rows], 0);
        {
            std::vector<int> fill(L.mptr.begin(), L.mptr.end() - 1);
            for (int p = 0; p < finer_rows; ++p)
                if (L.agg[p] >= 0)
                    L.midx[fill[L.agg[p]]++] = p;
        }
        bool coarsest = true;
        for (int g = 0; g < n_sys; ++g)
            coarsest = coarsest && cnt[g] <= max_coarse;
        if (!coarsest) {
            // the level's matrix in sliced ELLPACK (padding entries: column
            // of the row itself, value 0), 1 / diagonal, Gershgorin bound
            std::vector<int> src((size_t)rows, -1);
            for (int a = 0; a < C.n; ++a)
                src[pidx[a]] = a;
            L.sptr.assign((size_t)L.n_slices + 1, 0);
            for (int sl = 0; sl < L.n_slices; ++sl) {
                int w = 0;
                for (int k = 0; k < 32; ++k) {
                    const int a = src[32 * sl + k];
                    if (a >= 0)
                        w = std::max(w, C.ptr[a + 1] - C.ptr[a]);
                }
                L.sptr[sl + 1] = L.sptr[sl] + 32 * w;
            }
            L.col.assign((size_t)L.sptr[L.n_slices], 0);
            L.val.assign((size_t)L.sptr[L.n_slices], 0.0);
            L.dinv.assign((size_t)rows, 0.0);
            for (int sl = 0; sl < L.n_slices; ++sl) {
                const int w = (L.sptr[sl + 1] - L.sptr[sl]) / 32;
                for (int k = 0; k < 32; ++k) {
                    const int q = 32 * sl + k, a = src[q];
                    const int len = a >= 0 ? C.ptr[a + 1] - C.ptr[a] : 0;
                    for (int c = 0; c < w; ++c) {
                        const size_t e = (size_t)L.sptr[sl] + (size_t)c * 32 + k;
                        if (c < len) {
                            const int kk = C.ptr[a] + c;
                            L.col[e] = pidx[C.col[kk]];
                            L.val[e] = C.val[kk];
                            if (C.col[kk] == a)
                                L.dinv[q] = C.val[kk] > 0.0 ? 1.0 / C.val[kk] : 0.0;
                        } else {
                            L.col[e] = q;
                        }
                    }
                    if (a >= 0 && !(L.dinv[q] > 0.0))
                        return false;
                }
            }
            L.lmax = gershgorin(C);
        }
        out->lev.push_back(std::move(L));
        if (coarsest) {
            // each system's coarsest matrix, inverted (systems in parallel)
            out->cn = cnt;
            out->ioff.assign((size_t)n_sys + 1, 0);
            for (int g = 0; g < n_sys; ++g)
                out->ioff[g + 1] = out->ioff[g] + (long long)cnt[g] * cnt[g];
            out->inv.assign((size_t)out->ioff[n_sys], 0.f);
            std::vector<char> ok((size_t)n_sys, 1);
            auto work = [&](int t, int nt) {
                for (int g = t; g < n_sys; g += nt) {
                    const int m = cnt[g], a0 = first[g];
                    if (m == 0)
                        continue;
                    std::vector<double> D((size_t)m * m, 0.0);
                    for (int a = a0; a < a0 + m; ++a)
                        for (int k = C.ptr[a]; k < C.ptr[a + 1]; ++k)
                            D[(size_t)(a - a0) * m + (C.col[k] - a0)] = C.val[k];
                    for (int q = 0; q < m; ++q)
                        for (int r = 0; r < q; ++r) {
                            const double v = 0.5 * (D[(size_t)q * m + r] + D[(size_t)r * m + q]);
                            D[(size_t)q * m + r] = D[(size_t)r * m + q] = v;
                        }
                    std::vector<float> inv;
                    if (!dense_spd_inverse(std::move(D), m, inv)) {
                        ok[g] = 0;
                        continue;
                    }
                    std::copy(inv.begin(), inv.end(), out->inv.begin() + out->ioff[g]);
                }
            };
            int nt = (int)std::thread::hardware_concurrency();
            nt = std::max(1, std::min(nt, std::min(n_sys, 32)));
            std::vector<std::thread> th;
            for (int t = 1; t < nt; ++t)
                th.emplace_back(work, t, nt);
            work(0, nt);
            for (auto &t : th)
                t.join();
            for (int g = 0; g < n_sys; ++g)
                if (!ok[g])
                    return false;
            return true;
        }
        cur = std::move(C);
        part = std::move(cpart);
        pad_of = std::move(pidx);
        finer_rows = rows;
    }
    return false;
}

}  // namespace pf
