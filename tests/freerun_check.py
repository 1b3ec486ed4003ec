"""Free-running comparison of two PIC runs of the same mesh (the FP32+IR CUDA
path against the FP64 oracle) in which every difference must be explained.

Two correct runs that round differently can part ways in three discrete
places, and only there (Sec. II.B):

* injection (eq. rnd_nsp): the count of a quadrangle is ceil(n_sp - R0) with
  n_sp proportional to J_FN(F), so when the two fields give n_sp values that
  bracket an integer + R0, one run emits one more SP there.  An SP present
  in one run only and injected in step k is explained when its index j lies
  in [ceil(n_lo - R0), ceil(n_hi - R0)) for the two runs' n_sp of its
  quadrangle in that step (a relative slack of 1e-12 covers the rounding of
  exp/log between the two math libraries);
* location (the walk): when an SP ends a step on or within rounding of a
  face, the two runs may give it different, equally valid cells; from the
  next kick on it sees another (piecewise constant) field and its
  trajectory legitimately differs.  Such an SP is explained at the first
  step its cells differ if its positions then still agree to the position
  tolerance and each run's position lies within that distance (plus FP32
  rounding) of the other run's cell;
* exits: an SP within the position tolerance of Gamma_1 or Gamma_3 may leave
  one step earlier in one run; the survivor must lie within the tolerance
  of such a face.
* the periodic sides: an SP on (within rounding of) Gamma_2 may be wrapped
  in one run and not in the other; its positions then agree on the nearest
  periodic image, but it sits at the opposite side of the box, where its
  charge goes to other nodes (the field mesh is not periodic: zero-Neumann
  sides), so the potentials of the two runs differ near both sides.

Everything else is held to the bar: an SP whose cells have agreed at every
step must have its position within the tolerance (1e-5 of the box height)
at every step, and every id must be common to both runs unless explained as
above.  Periodic sides: position differences and cell tests are taken on the
periodic image nearest to the other run's position.

Pure numpy / scipy on the host (plus the oracle's emission numbers for a
given field); used by the GPU parity tests and pinned on the CPU against
oracle runs with planted mistakes."""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree

from oracle import oracle as O

ID_STEP_SHIFT = 42
ID_QUAD_SHIFT = 18
ID_POPULATION_BIT = 62          # ids of a given starting population
TOP, CATHODE = -1, -2
_FACE_LOCAL = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])


def injection_step(pid):
    pid = np.asarray(pid, np.int64)
    fresh = (pid >> np.int64(ID_POPULATION_BIT)) == 0
    return np.where(fresh, pid >> np.int64(ID_STEP_SHIFT), -1)


def count_of(n_sp, R0):
    """The rounded count of eq. rnd_nsp: floor(n) + (R0 < frac(n)), which is
    ceil(n - R0) for R0 in [0, 1)."""
    return np.ceil(np.asarray(n_sp) - np.asarray(R0)).astype(np.int64)


def injection_flip_explained(n_a, n_b, R0, j, rel=1e-12):
    """True where index j exists in one reading of the count but not in the
    other, for n_sp between n_a and n_b (widened by `rel`)."""
    lo = np.minimum(n_a, n_b) * (1.0 - rel)
    hi = np.maximum(n_a, n_b) * (1.0 + rel)
    return (count_of(lo, R0) <= j) & (j < count_of(hi, R0))


def point_triangle_distance(p, a, b, c):
    """Euclidean distance from points p[n,3] to triangles (a, b, c)[n,3]."""
    ab, ac = b - a, c - a
    nrm = np.cross(ab, ac)
    nn = np.einsum("ij,ij->i", nrm, nrm)
    ap = p - a
    # barycentric coordinates of the projection
    d00 = np.einsum("ij,ij->i", ab, ab)
    d01 = np.einsum("ij,ij->i", ab, ac)
    d11 = np.einsum("ij,ij->i", ac, ac)
    d20 = np.einsum("ij,ij->i", ap, ab)
    d21 = np.einsum("ij,ij->i", ap, ac)
    den = d00 * d11 - d01 * d01
    v = (d11 * d20 - d01 * d21) / den
    w = (d00 * d21 - d01 * d20) / den
    inside = (v >= 0) & (w >= 0) & (v + w <= 1)
    plane = np.abs(np.einsum("ij,ij->i", ap, nrm)) / np.sqrt(nn)

    def seg(p, x, y):
        d = y - x
        t = np.clip(np.einsum("ij,ij->i", p - x, d) / np.einsum("ij,ij->i", d, d), 0.0, 1.0)
        return np.linalg.norm(p - (x + t[:, None] * d), axis=1)

    edge = np.minimum(np.minimum(seg(p, a, b), seg(p, b, c)), seg(p, c, a))
    return np.where(inside, plane, edge)


def _by_id(state):
    r, v, cell, pid = state
    o = np.argsort(pid, kind="stable")
    return r[o], v[o], cell[o], pid[o]


class FreeRunCheck:
    """Accumulates the step-by-step comparison of run G (checked) against run
    O (the reference); `failures` lists what no rule explains."""

    def __init__(self, mesh, orc, seed, tol_rel=1e-5, fp32_positions=True):
        self.mesh, self.orc, self.seed = mesh, orc, int(seed)
        lo, hi = np.asarray(mesh.box_lo, float), np.asarray(mesh.box_hi, float)
        self.L = hi - lo
        self.tol = tol_rel * self.L[2]
        # rounding of a stored FP32 coordinate of the box: two units in the
        # last place at its largest magnitude (FP64 runs: far smaller)
        big = np.abs(np.concatenate([lo, hi])).max()
        self.eps = (2.0 ** -22 if fp32_positions else 2.0 ** -48) * big
        P = mesh.xyz[mesh.tet]
        J = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], axis=2)
        self.Jinv = np.linalg.inv(J)
        g = np.concatenate([-self.Jinv.sum(axis=1, keepdims=True), self.Jinv], axis=1)
        self.gnorm = np.linalg.norm(g, axis=2)          # |grad lambda_i|
        self.x0 = P[:, 0]
        tt, kk = np.nonzero((mesh.nbr == TOP) | (mesh.nbr == CATHODE))
        tri = mesh.xyz[mesh.tet[tt[:, None], _FACE_LOCAL[kk]]]   # (F, 3, 3)
        self.tri = tri
        self.tree = cKDTree(tri.mean(axis=1))
        self.prev_common = np.zeros(0, np.int64)
        self.diverged, self.flipped, self.exited = {}, {}, {}
        self.failures = []
        self.max_err_clean = 0.0
        self.steps = 0
        self.checked = 0
        self.divergence_gap = []       # |r_G - r_O| at each explained cell divergence
        self.divergence_excess = []    # distance of each position from the other cell
        # the first step after which the runs hold different SPs (an
        # injection rounding flip or an exit one step apart) or an SP on
        # different periodic images: from then on the space charge of the
        # two runs differs by whole SPs
        self.first_event = None
        self.image_flips = {}          # id -> step its runs took different images

    # geometry ----------------------------------------------------------------
    def lam(self, cell, r):
        l = np.einsum("nij,nj->ni", self.Jinv[cell], r - self.x0[cell])
        return np.concatenate([1.0 - l.sum(axis=1, keepdims=True), l], axis=1)

    def excess(self, cell, r):
        """Largest distance of r beyond one of the face planes of `cell`
        (0 inside): a lower bound of the distance from r to the cell."""
        return np.maximum(0.0, (-self.lam(cell, r) / self.gnorm[cell]).max(axis=1))

    def nearest_image(self, r, ref):
        """r moved by whole periods in x, y to the image nearest ref."""
        s = np.zeros_like(r)
        s[:, :2] = self.L[:2] * np.round((ref[:, :2] - r[:, :2]) / self.L[:2])
        return r + s

    def boundary_distance(self, r, k=16):
        _, idx = self.tree.query(r, k=min(k, len(self.tri)))
        idx = np.atleast_2d(idx)
        best = np.full(len(r), np.inf)
        for c in range(idx.shape[1]):
            t = self.tri[idx[:, c]]
            best = np.minimum(best, point_triangle_distance(r, t[:, 0], t[:, 1], t[:, 2]))
        return best

    @staticmethod
    def _ids(d):
        return np.fromiter(d.keys(), np.int64, len(d))

    def _fail(self, k, what, ids):
        ids = np.atleast_1d(ids)
        if len(ids):
            self.failures.append((k, what, int(len(ids)), [int(x) for x in ids[:5]]))

    # one step ------------------------------------------------------------------
    def step(self, k, g, o, E_g, E_o):
        """g, o: (r, v, cell, id) of both runs after step k; E_g, E_o: their
        fields at the start of step k (the fields the injection used)."""
        g, o = _by_id(g), _by_id(o)
        rg, _, cg, ig = g
        ro, _, co, io = o
        self.steps += 1
        # every SP of G lies in its cell (within the rounding of its position)
        out = self.excess(cg, rg) > self.eps
        self._fail(k, "position outside its cell", ig[out])
        common, a, b = np.intersect1d(ig, io, assume_unique=True, return_indices=True)
        self.checked += len(common)
        r_g, r_o = rg[a], self.nearest_image(ro[b], rg[a])
        img = np.any(r_o != ro[b], axis=1)
        new_img = img & ~np.isin(common, self._ids(self.image_flips))
        for x in common[new_img]:
            self.image_flips[int(x)] = k
        if new_img.any() and self.first_event is None:
            self.first_event = k
        gap = np.abs(r_g - r_o).max(axis=1)
        clean = ~np.isin(common, self._ids(self.diverged))
        same = cg[a] == co[b]
        if (clean & same).any():
            self.max_err_clean = max(self.max_err_clean, float(gap[clean & same].max()))
        self._fail(k, "cells agree but position beyond tolerance",
                   common[clean & same & (gap > self.tol)])
        new_div = clean & ~same
        if new_div.any():
            d2 = np.linalg.norm(r_g[new_div] - r_o[new_div], axis=1)
            # each position against the other run's cell, on the periodic
            # image nearest that run's own position
            r_g_at_o = self.nearest_image(r_g[new_div], ro[b][new_div])
            e1 = self.excess(co[b][new_div], r_g_at_o)
            e2 = self.excess(cg[a][new_div], r_o[new_div])
            ok = (gap[new_div] <= self.tol) & (e1 <= d2 + self.eps) & (e2 <= d2 + self.eps)
            ids = common[new_div]
            self._fail(k, "cells differ with positions apart", ids[~ok])
            for x in ids[ok]:
                self.diverged[int(x)] = k
            self.divergence_gap += list(d2[ok])
            self.divergence_excess += list(np.maximum(e1, e2)[ok])
        # ids of one run only
        only_g = np.setdiff1d(ig, io, assume_unique=True)
        only_o = np.setdiff1d(io, ig, assume_unique=True)
        need_emission = True
        n_g = n_o = None
        for side, ids, r_side, id_side in (("G", only_g, rg, ig), ("O", only_o, ro, io)):
            if not len(ids):
                continue
            known = (np.isin(ids, self._ids(self.diverged)) | np.isin(ids, self._ids(self.flipped))
                     | np.isin(ids, self._ids(self.exited)))
            ids = ids[~known]
            if not len(ids):
                continue
            born = injection_step(ids) == k
            if born.any():
                if need_emission:
                    n_g = self.orc.quad_emission(E_g)[2]
                    n_o = self.orc.quad_emission(E_o)[2]
                    need_emission = False
                nb = ids[born]
                q = (nb >> np.int64(ID_QUAD_SHIFT)) & np.int64((1 << 24) - 1)
                j = nb & np.int64((1 << ID_QUAD_SHIFT) - 1)
                R0 = np.array([O.uniform(self.seed, k, int(qq), 0, 0) for qq in q])
                ok = injection_flip_explained(n_g[q], n_o[q], R0, j)
                for x in nb[ok]:
                    self.flipped[int(x)] = k
                # injected in both, but left the other run within its first
                # step (an exit one step apart, below)
                rest = nb[~ok]
                if len(rest):
                    pos = r_side[np.searchsorted(id_side, rest)]
                    near = self.boundary_distance(pos) <= self.tol + self.eps
                    self._fail(k, f"injected in run {side} only, not a rounding flip",
                               rest[~near])
                    for x in rest[near]:
                        self.exited[int(x)] = k
            old = ids[~born]
            if len(old):
                was_common = np.isin(old, self.prev_common, assume_unique=True)
                self._fail(k, f"id of run {side} only, never common", old[~was_common])
                old = old[was_common]
                if len(old):
                    pos = r_side[np.searchsorted(id_side, old)]
                    near = self.boundary_distance(pos) <= self.tol + self.eps
                    self._fail(k, f"left run {'O' if side == 'G' else 'G'} away from Gamma_1/3",
                               old[~near])
                    for x in old[near]:
                        self.exited[int(x)] = k
        self.prev_common = common
        if self.first_event is None and (len(only_g) or len(only_o)):
            self.first_event = k

    def summary(self):
        return {"steps": self.steps, "sp_steps_checked": self.checked,
                "cell_divergences": len(self.diverged), "injection_flips": len(self.flipped),
                "exit_timing": len(self.exited), "max_err_clean_rel": self.max_err_clean / self.L[2],
                "max_gap_at_divergence_rel": (max(self.divergence_gap) / self.L[2]
                                              if self.divergence_gap else 0.0),
                "first_event_step": self.first_event,
                "image_flips": len(self.image_flips),
                "failures": self.failures[:10]}
