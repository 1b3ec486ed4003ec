"""FP64 reference for the derivative of the collected charge with respect to
the applied field E0 and the per-face work functions phi_f, by reverse mode
over the PIC steps of Sec. II.B.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): imported by the tests
and never by the CUDA library or its binding.

The paper's cycle has discrete decisions (stochastically rounded SP counts,
eq. rnd_nsp; tetrahedron crossings and exits in the walk) that make the
collected charge piecewise constant in (E0, phi).  The derivative is that of
the smooth model obtained by freezing those decisions at the recorded run
(theta0) and letting the continuous quantities move:

* every SP injected in step k from quadrangle q carries the weight
  omega = n_sp,q(theta) / n_sp,q(theta0) (eq. nsp: n_sp is proportional to
  J_FN(F_q, phi_f) with F_q = -E_k(t_f).n_f), so the injected charge follows
  the emission current continuously; SPs present at the start have omega = 1;
* the number of SPs per quadrangle, the random numbers, every SP's cell at the
  start of a step, its fate in the walk (alive / collected / absorbed), its
  final cell and its periodic shifts are those of the recorded run;
* the kick, drift and emission velocity/displacement follow eqs. leapfrog1-3,
  sp_velocity and sp_displacement with the field of the frozen cell; the
  deposit is sum_p omega_p 2^S N_i(r_p) without the integer rounding; the
  potential is the exact solution of M Phi = f (eqs. poisson_mat, poisson_rhs)
  and the field E = -grad Phi (Sec. II.B.2);
* the objective is Q = q w_sp sum over collected SPs of omega (the charge that
  left through Gamma_1 over the run).

``record`` runs the oracle forward and keeps those decisions; ``replay``
evaluates the smooth model at any (E0, phi) (central finite differences of it
pin the reverse pass); ``gradient`` is the reverse pass, written out step by
step in the order of the forward one.  The run starts with a deposit and a
Poisson solve of the SPs present, so Phi_0 depends on E0 as well.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import oracle as O

ID_QUAD_SHIFT = 18
A_FN, B_FN, CS2 = 1.541434e-6, 6.830890, 1.439964   # Murphy-Good constants, nm units


def fn_dlog(F, phi, model=O.FN_MURPHY_GOOD):
    """(d ln J / dF, d ln J / dphi) of the emission current density of
    Sec. II.B.3 (J in the Murphy-Good form with Forbes' v(f), t(f), f clamped to
    1: where the clamp is active, v and t are constants).  F in V/m, phi in eV.
    From ln J = ln a + 2 ln F_n - ln phi - 2 ln t(f) - v(f) b phi^(3/2) / F_n,
    F_n = F 1e-9, f = c_S^2 F_n / phi^2."""
    F = np.asarray(F, np.float64)
    phi = np.asarray(phi, np.float64)
    Fn = F * 1e-9
    if model == O.FN_MURPHY_GOOD:
        f_raw = CS2 * Fn / (phi * phi)
        clamp = f_raw > 1.0
        f = np.minimum(f_raw, 1.0)
        lf = np.log(f)
        v = 1.0 - f + f / 6.0 * lf
        t = 1.0 + f / 9.0 - f / 18.0 * lf
        dv = np.where(clamp, 0.0, -1.0 + lf / 6.0 + 1.0 / 6.0)
        dt = np.where(clamp, 0.0, 1.0 / 9.0 - lf / 18.0 - 1.0 / 18.0)
        df_dFn = CS2 / (phi * phi)
        df_dphi = -2.0 * f_raw / phi
    else:
        v = t = np.ones_like(Fn)
        dv = dt = df_dFn = df_dphi = np.zeros_like(Fn)
    s = phi * np.sqrt(phi)
    dlnJ_dFn = 2.0 / Fn - 2.0 * dt / t * df_dFn - B_FN * s * (dv * df_dFn / Fn - v / (Fn * Fn))
    dlnJ_dphi = (-1.0 / phi - 2.0 * dt / t * df_dphi
                 - B_FN * (dv * df_dphi * s + v * 1.5 * np.sqrt(phi)) / Fn)
    return dlnJ_dFn * 1e-9, dlnJ_dphi


@dataclasses.dataclass
class Step:
    step: int
    n_old: int
    cell_pre: np.ndarray      # [n] cell at the start of the step (new SPs: face tetrahedron)
    quad: np.ndarray          # [n_new] quadrangle of each new SP
    R3: np.ndarray            # [n_new] the shared draw of eqs. sp_velocity / sp_displacement
    point: np.ndarray         # [n_new, 3] emission point on the quadrangle
    fate: np.ndarray          # [n] FATE_* after the walk
    cell_end: np.ndarray      # [n] cell after the walk
    shift: np.ndarray         # [n, 3] periodic shifts of the walk
    J_ref: np.ndarray = None  # [n_new] emission current of the smooth model at theta0


@dataclasses.dataclass
class Tape:
    params: dict
    E0: float
    wf: np.ndarray
    r0: np.ndarray            # SPs present at the start
    v0: np.ndarray
    cell0: np.ndarray
    steps: list
    Q_recorded: float


# systems up to this many free DOFs are factored once (sparse LU); larger ones
# (the 1M-tet tip: a factor of ~600M entries) are solved by the oracle's own
# Jacobi-PCG to a relative residual of 1e-13 at every solve
LU_MAX_ROWS = 60_000
CG_RTOL = 1e-13


class Geometry:
    """P1 data of the oracle's mesh in numpy form.  direct: True factor M,
    False solve iteratively, None by size (LU_MAX_ROWS)."""

    def __init__(self, orc, direct=None):
        m = orc.mesh
        self.tet = m.tet.astype(np.int64)
        jinv, x0, _ = orc.geometry()
        self.jinv = jinv.reshape(-1, 3, 3)            # rows: grad N_1..3
        self.x0 = x0
        self.grad = np.concatenate([-self.jinv.sum(axis=1, keepdims=True), self.jinv], axis=1)
        dof, rowptr, col, val, fN = orc.matrix()
        self.dof = dof.astype(np.int64)               # -1 on Dirichlet nodes
        n = len(rowptr) - 1
        self.M = sp.csr_matrix((val, col, rowptr), shape=(n, n)).tocsc()
        self.direct = n <= LU_MAX_ROWS if direct is None else bool(direct)
        self.orc = orc
        self.lu = spla.splu(self.M) if self.direct else None
        self.fN_unit = fN / orc.params["E0"]          # Neumann load per unit E0
        xyz = m.xyz
        A, B, Cc = (xyz[m.face_nodes[:, k]] for k in range(3))
        nrm = np.cross(B - A, Cc - A)
        self.nhat = nrm / np.linalg.norm(nrm, axis=1, keepdims=True)
        self.face_tet = m.face_tet.astype(np.int64)
        self.n_nodes = m.n_nodes
        self.free = self.dof >= 0

    def msolve(self, f):
        """M^-1 f (M symmetric: the forward and the adjoint solves alike)"""
        if self.direct:
            return self.lu.solve(f)
        return self.orc.solve(f, rtol=CG_RTOL)

    def lam(self, cell, r):
        """barycentric coordinates N_0..N_3 of points r in tetrahedra cell"""
        l123 = np.einsum("nij,nj->ni", self.jinv[cell], r - self.x0[cell])
        return np.concatenate([1.0 - l123.sum(axis=1, keepdims=True), l123], axis=1)

    def deposit(self, cell, r, w, S):
        W = np.zeros(self.n_nodes)
        np.add.at(W, self.tet[cell], (w[:, None] * self.lam(cell, r)) * 2.0 ** S)
        return W

    def solve(self, W, E0, p):
        coef = p["q"] * p["w_sp"] / p["eps0"]
        f = coef * W[self.free] * 2.0 ** -p["quant_bits"] + E0 * self.fN_unit[self.dof[self.free]]
        phi = np.zeros(self.n_nodes)
        phi[self.free] = self.msolve(f)[self.dof[self.free]]
        return phi

    def field(self, phi):
        return -np.einsum("ti,tic->tc", phi[self.tet], self.grad)

    def field_adjoint(self, Ebar):
        """Phi_bar_i = d(sum_t Ebar_t . E_t)/d Phi_i"""
        pb = np.zeros(self.n_nodes)
        np.add.at(pb, self.tet, -np.einsum("tc,tic->ti", Ebar, self.grad))
        return pb

    def solve_adjoint(self, phibar):
        """f_bar = M^-1 Phi_bar on the free DOFs (M is symmetric), node indexed"""
        fb = np.zeros(self.n_nodes)
        rhs = np.zeros(self.M.shape[0])
        rhs[self.dof[self.free]] = phibar[self.free]
        fb[self.free] = self.msolve(rhs)[self.dof[self.free]]
        return fb


def record(orc, n_steps) -> Tape:
    """Run the oracle n_steps from its current SPs (deposit and solve first) and
    keep the discrete decisions of every step."""
    p = orc.params
    qmdt, dt = p["q_over_m"] * p["dt"], p["dt"]
    r0, v0, cell0, _ = orc.particles()
    orc.deposit()
    orc.poisson_solve()
    steps, n_col = [], 0
    for _ in range(n_steps):
        s = orc.step_index
        E = orc.field()
        _, _, _, pid_pre = orc.particles()
        n_old = len(pid_pre)
        orc.inject(s)
        r, v, cell, pid = orc.particles()
        new = pid[n_old:]
        quad = (new >> ID_QUAD_SHIFT) & ((1 << 24) - 1)
        j = new & ((1 << ID_QUAD_SHIFT) - 1)
        R3 = np.array([O.uniform(p["seed"], s, int(q), int(jj), 255) for q, jj in zip(quad, j)])
        point = r[n_old:] - v[n_old:] * (dt * R3)[:, None]
        # the drift of the push, to classify the SPs the walk removes
        vv = v.copy()
        vv[:n_old] = v[:n_old] + qmdt * E[cell[:n_old]]
        rr = r + dt * vv
        r_end, c_end, fate, _ = orc.locate(rr, cell)
        orc.push_relocate(s)
        r_post, _, c_post, pid_post = orc.particles()
        alive = fate == O.FATE_ALIVE
        assert np.array_equal(pid_post, pid[alive]) and np.array_equal(c_post, c_end[alive])
        assert np.array_equal(r_post, r_end[alive])
        n_col += int((fate == O.FATE_COLLECTED).sum())
        steps.append(Step(step=s, n_old=n_old, cell_pre=cell.copy(), quad=quad, R3=R3,
                          point=point, fate=fate, cell_end=c_end, shift=r_end - rr))
        orc.deposit()
        orc.poisson_solve()
        orc.step_index = s + 1
    return Tape(params=dict(p), E0=p["E0"], wf=orc.mesh.work_function.copy(), r0=r0, v0=v0,
                cell0=cell0, steps=steps, Q_recorded=p["q"] * p["w_sp"] * n_col)


def _emission(g, tape, E, wf, st):
    """F, J of the faces of the new SPs of a step"""
    f = st.quad // 3
    F = -np.einsum("nc,nc->n", E[g.face_tet[f]], g.nhat[f])
    model = tape.params["fn_model"]
    J = np.array([O.fn_current(a, b, model) for a, b in zip(F, wf[f])])
    return f, F, J


def replay(g, tape, E0, wf, keep=False):
    """Collected charge of the frozen-decision model at (E0, wf); with keep,
    also the per-step quantities the reverse pass needs."""
    p = tape.params
    S, qmdt, dt = p["quant_bits"], p["q_over_m"] * p["dt"], p["dt"]
    r, v, cell = tape.r0.copy(), tape.v0.copy(), tape.cell0.copy()
    w = np.ones(len(cell))
    phi = g.solve(g.deposit(cell, r, w, S), E0, p)
    E = g.field(phi)
    Q, saved = 0.0, []
    for st in tape.steps:
        n_old = st.n_old
        f, F, J = _emission(g, tape, E, wf, st)
        w_new = J / st.J_ref if st.J_ref is not None else np.ones(len(J))
        v_new = (qmdt * (0.5 + st.R3))[:, None] * E[g.face_tet[f]]
        r_new = st.point + v_new * (dt * st.R3)[:, None]
        v1 = np.concatenate([v + qmdt * E[st.cell_pre[:n_old]], v_new])
        r1 = np.concatenate([r, r_new]) + dt * v1
        r_end = r1 + st.shift
        w1 = np.concatenate([w, w_new])
        Q += p["q"] * p["w_sp"] * w1[st.fate == O.FATE_COLLECTED].sum()
        alive = st.fate == O.FATE_ALIVE
        if st.J_ref is None:
            st.J_ref = J                 # the pass at theta0 that defines omega = 1
        saved.append(dict(E=E, F=F, w1=w1, r_end=r_end) if keep else None)
        r, v, w, cell = r_end[alive], v1[alive], w1[alive], st.cell_end[alive]
        phi = g.solve(g.deposit(cell, r, w, S), E0, p)
        E = g.field(phi)
    return (Q, saved) if keep else Q


def prepare(orc, tape, direct=None):
    """Geometry of the oracle's mesh, and one pass of the smooth model at
    theta0 that fixes the reference emission currents (omega = 1 there)."""
    g = Geometry(orc, direct)
    for st in tape.steps:
        st.J_ref = None
    replay(g, tape, tape.E0, tape.wf)
    return g


def gradient(g, tape):
    """(Q, dQ/dE0, dQ/dphi_f) of the frozen-decision model at theta0, by the
    reverse pass of ``replay``."""
    p = tape.params
    S, qmdt, dt = p["quant_bits"], p["q_over_m"] * p["dt"], p["dt"]
    qw = p["q"] * p["w_sp"]
    Q, saved = replay(g, tape, tape.E0, tape.wf, keep=True)
    coef = p["q"] * p["w_sp"] / p["eps0"]
    gE0 = 0.0
    gwf = np.zeros(len(tape.wf))
    # adjoints of the state after the last step
    rb = vb = wb = None
    Ebar_next = np.zeros((len(g.tet), 3))
    for k in range(len(tape.steps) - 1, -1, -1):
        st, sv = tape.steps[k], saved[k]
        n_old, n = st.n_old, len(st.fate)
        alive = st.fate == O.FATE_ALIVE
        # E_{k+1} = field(Phi_{k+1}), Phi_{k+1} = M^-1 f(W_{k+1}, E0)
        fb = g.solve_adjoint(g.field_adjoint(Ebar_next))
        gE0 += float(fb[g.free] @ g.fN_unit[g.dof[g.free]])
        Wb = coef * 2.0 ** -S * fb
        # adjoints of this step's SPs after the walk
        r1b, v1b, w1b = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
        if rb is not None:
            r1b[alive], v1b[alive], w1b[alive] = rb, vb, wb
        # deposit W_{k+1} = sum_alive w 2^S N(r_end)
        ce, re = st.cell_end[alive], sv["r_end"][alive]
        lam = g.lam(ce, re)
        Wn = Wb[g.tet[ce]]                                   # [n_alive, 4]
        w1b[alive] += 2.0 ** S * (Wn * lam).sum(axis=1)
        r1b[alive] += (sv["w1"][alive] * 2.0 ** S)[:, None] * np.einsum("ni,nic->nc", Wn, g.grad[ce])
        # objective
        col = st.fate == O.FATE_COLLECTED
        w1b[col] += qw
        # drift r1 = r + dt v1 (+ constant shift)
        v1b = v1b + dt * r1b
        Ebar = np.zeros((len(g.tet), 3))
        # kick of the old SPs
        np.add.at(Ebar, st.cell_pre[:n_old], qmdt * v1b[:n_old])
        # emission of the new SPs: r_new = point + v_new dt R3, v_new = qmdt (1/2 + R3) E(t_f)
        f = st.quad // 3
        vnb = v1b[n_old:] + (dt * st.R3)[:, None] * r1b[n_old:]
        np.add.at(Ebar, g.face_tet[f], (qmdt * (0.5 + st.R3))[:, None] * vnb)
        # weights of the new SPs: w = J(F, phi_f) / J(theta0)
        dF, dphi = fn_dlog(sv["F"], tape.wf[f], p["fn_model"])
        wnb = w1b[n_old:]
        np.add.at(gwf, f, wnb * dphi)
        Fb = wnb * dF
        np.add.at(Ebar, g.face_tet[f], -Fb[:, None] * g.nhat[f])
        # state before the step: the old SPs in order
        rb, vb, wb = r1b[:n_old], v1b[:n_old], w1b[:n_old]
        Ebar_next = Ebar
    # Phi_0 = M^-1 f(W_0, E0)
    fb = g.solve_adjoint(g.field_adjoint(Ebar_next))
    gE0 += float(fb[g.free] @ g.fN_unit[g.dof[g.free]])
    return Q, gE0, gwf
