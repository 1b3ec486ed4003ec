"""Pins of the oracle's reverse-mode derivative of the collected charge
(oracle/adjoint.py): the FN log-derivatives against finite differences of the
oracle's emission current; the smooth frozen-decision model at theta0 against
the recorded run; the reverse pass against central finite differences of the
smooth model (dQ/dE0, a random direction in the work functions, single
faces); and, without space charge, against the closed form
dQ/dphi_f = q w_sp sum_{collected SPs of face f} d ln J / d phi."""
import numpy as np
import pytest

from paper_1906_08125_gb300 import configs as K
from paper_1906_08125_gb300 import inputs

from oracle import adjoint as A
from oracle import oracle as O


@pytest.mark.parametrize("model", [O.FN_MURPHY_GOOD, O.FN_ELEMENTARY])
def test_fn_dlog_matches_finite_differences(model):
    for F in (2e9, 5e9, 1e10, 2e10, 4e10):
        for phi in (3.0, 4.5, 5.5):
            dF, dphi = A.fn_dlog(F, phi, model)
            lnJ = lambda a, b: np.log(O.fn_current(a, b, model))
            h = 1e-6
            fdF = (lnJ(F * (1 + h), phi) - lnJ(F * (1 - h), phi)) / (2 * h * F)
            fdp = (lnJ(F, phi * (1 + h)) - lnJ(F, phi * (1 - h))) / (2 * h * phi)
            assert abs(dF - fdF) <= 1e-6 * abs(fdF) + 1e-16, (F, phi)
            assert abs(dphi - fdp) <= 1e-6 * abs(fdp), (F, phi)


def small_run(n_steps=6, eps0=K.EPS0, w_sp=0.02, seed=1):
    mesh = inputs.plate_mesh(nx=4, ny=4, nz=8, lx=20e-9, ly=20e-9, lz=40e-9,
                             work_function=4.5, name="plate_tiny")
    mesh.work_function = 4.5 + 0.2 * np.random.default_rng(5).uniform(-1, 1, mesh.n_faces)
    p = K.params(E0=1e10, w_sp=w_sp, pcg_rtol=1e-13, pcg_max_iter=50000, capacity=200_000,
                 seed=seed)
    p["eps0"] = eps0
    orc = O.Oracle(mesh, p)
    parts = inputs.random_particles(mesh, 300, seed=seed, v_scale=2e6, v_up=4e6)
    orc.set_particles(*parts)
    tape = A.record(orc, n_steps)
    g = A.prepare(orc, tape)
    return mesh, p, tape, g


@pytest.fixture(scope="module")
def run():
    return small_run()


def test_replay_at_theta0_is_the_recorded_run(run):
    mesh, p, tape, g = run
    n_col = sum(int((st.fate == O.FATE_COLLECTED).sum()) for st in tape.steps)
    n_new = sum(len(st.quad) for st in tape.steps)
    assert n_col > 20 and n_new > 20
    Q = A.replay(g, tape, tape.E0, tape.wf)
    assert Q == pytest.approx(tape.Q_recorded, rel=1e-13)


def test_iterative_solves_match_the_factorisation(run):
    """The reverse pass with the oracle's own Jacobi-PCG at every solve (the
    path meshes above LU_MAX_ROWS take) gives the collected charge and the
    gradient of the factored path."""
    mesh, p, tape, g = run
    Q1, gE1, gw1 = A.gradient(g, tape)
    g2 = A.prepare(g.orc, tape, direct=False)
    assert g.direct and not g2.direct
    Q2, gE2, gw2 = A.gradient(g2, tape)
    assert Q2 == pytest.approx(Q1, rel=1e-11)
    assert gE2 == pytest.approx(gE1, rel=1e-9)
    assert np.abs(gw2 - gw1).max() <= 1e-9 * np.abs(gw1).max()
    assert A.replay(g2, tape, tape.E0 * 1.01, tape.wf) == pytest.approx(
        A.replay(g, tape, tape.E0 * 1.01, tape.wf), rel=1e-11)


def test_gradient_matches_central_differences(run):
    mesh, p, tape, g = run
    Q, gE0, gwf = A.gradient(g, tape)
    h = 1e-6
    fd = (A.replay(g, tape, tape.E0 * (1 + h), tape.wf)
          - A.replay(g, tape, tape.E0 * (1 - h), tape.wf)) / (2 * h * tape.E0)
    assert gE0 == pytest.approx(fd, rel=1e-5)
    d = np.random.default_rng(3).normal(size=len(tape.wf))
    hw = 1e-6
    fdw = (A.replay(g, tape, tape.E0, tape.wf + hw * d)
           - A.replay(g, tape, tape.E0, tape.wf - hw * d)) / (2 * hw)
    assert float(gwf @ d) == pytest.approx(fdw, rel=1e-5)
    for f in np.argsort(-np.abs(gwf))[:3]:
        e = np.zeros(len(tape.wf))
        e[f] = 1.0
        fdf = (A.replay(g, tape, tape.E0, tape.wf + hw * e)
               - A.replay(g, tape, tape.E0, tape.wf - hw * e)) / (2 * hw)
        assert gwf[f] == pytest.approx(fdf, rel=1e-5, abs=1e-9 * np.abs(gwf).max())


def test_gradient_closed_form_without_space_charge():
    """With the space-charge term switched off (eps0 huge) the field is
    E0 times a fixed pattern, so only the emission weights depend on theta:
    dQ/dphi_f = q w_sp sum_p dlnJ/dphi, dQ/dE0 = q w_sp sum_p dlnJ/dF F_p / E0
    over the collected SPs p injected from face f."""
    mesh, p, tape, g = small_run(eps0=1e30)
    Q, gE0, gwf = A.gradient(g, tape)
    qw = p["q"] * p["w_sp"]
    want_wf = np.zeros(len(tape.wf))
    want_E0 = 0.0
    _, saved = A.replay(g, tape, tape.E0, tape.wf, keep=True)
    # follow every SP from its emission (face, d ln J) to its exit
    face = np.full(len(tape.cell0), -1)
    lnJ_F, lnJ_phi = np.zeros(len(face)), np.zeros(len(face))
    for st, sv in zip(tape.steps, saved):
        f = st.quad // 3
        dF, dphi = A.fn_dlog(sv["F"], tape.wf[f], p["fn_model"])
        face = np.concatenate([face, f])
        lnJ_F = np.concatenate([lnJ_F, dF * sv["F"] / tape.E0])
        lnJ_phi = np.concatenate([lnJ_phi, dphi])
        col = (st.fate == O.FATE_COLLECTED) & (face >= 0)
        np.add.at(want_wf, face[col], qw * lnJ_phi[col])
        want_E0 += qw * float(lnJ_F[col].sum())
        alive = st.fate == O.FATE_ALIVE
        face, lnJ_F, lnJ_phi = face[alive], lnJ_F[alive], lnJ_phi[alive]
    assert np.abs(want_wf).max() > 0
    assert np.allclose(gwf, want_wf, rtol=1e-9, atol=1e-12 * np.abs(want_wf).max())
    assert gE0 == pytest.approx(want_E0, rel=1e-6)
