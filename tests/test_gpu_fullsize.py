"""Parity at full size: the 1M-tetrahedron tip workload in the configuration
the benchmark times (FP32 push, FP32 Chebyshev-PCG inside FP64 refinement,
fused pic_step), against the FP64 oracle on sampled outputs: a seeded
population of 2e5 SPs (the oracle handles it in seconds) stepped once from
identical state, and the potentials of the charge-free and space-charge
solves.  Also the FP64 split path at full size, bit for bit."""
import os

import numpy as np
import pytest

from paper_1906_08125_gb300 import configs as K
from paper_1906_08125_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N_SAMPLE = 200_000


@pytest.fixture(scope="module")
def picfem():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_08125_gb300 import picfem as P
    P.load()
    return P


@pytest.fixture(scope="module")
def tip1m():
    mesh, p, _ = K.workload("tip_1m")
    return mesh, p


@pytest.fixture(scope="module")
def oracle_state(oracle_mod, tip1m):
    """Oracle with the charge-free potential solved tightly, then the seeded
    sample population deposited and its potential solved tightly."""
    mesh, p = tip1m
    orc = oracle_mod.Oracle(mesh, dict(p, precision=K.PREC_FP64, pcg_rtol=1e-11,
                                       pcg_max_iter=50000), parallel=True)
    orc.init_potential()
    phi0 = orc.potential()
    parts = inputs.random_particles(mesh, N_SAMPLE, seed=77, v_scale=3e6, v_up=1.5e7)
    orc.set_particles(*parts)
    orc.deposit()
    orc.poisson_solve()
    return orc, phi0, parts


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def by_id(state):
    r, v, cell, pid = state
    o = np.argsort(pid, kind="stable")
    return r[o], v[o], cell[o], pid[o]


def bary(mesh, cell, r):
    P = mesh.xyz[mesh.tet[cell]]
    J = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], axis=2)
    lam = np.linalg.solve(J, (r - P[:, 0])[..., None])[..., 0]
    return np.concatenate([1 - lam.sum(1, keepdims=True), lam], axis=1)


def test_potentials_at_bench_tolerance(picfem, tip1m, oracle_state):
    """The GPU forms (FP32_IR with the standard and the merged inner solver,
    plain FP64), at the solver tolerance the benchmark uses, reach 1e-6
    relative potential accuracy against the oracle's tight solve."""
    mesh, p = tip1m
    orc, phi0, parts = oracle_state
    for form in ({}, {"pcg_variant": K.PCG_MERGED},
                 {"precision": K.PREC_FP64, "pcg_cheb_degree": 0}):
        ctx = picfem.Context(dict(p, **form)).mesh_load(mesh)
        ctx.init_potential()
        e0 = rel(ctx.potential(), phi0)
        ctx.set_particles(*parts)
        ctx.deposit()
        ctx.set_potential(phi0)
        ctx.poisson_solve()
        e1 = rel(ctx.potential(), orc.potential())
        ctx.close()
        assert e0 <= 1e-6 and e1 <= 1e-6, (form, e0, e1)


def test_one_bench_step_fp32ir(picfem, oracle_mod, tip1m, oracle_state):
    """One fused step in the benchmark's configuration from identical state
    (the oracle's tight potential and the seeded sample): same SP ids up to
    rounding flips of the injection count, positions within 1e-5 of the box
    height, differing cells only within FP32 rounding of a face, exact charge
    conservation, and the new potential within 1e-6."""
    mesh, p = tip1m
    orc, phi0, parts = oracle_state
    phi_start = orc.potential()
    o2 = oracle_mod.Oracle(mesh, dict(p, precision=K.PREC_FP64, pcg_rtol=1e-11,
                                      pcg_max_iter=50000), parallel=True)
    o2.set_potential(phi_start)
    o2.set_particles(*parts)
    o2.step_index = 5
    so = o2.step(1)[0]

    ctx = picfem.Context(p).mesh_load(mesh)
    ctx.set_potential(phi_start)
    ctx.set_particles(*parts)
    ctx.step_index = 5
    sg = ctx.step(1)[0]

    g, o = by_id(ctx.particles()), by_id(o2.particles())
    common, ig, io = np.intersect1d(g[3], o[3], return_indices=True)
    assert len(common) >= len(o[3]) - 10 and len(common) >= len(g[3]) - 10
    Lz = mesh.box_hi[2] - mesh.box_lo[2]
    assert np.abs(g[0][ig] - o[0][io]).max() <= 1e-5 * Lz
    diff = g[2][ig] != o[2][io]
    assert diff.mean() <= 1e-3
    if diff.any():
        assert bary(mesh, g[2][ig][diff], g[0][ig][diff]).min() >= -1e-5
    assert abs(sg.injected - so.injected) <= 10
    W = ctx.charge()
    assert int(W.sum()) == len(g[3]) * 2 ** 32
    assert rel(ctx.potential(), o2.potential()) <= 1e-6


TF_STEPS = int(os.environ.get("PIC_PARITY_TIP_STEPS", "20"))


def test_teacher_forced_bench_fp32ir(picfem, oracle_mod, tip1m, oracle_state):
    """The benchmark's configuration (FP32 push, FP32 Chebyshev-PCG inside
    FP64 refinement to the benchmark's 1e-6, fused pic_step) against the FP64
    oracle (rtol 1e-10) over TF_STEPS steps (PIC_PARITY_TIP_STEPS; 20 by
    default) of the evolving sample population, each step started from the
    oracle's state: every SP within 1e-5 of the box height, every differing
    cell, injection count, exit and periodic image explained by
    tests/freerun_check.py, exact charge conservation, and the new potential
    within 1e-6 after every step in which both runs deposited the same SPs
    on the same side of the box."""
    from freerun_check import FreeRunCheck
    mesh, p = tip1m
    orc0, phi0, parts = oracle_state
    orc = oracle_mod.Oracle(mesh, dict(p, precision=K.PREC_FP64, pcg_rtol=1e-10,
                                       pcg_max_iter=50000), parallel=True)
    orc.set_potential(orc0.potential())
    orc.set_particles(*parts)
    ctx = picfem.Context(p).mesh_load(mesh)
    worst, flips, div, checked, events = 0.0, 0, 0, 0, []
    for _ in range(TF_STEPS):
        k = orc.step_index
        ctx.set_potential(orc.potential())
        ctx.set_particles(*orc.particles())
        ctx.step_index = k
        E_g, E_o = ctx.field(), orc.field()
        ctx.step(1)
        orc.step(1)
        chk = FreeRunCheck(mesh, orc, p["seed"])
        g = ctx.particles()
        chk.step(k, g, orc.particles(), E_g, E_o)
        assert not chk.failures, (k, chk.summary())
        s = chk.summary()
        flips += s["injection_flips"]
        div += s["cell_divergences"]
        checked += s["sp_steps_checked"]
        assert int(ctx.charge().sum()) == len(g[3]) * 2 ** 32
        if s["first_event_step"] is None:
            worst = max(worst, rel(ctx.potential(), orc.potential()))
        else:
            events.append((k, rel(ctx.potential(), orc.potential())))
    print(f"tip_1m FP32+IR teacher-forced {TF_STEPS} steps: {checked} SP-steps, "
          f"{div} face flips, {flips} injection flips, potential {worst:.2e}, steps with a "
          f"charge event (step, potential): {events}")
    assert worst <= 1e-6


SENS_STEPS = int(os.environ.get("PIC_SENS_TIP_STEPS", "20"))


def test_free_running_bench_fp32ir(picfem, oracle_mod, tip1m, oracle_state):
    """Free-running from identical state.  SPs near the apex cross the box in
    a step or two, so a potential that differs at the solver's tolerance
    (1e-6), or an SP more or fewer from one rounding of eq. rnd_nsp, moves
    them by more than 1e-5 of the box height within a few steps, and their
    charge feeds back into the potential: any two correct runs part ways.
    The benchmark's form (rtol 1e-6) against the oracle (rtol 1e-10) is
    therefore held to the spread of the oracle itself when its state is
    rounded to FP32 after every step and it solves to the benchmark's 1e-6:
    at every step at most ten times the fraction of SPs beyond 1e-5 of the
    box height (plus 1e-3) and ten times the 99.9th percentile of the
    distance (plus 1e-5); the first step, from identical state, within the
    bar outright."""
    mesh, p = tip1m
    orc0, phi0, parts = oracle_state
    L = mesh.box_hi - mesh.box_lo

    def start(rtol):
        o = oracle_mod.Oracle(mesh, dict(p, precision=K.PREC_FP64, pcg_rtol=rtol,
                                         pcg_max_iter=50000), parallel=True)
        o.set_potential(orc0.potential())
        o.set_particles(*parts)
        return o

    ref, r32 = start(1e-10), start(1e-6)
    ctx = picfem.Context(p).mesh_load(mesh)
    ctx.set_potential(orc0.potential())
    ctx.set_particles(*parts)

    def spread(x, y):
        common, ix, iy = np.intersect1d(x[3], y[3], return_indices=True)
        d = x[0][ix] - y[0][iy]
        d[:, :2] -= L[:2] * np.round(d[:, :2] / L[:2])
        e = np.abs(d).max(axis=1) / L[2]
        return float(np.mean(e > 1e-5)), float(np.quantile(e, 0.999))

    rows = []
    for _ in range(SENS_STEPS):
        k = ref.step_index
        ctx.step(1)
        ref.step(1)
        r32.step(1)
        r, v, c, i = r32.particles()
        r32.set_particles(r.astype(np.float32).astype(np.float64),
                          v.astype(np.float32).astype(np.float64), c, i)
        g, o = ctx.particles(), ref.particles()
        rows.append((k,) + spread(g, o) + spread(r32.particles(), o))
    print("tip_1m FP32+IR free-running spread (step, GPU frac > 1e-5 Lz, GPU q999, "
          "oracle-FP32-state frac, q999):", rows)
    assert rows[0][1] == 0.0 and rows[0][2] <= 1e-5
    for k, gf, gq, of, oq in rows:
        assert gf <= 10 * of + 1e-3, rows
        assert gq <= 10 * oq + 1e-5, rows


def test_fp64_split_step_bit_exact_full_size(picfem, oracle_mod, tip1m, oracle_state):
    """FP64 form at full size: injection, push, walk and deposit of the
    sample from identical state are bit-exact."""
    mesh, p = tip1m
    orc, phi0, parts = oracle_state
    pp = dict(p, precision=K.PREC_FP64, pcg_cheb_degree=0)
    o2 = oracle_mod.Oracle(mesh, pp, parallel=True)
    o2.set_potential(orc.potential())
    o2.set_particles(*parts)
    ctx = picfem.Context(pp).mesh_load(mesh)
    ctx.set_potential(orc.potential())
    ctx.set_particles(*parts)
    assert ctx.inject(9) == o2.inject(9)
    sg, so = ctx.push_relocate(9), o2.push_relocate(9)
    for f in ("collected", "absorbed", "wrapped", "crossings", "max_walk", "alive"):
        assert getattr(sg, f) == getattr(so, f), f
    for a, b in zip(by_id(ctx.particles()), by_id(o2.particles())):
        assert np.array_equal(a, b)
    ctx.deposit()
    assert np.array_equal(ctx.charge(), o2.deposit())


def test_one_step_large_tip_fp32ir(picfem, oracle_mod):
    """The large tip (7.9M tets, 1.35M free DOFs: the general solver kernels)
    in its benchmark configuration: one fused FP32+IR step of a seeded 2e5-SP
    sample from identical state (the GPU's FP64 solve at rtol 1e-12 as the
    common starting potential) against the OpenMP oracle (rtol 1e-10): every
    SP within 1e-5 of the box height, every differing cell, injection count,
    exit and periodic image explained, exact charge conservation, and the new
    potential within 1e-6 unless the step had a charge event."""
    from freerun_check import FreeRunCheck
    mesh, p, _ = K.workload("tip_8m")
    parts = inputs.random_particles(mesh, N_SAMPLE, seed=88, v_scale=3e6, v_up=1.5e7)
    ref = picfem.Context(dict(p, precision=K.PREC_FP64, pcg_rtol=1e-12, pcg_cheb_degree=0,
                              pcg_max_iter=200_000)).mesh_load(mesh)
    assert ref.info()["pcg_resident"] == 0 and ref.info()["n_tets"] >= 7_500_000
    ref.init_potential()
    ref.set_particles(*parts)
    ref.deposit()
    ref.poisson_solve()
    phi = ref.potential()
    ref.close()
    orc = oracle_mod.Oracle(mesh, dict(p, precision=K.PREC_FP64, pcg_rtol=1e-10,
                                       pcg_max_iter=200_000), parallel=True)
    orc.set_potential(phi)
    orc.set_particles(*parts)
    orc.step_index = 3
    ctx = picfem.Context(p).mesh_load(mesh)
    ctx.set_potential(phi)
    ctx.set_particles(*parts)
    ctx.step_index = 3
    E_g, E_o = ctx.field(), orc.field()
    ctx.step(1)
    orc.step(1)
    chk = FreeRunCheck(mesh, orc, p["seed"])
    g = ctx.particles()
    chk.step(3, g, orc.particles(), E_g, E_o)
    s = chk.summary()
    print("tip_8m FP32+IR one step:", s, "potential", rel(ctx.potential(), orc.potential()))
    assert not chk.failures, s
    assert s["sp_steps_checked"] > 0.9 * N_SAMPLE
    assert int(ctx.charge().sum()) == len(g[3]) * 2 ** 32
    if s["first_event_step"] is None:
        assert rel(ctx.potential(), orc.potential()) <= 1e-6
    ctx.close()
