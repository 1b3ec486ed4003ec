"""Parity of pic_adjoint (the reverse-mode derivative of the collected charge
with respect to E0 and the per-face work functions) with the oracle's FP64
reverse pass (oracle/adjoint.py, itself pinned by central finite differences
and a closed form): same collected charge, gradients within 1e-6 relative in
FP64; independence of the checkpoint interval; the FP32_IR form; replicas of
a batch; the torch.autograd bridge; and the state the call leaves behind."""
import numpy as np
import pytest

from paper_1906_08125_gb300 import configs as K
from paper_1906_08125_gb300 import inputs

pytestmark = pytest.mark.gpu

N_STEPS = 6


@pytest.fixture(scope="module")
def picfem():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_08125_gb300 import picfem as P
    P.load()
    return P


def case(seed=1):
    mesh = inputs.plate_mesh(nx=4, ny=4, nz=8, lx=20e-9, ly=20e-9, lz=40e-9,
                             work_function=4.5, name="plate_tiny")
    mesh.work_function = 4.5 + 0.2 * np.random.default_rng(5).uniform(-1, 1, mesh.n_faces)
    parts = inputs.random_particles(mesh, 300, seed=seed, v_scale=2e6, v_up=4e6)
    p = K.params(E0=1e10, w_sp=0.02, pcg_rtol=1e-13, pcg_max_iter=50000, capacity=200_000,
                 seed=seed, precision=K.PREC_FP64, pcg_cheb_degree=0)
    return mesh, parts, p


@pytest.fixture(scope="module")
def oracle_grad(oracle_mod):
    from oracle import adjoint as A
    mesh, parts, p = case()
    orc = oracle_mod.Oracle(mesh, p)
    orc.set_particles(*parts)
    tape = A.record(orc, N_STEPS)
    g = A.prepare(orc, tape)
    return A.gradient(g, tape), tape


def gpu_adjoint(picfem, ckpt, **over):
    mesh, parts, p = case()
    c = picfem.Context(dict(p, **over)).mesh_load(mesh)
    c.set_particles(*parts)
    return c, c.adjoint(N_STEPS, ckpt_every=ckpt)


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


def test_adjoint_fp64_matches_oracle(picfem, oracle_grad):
    (Qo, gE0o, gwfo), tape = oracle_grad
    c, (Q, gE0, gwf) = gpu_adjoint(picfem, ckpt=4)      # segments of 4 and 2 steps
    assert Q == pytest.approx(tape.Q_recorded, rel=1e-14)
    assert gE0[0] == pytest.approx(gE0o, rel=1e-6)
    assert rel(gwf, gwfo) <= 1e-6
    assert np.abs(gwfo).max() > 0 and gE0o != 0


def test_adjoint_independent_of_checkpoint_interval(picfem):
    ref = gpu_adjoint(picfem, ckpt=100)[1]
    for ck in (1, 3):
        Q, gE0, gwf = gpu_adjoint(picfem, ckpt=ck)[1]
        assert Q == ref[0]
        assert gE0[0] == pytest.approx(ref[1][0], rel=1e-11)
        assert rel(gwf, ref[2]) <= 1e-11


def test_adjoint_leaves_the_forward_state(picfem):
    """After pic_adjoint the context holds the state of n_steps ordinary steps."""
    mesh, parts, p = case()
    a = picfem.Context(p).mesh_load(mesh)
    a.set_particles(*parts)
    a.adjoint(N_STEPS, ckpt_every=4)
    b = picfem.Context(p).mesh_load(mesh)
    b.set_particles(*parts)
    b.deposit()
    b.poisson_solve()
    b.step(N_STEPS)
    assert a.step_index == b.step_index == N_STEPS
    sa, sb = a.particles(), b.particles()
    oa, ob = np.argsort(sa[3]), np.argsort(sb[3])
    for x, y in zip(sa, sb):
        assert np.array_equal(x[oa], y[ob])
    assert np.abs(a.potential() - b.potential()).max() <= 1e-9 * np.abs(b.potential()).max()


def same_decisions(a, b):
    """Two runs took the same discrete decisions (which SPs survive, in which
    cell, with which ids) when their final states agree on ids and cells."""
    pa, pb = a.particles(), b.particles()
    if len(pa[3]) != len(pb[3]):
        return False
    oa, ob = np.argsort(pa[3]), np.argsort(pb[3])
    return bool(np.array_equal(pa[3][oa], pb[3][ob]) and np.array_equal(pa[2][oa], pb[2][ob]))


def _fp32_against_fp64(r32, r64, label):
    """The FP32+IR gradient is the derivative of its own frozen-decision
    model.  Where its run took every decision of the FP64 run (same collected
    charge, same surviving SPs in the same cells) the two models are the same
    and the gradients differ by FP32 rounding of the states only (2^-24 per
    stored position, velocity and field value, carried through the steps'
    derivatives): 1e-5 (measured on a GB300: 2e-10 / 1e-9 on the plate, 3.5e-7
    / 1.5e-6 on the tip).  Where a decision differs (an SP on a face, a
    quadrangle count rounding the other way) the models differ by whole SPs
    and the bar is 2 % / 5 %."""
    (c32, (Q, gE0, gwf)), (c64, (Q64, gE0o, gwfo)) = r32, r64
    same = Q == Q64 and same_decisions(c32, c64)
    print(f"{label}: FP32_IR against FP64: same decisions {same}, Q {Q / Q64 - 1 if Q64 else 0.0}, "
          f"dQ/dE0 {gE0[0] / gE0o[0] - 1}, dQ/dphi {rel(gwf, gwfo)}")
    if same:
        assert gE0[0] == pytest.approx(gE0o[0], rel=1e-5)
        assert rel(gwf, gwfo) <= 1e-5
    else:
        assert abs(Q - Q64) <= 2 * abs(Q64) / 100
        assert gE0[0] == pytest.approx(gE0o[0], rel=2e-2)
        assert rel(gwf, gwfo) <= 5e-2
    return same


def test_adjoint_fp32ir_close_to_fp64(picfem, oracle_grad):
    (Qo, gE0o, gwfo), tape = oracle_grad
    r32 = gpu_adjoint(picfem, ckpt=4, precision=K.PREC_FP32_IR, pcg_rtol=1e-8,
                      pcg_cheb_degree=4)
    r64 = gpu_adjoint(picfem, ckpt=4)
    assert r64[1][0] == pytest.approx(tape.Q_recorded, rel=1e-14)
    assert r64[1][1][0] == pytest.approx(gE0o, rel=1e-6)
    # this seeded case takes every decision of the FP64 run, so the tight bar applies
    assert _fp32_against_fp64(r32, r64, "plate")


def test_adjoint_batch_replicas(picfem):
    """Each replica's dQ/dE0 and dQ/dphi equal a one-replica adjoint of its
    mesh with seed + r (FP64)."""
    mesh, parts, p = case()
    E0 = [1.0e10, 9.0e9]
    b = inputs.batch_meshes([mesh, mesh], E0)
    cb = picfem.Context(dict(p, seed=3)).mesh_load_batch(b)
    cat = (np.concatenate([parts[0], parts[0]]), np.concatenate([parts[1], parts[1]]),
           np.concatenate([parts[2], parts[2] + mesh.n_tets]).astype(np.int32),
           np.concatenate([parts[3], parts[3] + (1 << 32)]))
    cb.set_particles(*cat)
    Qb, gE0b, gwfb = cb.adjoint(N_STEPS, ckpt_every=4)
    Qs = 0.0
    for r in range(2):
        c = picfem.Context(dict(p, seed=3 + r, E0=E0[r])).mesh_load(mesh)
        pr = (parts[0], parts[1], parts[2], parts[3] + (r << 32))
        c.set_particles(*pr)
        Q, gE0, gwf = c.adjoint(N_STEPS, ckpt_every=4)
        Qs += Q
        assert gE0b[r] == pytest.approx(gE0[0], rel=1e-8)
        sl = slice(b.face_off[r], b.face_off[r + 1])
        assert rel(gwfb[sl], gwf) <= 1e-8
    assert Qb == pytest.approx(Qs, rel=1e-14)


def test_autograd_bridge(picfem):
    import torch
    from paper_1906_08125_gb300.autograd import collected_charge
    mesh, parts, p = case()
    c = picfem.Context(p).mesh_load(mesh)
    c.set_particles(*parts)
    E0 = torch.tensor([1e10], dtype=torch.float64, requires_grad=True)
    wf = torch.tensor(mesh.work_function, dtype=torch.float64, requires_grad=True)
    Q = collected_charge(c, E0, wf, N_STEPS, ckpt_every=4)
    (2.0 * Q).backward()
    ref = gpu_adjoint(picfem, ckpt=4)[1]
    assert float(Q.detach()) == ref[0]
    assert E0.grad.item() == pytest.approx(2 * ref[1][0], rel=1e-11)
    assert rel(wf.grad.numpy(), 2 * ref[2]) <= 1e-11


def tip_case(seed=2):
    """The adjoint on a tip: emission from the curved surface and the plane
    around it (work functions 4.5 +/- 0.2 eV per face), SPs with fast
    lateral velocities so that the periodic wrap of Gamma_2 is taken."""
    mesh = inputs.tip_mesh(radius=3e-9, height=12e-9, width=24e-9, box_height=40e-9,
                           h_fine=0.8e-9, lateral_growth=1.3, h_lat_max=3e-9, h_shank=2e-9,
                           h_top_max=4e-9, vertical_growth=1.3, name="tip_small")
    mesh.work_function = 4.5 + 0.2 * np.random.default_rng(6).uniform(-1, 1, mesh.n_faces)
    parts = inputs.random_particles(mesh, 400, seed=seed, v_scale=8e6, v_up=2e6)
    p = K.params(E0=1e10, w_sp=0.05, pcg_rtol=1e-13, pcg_max_iter=50000, capacity=200_000,
                 seed=seed, precision=K.PREC_FP64, pcg_cheb_degree=0)
    return mesh, parts, p


def test_adjoint_fp64_matches_oracle_on_a_tip(picfem, oracle_mod):
    """FP64 pic_adjoint on a tip with the periodic wrap active, against the
    oracle's reverse pass: same collected charge, dQ/dE0 and dQ/dphi within
    1e-6, and faces of the tip's curved surface carry gradient."""
    from oracle import adjoint as A
    mesh, parts, p = tip_case()
    probe = oracle_mod.Oracle(mesh, p)
    probe.set_particles(*parts)
    probe.deposit()
    probe.poisson_solve()
    st = probe.step(N_STEPS)
    assert sum(s.wrapped for s in st) > 0 and sum(s.collected for s in st) > 0
    orc = oracle_mod.Oracle(mesh, p)
    orc.set_particles(*parts)
    tape = A.record(orc, N_STEPS)
    g = A.prepare(orc, tape)
    Qo, gE0o, gwfo = A.gradient(g, tape)
    c = picfem.Context(p).mesh_load(mesh)
    c.set_particles(*parts)
    Q, gE0, gwf = c.adjoint(N_STEPS, ckpt_every=4)
    assert Q == pytest.approx(tape.Q_recorded, rel=1e-14)
    assert gE0[0] == pytest.approx(gE0o, rel=1e-6)
    assert rel(gwf, gwfo) <= 1e-6
    # the emitting faces on the tip (above the cathode plane) take part
    fz = mesh.xyz[mesh.face_nodes].mean(axis=1)[:, 2]
    assert np.abs(gwfo[fz > 1e-9]).max() > 0
    # the FP32+IR form on the same tip against this FP64 run
    c32 = picfem.Context(dict(p, precision=K.PREC_FP32_IR, pcg_rtol=1e-8,
                              pcg_cheb_degree=4)).mesh_load(mesh)
    c32.set_particles(*parts)
    r32 = (c32, c32.adjoint(N_STEPS, ckpt_every=4))
    _fp32_against_fp64(r32, (c, (Q, gE0, gwf)), "tip")


def test_adjoint_on_the_full_tip_against_oracle_and_central_differences(picfem, oracle_mod):
    """The C4 mesh (the 1M-tet tip), FP64, 3 steps of a seeded 3,000-SP
    population (collected charge and emission from the apex), work functions
    4.5 +/- 0.1 eV per face: pic_adjoint against the oracle's reverse pass
    (same collected charge; dQ/dE0 and dQ/dphi within 1e-6), and the oracle's
    reverse pass at this size against central differences of its smooth model
    at h = 1e-4 (relative in E0; 1e-4 eV on the face of the largest
    sensitivity): the reverse pass is pinned at the benchmark's own mesh, not
    only on the small cases."""
    import bench
    from oracle import adjoint as A
    from oracle import oracle as O
    mesh, p0, _ = K.workload("tip_1m")
    mesh.work_function = 4.5 + 0.1 * np.random.default_rng(3).uniform(-1, 1, mesh.n_faces)
    parts = bench.bench_population(mesh, 3000, seed=17)
    p = dict(p0, precision=K.PREC_FP64, pcg_rtol=1e-13, pcg_max_iter=200_000,
             pcg_cheb_degree=0)
    steps = 3
    orc = O.Oracle(mesh, p, parallel=True)
    orc.set_particles(*parts)
    tape = A.record(orc, steps)
    g = A.prepare(orc, tape)
    assert not g.direct                       # iterative solves at this size
    Qo, gE0o, gwfo = A.gradient(g, tape)
    assert Qo != 0.0 and gE0o != 0.0
    h = 1e-4
    fd = (A.replay(g, tape, tape.E0 * (1 + h), tape.wf)
          - A.replay(g, tape, tape.E0 * (1 - h), tape.wf)) / (2 * h * tape.E0)
    assert gE0o == pytest.approx(fd, rel=1e-4)
    f = int(np.argmax(np.abs(gwfo)))
    e = np.zeros_like(tape.wf)
    e[f] = 1.0
    fdf = (A.replay(g, tape, tape.E0, tape.wf + 1e-4 * e)
           - A.replay(g, tape, tape.E0, tape.wf - 1e-4 * e)) / 2e-4
    assert gwfo[f] == pytest.approx(fdf, rel=1e-4)
    c = picfem.Context(p).mesh_load(mesh)
    c.set_particles(*parts)
    Q, gE0, gwf = c.adjoint(steps, ckpt_every=2)
    c.close()
    print(f"tip_1m adjoint: Q {Q:.6e} ({Q / Qo - 1:.1e}), dQ/dE0 {gE0[0] / gE0o - 1:.1e}, "
          f"dQ/dphi {rel(gwf, gwfo):.1e}, FD E0 {gE0o / fd - 1:.1e}, FD face {gwfo[f] / fdf - 1:.1e}")
    assert Q == pytest.approx(tape.Q_recorded, rel=1e-14)
    assert gE0[0] == pytest.approx(gE0o, rel=1e-6)
    assert rel(gwf, gwfo) <= 1e-6
