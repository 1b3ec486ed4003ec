"""The free-running checker (tests/freerun_check.py) on the CPU: two oracle
runs from identical state agree with nothing to explain; mistakes planted in
one of them (a displaced SP, a dropped SP) are reported as unexplained; an SP
started on a shared face with a different owning cell in each run is
explained as a cell divergence however far its trajectories then part; the
injection rule explains exactly the indices one reading of eq. rnd_nsp has
and the other has not."""
import numpy as np
import pytest

from paper_1906_08125_gb300 import configs as K
from paper_1906_08125_gb300 import inputs

from freerun_check import (FreeRunCheck, count_of, injection_flip_explained,
                           point_triangle_distance)


def _pair(oracle_mod, mesh, n=600, seed=5):
    p = K.params(E0=3e9, w_sp=0.02, pcg_rtol=1e-12, capacity=100_000)
    runs = []
    for _ in range(2):
        o = oracle_mod.Oracle(mesh, p)
        o.init_potential()
        runs.append(o)
    parts = inputs.random_particles(mesh, n, seed=seed, v_scale=5e5, v_up=0.0)
    for o in runs:
        o.set_particles(*parts)
    return runs, p


def _run(chk, a, b, steps, plant=None):
    for k in range(steps):
        if plant:
            plant(k, a, b)
        Ea, Eb = a.field(), b.field()
        a.step(1)
        b.step(1)
        chk.step(k, a.particles(), b.particles(), Ea, Eb)


def test_identical_runs_have_nothing_to_explain(oracle_mod, tip_small):
    (a, b), p = _pair(oracle_mod, tip_small)
    chk = FreeRunCheck(tip_small, b, p["seed"], fp32_positions=False)
    _run(chk, a, b, 8)
    s = chk.summary()
    assert not chk.failures and s["cell_divergences"] == 0 and s["injection_flips"] == 0
    assert s["max_err_clean_rel"] == 0.0 and s["sp_steps_checked"] > 800


def test_displaced_sp_is_unexplained(oracle_mod, tip_small):
    (a, b), p = _pair(oracle_mod, tip_small)
    chk = FreeRunCheck(tip_small, b, p["seed"], fp32_positions=False)
    Lz = tip_small.box_hi[2] - tip_small.box_lo[2]

    def plant(k, a, b):
        if k == 3:
            r, v, cell, pid = a.particles()
            i = int(np.nonzero((r[:, 2] > 0.4 * Lz) & (r[:, 2] < 0.5 * Lz))[0][0])
            r[i, 0] += 3e-5 * Lz                  # stays in its cell or a neighbour
            a.set_particles(r, v, a.locate(r, cell)[1], pid)
    _run(chk, a, b, 6, plant)
    assert any("position" in f[1] or "apart" in f[1] for f in chk.failures), chk.failures


def test_dropped_sp_is_unexplained(oracle_mod, tip_small):
    (a, b), p = _pair(oracle_mod, tip_small)
    chk = FreeRunCheck(tip_small, b, p["seed"], fp32_positions=False)
    Lz = tip_small.box_hi[2] - tip_small.box_lo[2]

    def plant(k, a, b):
        if k == 2:
            r, v, cell, pid = a.particles()
            mid = np.nonzero((r[:, 2] > 0.4 * Lz) & (r[:, 2] < 0.6 * Lz))[0][0]
            keep = np.arange(len(pid)) != mid
            a.set_particles(r[keep], v[keep], cell[keep], pid[keep])
    _run(chk, a, b, 4, plant)
    assert any("Gamma" in f[1] for f in chk.failures), chk.failures


def test_sp_on_a_face_with_two_owners_is_explained(oracle_mod, tip_small):
    """One SP starts on the face shared by two tetrahedra with a different
    owner in each run: its fields, and so its trajectories, differ from the
    first kick on; the divergence is explained at the start, and nothing else
    differs beyond what that one SP's space charge explains."""
    mesh = tip_small
    p = K.params(E0=1e9, w_sp=1e-6, pcg_rtol=1e-12, capacity=10_000)
    a, b = (oracle_mod.Oracle(mesh, p) for _ in range(2))
    for o in (a, b):
        o.init_potential()
        o.set_work_function(np.full(mesh.n_faces, 1000.0))     # no emission
    E = a.field()
    # an interior face whose two tetrahedra have clearly different fields
    t = np.arange(mesh.n_tets)
    k = np.argmax(mesh.nbr >= 0, axis=1)
    nb = mesh.nbr[t, k]
    dE = np.linalg.norm(E[t] - E[np.maximum(nb, 0)], axis=1) * (nb >= 0)
    zc = mesh.xyz[mesh.tet].mean(axis=1)[:, 2]
    dE[zc < 0.2 * mesh.box_hi[2]] = 0
    A = int(np.argmax(dE))
    B = int(mesh.nbr[A, k[A]])
    loc = [i for i in range(4) if i != k[A]]
    r0 = mesh.xyz[mesh.tet[A, loc]].mean(axis=0)
    pid = np.array([1 << 62], np.int64)
    v0 = np.zeros((1, 3))
    a.set_particles(r0[None], v0, np.array([A], np.int32), pid)
    b.set_particles(r0[None], v0, np.array([B], np.int32), pid)
    chk = FreeRunCheck(mesh, b, p["seed"], fp32_positions=False)
    chk.step(-1, a.particles(), b.particles(), E, E)
    _run(chk, a, b, 2)
    assert not chk.failures, chk.failures
    s = chk.summary()
    assert s["cell_divergences"] == 1 and s["sp_steps_checked"] == 3
    ra, rb = a.particles()[0], b.particles()[0]
    assert np.abs(ra - rb).max() > 1e-5 * mesh.box_hi[2]    # they did part ways


def test_injection_flip_rule():
    # count_of is floor(n) + (R0 < frac(n))
    rng = np.random.default_rng(0)
    n = rng.uniform(0, 5, 1000)
    R0 = rng.uniform(0, 1, 1000)
    fl = np.floor(n)
    assert np.array_equal(count_of(n, R0), (fl + (R0 < n - fl)).astype(np.int64))
    # 2.30 -> 2 SPs, 2.31 -> 3 SPs at R0 = 0.305: only index 2 is explained
    j = np.array([0, 1, 2, 3])
    assert list(injection_flip_explained(2.30, 2.31, 0.305, j)) == [False, False, True, False]
    assert list(injection_flip_explained(2.31, 2.30, 0.305, j)) == [False, False, True, False]
    # R0 outside the bracket: no index differs, none is explained
    assert not injection_flip_explained(2.30, 2.31, 0.5, j).any()


def test_point_triangle_distance():
    a = np.array([[0.0, 0, 0]])
    b = np.array([[1.0, 0, 0]])
    c = np.array([[0.0, 1, 0]])
    pts = np.array([[0.2, 0.2, 0.5], [2.0, 0, 0], [-1.0, -1.0, 0.0], [0.5, 0.5, -1.0]])
    want = [0.5, 1.0, np.sqrt(2.0), 1.0]
    got = point_triangle_distance(pts, np.repeat(a, 4, 0), np.repeat(b, 4, 0), np.repeat(c, 4, 0))
    assert np.allclose(got, want)


def test_sp_on_the_periodic_side_with_two_images_is_explained(oracle_mod, plate_small):
    """One SP exactly on Gamma_2: one run holds it at x = x_lo, the other at
    x = x_hi (wrapped).  Positions agree on the nearest image, the step is a
    charge event (the charge lands on the nodes of opposite sides), and
    nothing is reported as unexplained."""
    mesh = plate_small
    p = K.params(E0=1e9, w_sp=1e-6, pcg_rtol=1e-12, capacity=10_000)
    a, b = (oracle_mod.Oracle(mesh, p) for _ in range(2))
    for o in (a, b):
        o.init_potential()
        o.set_work_function(np.full(mesh.n_faces, 1000.0))     # no emission
    lo, hi = mesh.box_lo, mesh.box_hi
    ra = np.array([[lo[0], 0.37 * (lo[1] + hi[1]), 0.5 * hi[2]]])
    rb = ra.copy()
    rb[0, 0] = hi[0]
    ca = a.locate(ra + [[1e-12, 0, 0]], np.array([0], np.int32))[1]
    cb = b.locate(rb - [[1e-12, 0, 0]], np.array([0], np.int32))[1]
    pid = np.array([1 << 62], np.int64)
    v = np.array([[0.0, 1e5, 0.0]])
    a.set_particles(ra, v, ca, pid)
    b.set_particles(rb, v, cb, pid)
    chk = FreeRunCheck(mesh, b, p["seed"], fp32_positions=False)
    E = a.field()
    chk.step(-1, a.particles(), b.particles(), E, E)
    _run(chk, a, b, 2)
    s = chk.summary()
    assert not chk.failures, chk.failures
    assert s["image_flips"] == 1 and s["first_event_step"] == -1
    assert not np.array_equal(a.charge(), b.charge())   # the charge sits on other nodes
