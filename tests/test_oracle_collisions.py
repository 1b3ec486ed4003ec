"""Pins of the oracle's Monte Carlo binary collisions (App. F): momentum and
kinetic energy conserved by every collision, SPs alone in their cell left
alone, pairs fixed by the random keys and not by the SPs' buffer order, and
the scattering angle distributed as the appendix states: recovering
delta^2 = tan^2(theta/2) = (1 - cos theta) / (1 + cos theta) from each pair's
rotation, its mean over many independent cells equals the variance
q^4 n Lambda dt / (2 pi eps0^2 m^2 |w|^3 V_cell)."""
import numpy as np
import pytest

from paper_1906_08125_gb300 import configs as K
from paper_1906_08125_gb300 import inputs


def oracle(O, mesh, **kw):
    return O.Oracle(mesh, K.params(**dict(dict(capacity=200_000, collisions=1), **kw)))


def centroid_states(mesh, per_cell, v_of, seed=0):
    """`per_cell` SPs at the centroid of every tetrahedron with velocities v_of(rng, n)."""
    rng = np.random.default_rng(seed)
    T = mesh.n_tets
    cell = np.repeat(np.arange(T, dtype=np.int32), per_cell)
    r = mesh.xyz[mesh.tet[cell]].mean(axis=1)
    v = v_of(rng, len(cell))
    pid = (np.int64(1) << np.int64(62)) + np.arange(len(cell), dtype=np.int64)
    return r, v, cell, pid


def test_conservation_and_lone_sps(oracle_mod, plate_small):
    parts = inputs.random_particles(plate_small, 6000, seed=3, v_scale=2e6, v_up=1e6)
    o = oracle(oracle_mod, plate_small, w_sp=50.0)
    o.set_particles(*parts)
    r0, v0, c0, id0 = o.particles()
    o.collide(7)
    r1, v1, c1, id1 = o.particles()
    assert np.array_equal(id0, id1) and np.array_equal(r0, r1) and np.array_equal(c0, c1)
    counts = np.bincount(c0, minlength=plate_small.n_tets)[c0]
    moved = np.any(v1 != v0, axis=1)
    assert not moved[counts == 1].any()
    assert moved[counts >= 2].mean() > 0.99
    for cell in np.unique(c0[counts >= 2])[:400]:
        s = c0 == cell
        p0, p1 = v0[s].sum(0), v1[s].sum(0)
        assert np.abs(p1 - p0).max() <= 1e-9 * np.abs(v0[s]).max()
        e0, e1 = (v0[s] ** 2).sum(), (v1[s] ** 2).sum()
        assert e1 == pytest.approx(e0, rel=1e-12)


def test_pairs_do_not_depend_on_buffer_order(oracle_mod, plate_small):
    parts = inputs.random_particles(plate_small, 4000, seed=5, v_scale=2e6, v_up=1e6)
    out = []
    for perm in (np.arange(4000), np.random.default_rng(1).permutation(4000)):
        o = oracle(oracle_mod, plate_small, w_sp=20.0)
        o.set_particles(*(a[perm] for a in parts))
        o.collide(11)
        r, v, c, i = o.particles()
        k = np.argsort(i)
        out.append(v[k])
    assert np.array_equal(out[0], out[1])


def test_scattering_variance(oracle_mod, plate_small):
    """Two SPs per cell with a fixed relative velocity w: the mean of
    tan^2(theta/2) / <delta^2>_cell over the cells is 1 (sd sqrt(2/N))."""
    w = np.array([1.2e5, -0.4e5, 0.7e5])
    u = np.linalg.norm(w)

    def vel(rng, n):
        v = np.zeros((n, 3))
        v[0::2] = 0.5 * w
        v[1::2] = -0.5 * w
        return v

    mesh = plate_small
    w_sp = 3e-5
    o = oracle(oracle_mod, mesh, w_sp=w_sp, dt=4e-15)
    r, v, cell, pid = centroid_states(mesh, 2, vel)
    o.set_particles(r, v, cell, pid)
    o.collide(2)
    _, v1, c1, i1 = o.particles()
    k = np.argsort(i1)
    v1, c1 = v1[k], c1[k]
    w1 = v1[0::2] - v1[1::2]
    assert np.allclose(np.linalg.norm(w1, axis=1), u, rtol=1e-12)
    cos_t = (w1 @ w) / (u * u)
    d2 = (1 - cos_t) / (1 + cos_t)
    jinv, x0, vol = o.geometry()
    V = vol[c1[0::2]]
    m = K.M_E
    q = K.Q_ELECTRON
    var = q ** 4 * (2 * w_sp) * 13.0 * 4e-15 / (2 * np.pi * K.EPS0 ** 2 * m * m * u ** 3 * V)
    ratio = d2 / var
    N = len(ratio)
    assert 0.01 < var.mean() < 1.0
    assert abs(ratio.mean() - 1.0) <= 4 * np.sqrt(2.0 / N)
    # the azimuth is uniform: the deflections average out around w
    perp = w1 - np.outer(cos_t, w)
    assert np.linalg.norm(perp.mean(axis=0)) <= 4 * np.linalg.norm(perp, axis=1).mean() / np.sqrt(N)


def test_odd_cells_collide_three_ways(oracle_mod, plate_small):
    def vel(rng, n):
        return rng.normal(0, 1e5, size=(n, 3))

    o = oracle(oracle_mod, plate_small, w_sp=5.0)
    r, v, cell, pid = centroid_states(plate_small, 3, vel, seed=2)
    o.set_particles(r, v, cell, pid)
    o.collide(1)
    _, v1, c1, i1 = o.particles()
    k = np.argsort(i1)
    v1 = v1[k]
    assert np.all(np.any(v1 != v, axis=1))
    p0 = v.reshape(-1, 3, 3).sum(1)
    p1 = v1.reshape(-1, 3, 3).sum(1)
    assert np.abs(p1 - p0).max() <= 1e-9 * np.abs(v).max()
    e0 = (v.reshape(-1, 3, 3) ** 2).sum((1, 2))
    e1 = (v1.reshape(-1, 3, 3) ** 2).sum((1, 2))
    assert np.allclose(e1, e0, rtol=1e-12)
