"""Parity of the CUDA binary collisions (pic_collide, App. F) with the oracle:
the same pairs (fixed by the random order keys) and the same velocities to
the rounding of the transcendental functions; the collisions inside
pic_step (graph replays equal direct launches); replicas of a batch equal
one-replica runs; and the adjoint refuses a run with collisions."""
import numpy as np
import pytest

from paper_1906_08125_gb300 import configs as K
from paper_1906_08125_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def picfem():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_08125_gb300 import picfem as P
    P.load()
    return P


def by_id(state):
    r, v, cell, pid = state
    o = np.argsort(pid, kind="stable")
    return r[o], v[o], cell[o], pid[o]


def test_collide_matches_oracle(picfem, oracle_mod, plate_small, tip_small):
    for mesh, n in ((plate_small, 8000), (tip_small, 20000)):
        p = K.params(w_sp=20.0, capacity=100_000, precision=K.PREC_FP64, collisions=1)
        parts = inputs.random_particles(mesh, n, seed=9, v_scale=2e6, v_up=1e6)
        ctx = picfem.Context(p).mesh_load(mesh)
        orc = oracle_mod.Oracle(mesh, p)
        for c in (ctx, orc):
            c.set_particles(*parts)
            c.collide(13)
        g, o = by_id(ctx.particles()), by_id(orc.particles())
        assert np.array_equal(g[0], o[0]) and np.array_equal(g[2], o[2])
        vmax = np.abs(o[1]).max()
        assert np.abs(g[1] - o[1]).max() <= 1e-12 * vmax
        moved = np.any(g[1] != parts[1][np.argsort(parts[3])], axis=1)
        assert moved.mean() > 0.2


def test_steps_with_collisions_graph_and_oracle(picfem, oracle_mod, plate_small):
    base = dict(E0=1e10, w_sp=0.5, capacity=100_000, precision=K.PREC_FP64, collisions=1,
                pcg_rtol=1e-12)
    parts = inputs.random_particles(plate_small, 6000, seed=2, v_scale=2e6, v_up=3e6)
    ctx = {g: picfem.Context(K.params(graph=g, **base)).mesh_load(plate_small) for g in (0, 1)}
    orc = oracle_mod.Oracle(plate_small, K.params(**base))
    orc.init_potential()
    for c in ctx.values():
        c.set_potential(orc.potential())
        c.set_particles(*parts)
    orc.set_particles(*parts)
    sg = {g: c.step(3) for g, c in ctx.items()}
    so = orc.step(3)
    assert ctx[1].info()["graph"] == 1
    for x, y in zip(by_id(ctx[0].particles()), by_id(ctx[1].particles())):
        assert np.array_equal(x, y)
    g, o = by_id(ctx[0].particles()), by_id(orc.particles())
    assert [s.injected for s in sg[0]] == [s.injected for s in so]
    assert np.array_equal(g[3], o[3])
    Lz = plate_small.box_hi[2]
    assert np.abs(g[0] - o[0]).max() <= 1e-9 * Lz
    assert np.abs(g[1] - o[1]).max() <= 1e-9 * np.abs(o[1]).max()


def test_batch_replica_collisions_equal_single(picfem, plate_small, tip_small):
    b = inputs.batch_meshes([tip_small, plate_small], [1e10, 9e9])
    p = K.params(w_sp=20.0, capacity=100_000, precision=K.PREC_FP64, collisions=1, seed=4)
    parts = [inputs.random_particles(m, 5000, seed=20 + r, v_scale=2e6, v_up=1e6)
             for r, m in enumerate(b.members)]
    cat = tuple(np.concatenate([pp[k] + (b.tet_off[r] if k == 2 else 0) + ((r << 32) if k == 3 else 0)
                                for r, pp in enumerate(parts)]) for k in range(4))
    cb = picfem.Context(p).mesh_load_batch(b)
    cb.set_particles(cat[0], cat[1], cat[2].astype(np.int32), cat[3])
    cb.collide(6)
    vb = by_id(cb.particles())
    for r, m in enumerate(b.members):
        c = picfem.Context(dict(p, seed=4 + r)).mesh_load(m)
        pr = parts[r]
        c.set_particles(pr[0], pr[1], pr[2], pr[3] + (r << 32))
        c.collide(6)
        s = by_id(c.particles())
        sel = (vb[2] >= b.tet_off[r]) & (vb[2] < b.tet_off[r + 1])
        assert np.array_equal(vb[1][sel], s[1])


def test_adjoint_refuses_collisions(picfem, plate_small):
    c = picfem.Context(K.params(collisions=1, capacity=1000)).mesh_load(plate_small)
    with pytest.raises(picfem.PicError) as e:
        c.adjoint(2)
    assert e.value.code == -7
