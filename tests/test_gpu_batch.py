"""Parity of the batched form (mesh_load_batch): every replica of a batch is
an independent simulation of its own mesh with its own applied field and the
random stream seed + r.  Fed the same potential, each replica's injection,
push, walk and deposit equal a one-replica run of its mesh bit for bit (ids
shifted by the replica's quadrangle offset, cells by its tetrahedron
offset); each replica's potential agrees with the oracle's tight solve of its
own system, and each replica's CG stops on its own residual."""
import numpy as np
import pytest

from paper_1906_08125_gb300 import configs as K
from paper_1906_08125_gb300 import inputs

pytestmark = pytest.mark.gpu

SEED = 11
FATES = ("collected", "absorbed", "wrapped", "crossings", "alive")


@pytest.fixture(scope="module")
def picfem():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_08125_gb300 import picfem as P
    P.load()
    return P


@pytest.fixture(scope="module")
def batch(plate_small, tip_small):
    """Four uneven replicas: two tips, two plates of different boxes; the
    last one at a field too weak to emit much."""
    plate_b = inputs.plate_mesh(nx=8, ny=5, nz=10, lx=40e-9, ly=25e-9, lz=50e-9, name="plate_b")
    return inputs.batch_meshes([tip_small, plate_small, plate_b, tip_small],
                               [1.0e10, 9.0e9, 1.2e10, 3.0e9])


def kw(prec, **extra):
    return dict(dict(w_sp=0.5, pcg_rtol=1e-12, capacity=200_000, precision=prec,
                     pcg_cheb_degree=0), **extra)


def replica_params(batch, r, prec, **extra):
    return K.params(**kw(prec, **extra), E0=float(batch.E0[r]), seed=SEED + r)


def start_state(batch):
    """Seeded SPs per replica (ids distinct across replicas) and the same
    set concatenated in batch numbering."""
    parts = []
    for r, m in enumerate(batch.members):
        x, v, cell, pid = inputs.random_particles(m, 3000 + 1000 * r, seed=40 + r,
                                                  v_scale=4e6, v_up=6e6)
        parts.append((x, v, cell, pid + (np.int64(r) << np.int64(32))))
    cat = tuple(np.concatenate([p[k] + (batch.tet_off[r] if k == 2 else 0)
                                for r, p in enumerate(parts)]) for k in range(4))
    return parts, (cat[0], cat[1], cat[2].astype(np.int32), cat[3])


def split(batch, state):
    """Batch particles -> per replica, in that replica's own numbering."""
    x, v, cell, pid = state
    out = []
    for r in range(batch.n_rep):
        sel = (cell >= batch.tet_off[r]) & (cell < batch.tet_off[r + 1])
        ids = pid[sel].copy()
        injected = (ids >> np.int64(62)) == 0
        ids[injected] -= np.int64(3 * batch.face_off[r]) << np.int64(18)
        out.append(by_id((x[sel], v[sel], cell[sel] - batch.tet_off[r], ids)))
    return out


def by_id(state):
    r, v, cell, pid = state
    o = np.argsort(pid, kind="stable")
    return r[o], v[o], cell[o], pid[o]


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def solo_runs(picfem, batch, prec, **extra):
    return [picfem.Context(replica_params(batch, r, prec, **extra)).mesh_load(m)
            for r, m in enumerate(batch.members)]


@pytest.mark.parametrize("prec", [K.PREC_FP64, K.PREC_FP32_IR])
def test_batch_split_step_equals_replicas(picfem, batch, prec):
    solo = solo_runs(picfem, batch, prec)
    phis = []
    for c in solo:
        c.init_potential()
        phis.append(c.potential())
    b = picfem.Context(K.params(**kw(prec), seed=SEED)).mesh_load_batch(batch)
    info = b.info()
    assert info["n_rep"] == batch.n_rep and info["n_rows"] % 32 == 0
    assert info["n_rows"] >= sum(c.info()["n_free"] for c in solo)
    b.set_potential(np.concatenate(phis))
    parts, cat = start_state(batch)
    b.set_particles(*cat)
    for c, p in zip(solo, parts):
        c.set_particles(*p)
    step = 4
    n_b = b.inject(step)
    n_s = [c.inject(step) for c in solo]
    assert n_b == sum(n_s) and n_s[0] > 0 and n_s[2] > 0
    st_b = b.push_relocate(step)
    st_s = [c.push_relocate(step) for c in solo]
    for f in FATES:
        assert getattr(st_b, f) == sum(getattr(s, f) for s in st_s), f
    assert st_b.max_walk == max(s.max_walk for s in st_s)
    for r, (g, c) in enumerate(zip(split(batch, b.particles()), solo)):
        for x, y in zip(g, by_id(c.particles())):
            assert np.array_equal(x, y), r
    b.deposit()
    W = b.charge()
    for r, c in enumerate(solo):
        c.deposit()
        assert np.array_equal(W[batch.node_off[r]:batch.node_off[r + 1]], c.charge()), r
    it_b, rr_b = b.poisson_solve()
    assert rr_b <= (1e-12 if prec == K.PREC_FP64 else 1e-11)
    phi = b.potential()
    for r, c in enumerate(solo):
        c.poisson_solve()
        got = phi[batch.node_off[r]:batch.node_off[r + 1]]
        assert rel(got, c.potential()) <= 1e-9, r
        c.close()
    b.close()


@pytest.mark.parametrize("form", [dict(precision=K.PREC_FP64),
                                  dict(precision=K.PREC_FP32_IR, pcg_rtol=1e-6,
                                       pcg_cheb_degree=6)])
def test_batch_potential_vs_oracle(picfem, oracle_mod, batch, form):
    """Charge-free and space-charge potentials of every replica against the
    oracle's tight solve of that replica alone."""
    p = K.params(**dict(kw(K.PREC_FP64), **form), seed=SEED)
    b = picfem.Context(p).mesh_load_batch(batch)
    parts, cat = start_state(batch)
    b.init_potential()
    phi0 = b.potential()
    b.set_particles(*cat)
    b.deposit()
    b.poisson_solve()
    phi1 = b.potential()
    tol = 1e-9 if form["precision"] == K.PREC_FP64 else 1e-6
    for r, m in enumerate(batch.members):
        o = oracle_mod.Oracle(m, replica_params(batch, r, K.PREC_FP64, pcg_rtol=1e-13,
                                                pcg_max_iter=50000))
        o.init_potential()
        sl = slice(batch.node_off[r], batch.node_off[r + 1])
        assert rel(phi0[sl], o.potential()) <= tol, (r, "charge-free")
        o.set_particles(*parts[r])
        o.deposit()
        o.poisson_solve()
        assert rel(phi1[sl], o.potential()) <= tol, (r, "space charge")
    b.close()


def test_one_replica_batch_equals_mesh_load(picfem, tip_small):
    """A batch of one replica is the single-mesh context, bit for bit, over
    fused FP32_IR steps (solver included)."""
    p = K.params(**kw(K.PREC_FP32_IR, pcg_rtol=1e-6, pcg_cheb_degree=6), E0=1e10, seed=SEED)
    a = picfem.Context(p).mesh_load(tip_small)
    b = picfem.Context(p).mesh_load_batch(inputs.batch_meshes([tip_small], [1e10]))
    for c in (a, b):
        c.init_potential()
        c.step(3)
    for x, y in zip(by_id(a.particles()), by_id(b.particles())):
        assert np.array_equal(x, y)
    assert np.array_equal(a.charge(), b.charge())
    assert np.array_equal(a.potential(), b.potential())


def test_batch_fused_steps_conserve_and_converge(picfem, batch):
    """Fused FP32_IR steps of the batch: charge conservation over the whole
    batch, every replica's SPs stay inside its own tetrahedra, and the
    per-replica potentials stay close to one-replica runs fed the same
    starting state (they differ only by solver rounding)."""
    p = K.params(**kw(K.PREC_FP32_IR, pcg_rtol=1e-6, pcg_cheb_degree=6), seed=SEED)
    b = picfem.Context(p).mesh_load_batch(batch)
    b.init_potential()
    parts, cat = start_state(batch)
    b.set_particles(*cat)
    stats = b.step(3)
    assert all(s.pcg_relres <= 1e-6 for s in stats)
    x, v, cell, pid = b.particles()
    assert int(b.charge().sum()) == len(pid) * 2 ** 32
    assert len(np.unique(pid)) == len(pid)
    for r in range(batch.n_rep):
        sel = (cell >= batch.tet_off[r]) & (cell < batch.tet_off[r + 1])
        m = batch.members[r]
        assert np.all(x[sel] >= m.box_lo - 1e-12) and np.all(x[sel] <= m.box_hi + 1e-12)
        inj = pid[sel][(pid[sel] >> np.int64(62)) == 0]
        q = (inj >> np.int64(18)) & np.int64((1 << 24) - 1)
        assert np.all((q >= 3 * batch.face_off[r]) & (q < 3 * batch.face_off[r + 1])), r
    b.close()


def test_batch_argument_errors(picfem, batch, plate_small):
    p = K.params(**kw(K.PREC_FP64))
    c = picfem.Context(p)
    bad = inputs.batch_meshes(batch.members, batch.E0)
    bad.tet_off = bad.tet_off.copy()
    bad.tet_off[1] += 1        # tetrahedron offsets disagree with node offsets
    with pytest.raises(picfem.PicError):
        c.mesh_load_batch(bad)
    bad = inputs.batch_meshes(batch.members, batch.E0)
    bad.E0 = bad.E0[:2]        # offsets for 4 replicas, E0 for 2
    with pytest.raises(picfem.PicError):
        c.mesh_load_batch(bad)
    two = inputs.batch_meshes([plate_small, plate_small], [1e10, 1e10])
    nbr = two.mesh.nbr.copy()
    t = int(np.argmax((nbr[:plate_small.n_tets] == inputs.TOP).any(axis=1)))
    k = int(np.argmax(nbr[t] == inputs.TOP))
    nbr[t, k] = plate_small.n_tets          # reaches into the second replica
    two.mesh.nbr = nbr
    with pytest.raises(picfem.PicError):
        c.mesh_load_batch(two)
    c.mesh_load_batch(batch)                # the context is still usable
    assert c.info()["n_rep"] == batch.n_rep
    c.close()
