"""pic_step replayed from captured CUDA graphs equals direct launches bit for
bit: the step index and the per-step statistics live on the device, so one
graph per particle-buffer parity serves every step."""
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


STAT_FIELDS = ("injected", "collected", "absorbed", "wrapped", "crossings", "alive",
               "max_walk", "pcg_iters", "pcg_relres", "pcg_outer")


@pytest.mark.parametrize("form", [dict(precision=K.PREC_FP64, pcg_rtol=1e-10),
                                  dict(precision=K.PREC_FP32_IR, pcg_rtol=1e-6,
                                       pcg_cheb_degree=6)])
def test_graph_steps_equal_direct(picfem, tip_small, form):
    base = dict(E0=1e10, w_sp=0.5, capacity=100_000, seed=3, **form)
    ctx = {g: picfem.Context(K.params(graph=g, **base)).mesh_load(tip_small) for g in (0, 1)}
    parts = inputs.random_particles(tip_small, 4000, seed=5, v_scale=4e6, v_up=6e6)
    for c in ctx.values():
        c.init_potential()
        c.set_particles(*parts)
        c.step_index = 17
    l0 = {g: c.launch_count() for g, c in ctx.items()}
    st = {g: c.step(3) + c.step(4) for g, c in ctx.items()}   # odd count: both parities
    assert ctx[1].info()["graph"] == 1 and ctx[0].info()["graph"] == 0
    for a, b in zip(st[0], st[1]):
        for f in STAT_FIELDS:
            assert getattr(a, f) == getattr(b, f), f
    assert [s.injected for s in st[1]] != [0] * 7
    for x, y in zip(by_id(ctx[0].particles()), by_id(ctx[1].particles())):
        assert np.array_equal(x, y)
    assert np.array_equal(ctx[0].charge(), ctx[1].charge())
    assert np.array_equal(ctx[0].potential(), ctx[1].potential())
    assert ctx[0].step_index == ctx[1].step_index == 24
    assert ctx[1].launch_count() - l0[1] == ctx[0].launch_count() - l0[0]
    # split calls after graph replays use the step they are given
    for c in ctx.values():
        assert c.inject(30) >= 0
    for x, y in zip(by_id(ctx[0].particles()), by_id(ctx[1].particles())):
        assert np.array_equal(x, y)


def test_graph_off_while_profiling(picfem, plate_small):
    c = picfem.Context(K.params(E0=1e10, w_sp=0.5, capacity=20000, graph=1)).mesh_load(plate_small)
    c.init_potential()
    c.profile(True)
    c.step(2)
    assert c.info()["graph"] == 0
    rep = c.profile_read()
    assert rep["step_fused"][0] == 2
    c.profile(False)
    c.step(2)
    assert c.info()["graph"] == 1


def test_tuning_knobs_keep_results(picfem, tip_small, plate_small):
    """Launch knobs change nothing that is computed: the particle grid and the
    walk form leave every SP and the node charge bit-identical; the batch
    solver's block budget changes only the reduction order."""
    base = dict(E0=1e10, w_sp=0.5, capacity=100_000, seed=3, precision=K.PREC_FP32_IR,
                pcg_rtol=1e-8, pcg_cheb_degree=6)
    parts = inputs.random_particles(tip_small, 4000, seed=5, v_scale=4e6, v_up=6e6)
    runs = []
    for knobs in ({}, dict(particle_blocks_per_sm=2, walk_form=2),
                  dict(particle_blocks_per_sm=16, walk_form=1),
                  dict(particle_blocks_per_sm=8, walk_form=3)):
        c = picfem.Context(K.params(**base)).mesh_load(tip_small)
        c.set_tuning(**knobs)
        c.init_potential()
        c.set_particles(*parts)
        c.step(3)
        runs.append((by_id(c.particles()), c.charge(), c.potential()))
        assert all(c.tuning()[k] == v for k, v in knobs.items())
    for r in runs[1:]:
        for x, y in zip(r[0], runs[0][0]):
            assert np.array_equal(x, y)
        assert np.array_equal(r[1], runs[0][1])
        assert np.array_equal(r[2], runs[0][2])
    b = inputs.batch_meshes([tip_small, plate_small, tip_small], [1e10, 9e9, 1.1e10])
    phis = []
    for bps in (0, 1, 3):
        c = picfem.Context(K.params(**dict(base, precision=K.PREC_FP64, pcg_rtol=1e-12,
                                           pcg_cheb_degree=0))).mesh_load_batch(b)
        c.set_tuning(pcg_blocks_per_sm=bps)
        g0 = c.info()["pcg_grid"]
        c.init_potential()
        phis.append(c.potential())
        import torch
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        assert bps == 0 or g0 <= bps * sms
    for p in phis[1:]:
        assert np.abs(p - phis[0]).max() <= 1e-9 * np.abs(phis[0]).max()
    with pytest.raises(picfem.PicError):
        c.set_tuning(walk_form=7)
