"""The autotuner: it restores the caller's state after timing candidates,
applies the fastest knobs, and a second call for the same workload is served
from its cache."""
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


def test_autotune_restores_state_and_caches(picfem, tip_small, plate_small, tmp_path):
    from paper_1906_08125_gb300 import autotune
    b = inputs.batch_meshes([tip_small, plate_small], [1e10, 9e9])
    p = K.params(w_sp=0.5, capacity=100_000, precision=K.PREC_FP32_IR, pcg_rtol=1e-6,
                 pcg_cheb_degree=6)
    c = picfem.Context(p).mesh_load_batch(b)
    c.init_potential()
    parts = inputs.random_particles(tip_small, 3000, seed=2, v_scale=4e6, v_up=6e6)
    c.set_particles(*parts)
    c.step_index = 9
    before, phi = by_id(c.particles()), c.potential()
    space = {"particle_blocks_per_sm": (4, 8), "walk_form": (1, 2), "pcg_blocks_per_sm": (0, 1),
             "pcg_cheb_degree": (4, 6)}
    cache = str(tmp_path / "tune.json")
    knobs, ms, trials = autotune.tune(c, steps=2, warmup=1, space=space, cache_path=cache)
    assert len(trials) >= 5 and ms > 0
    assert c.tuning() == knobs
    for x, y in zip(by_id(c.particles()), before):
        assert np.array_equal(x, y)
    assert np.array_equal(c.potential(), phi) and c.step_index == 9
    c.set_tuning(particle_blocks_per_sm=2)
    knobs2, ms2, trials2 = autotune.tune(c, space=space, cache_path=cache)
    assert trials2 == [] and knobs2 == knobs and c.tuning() == knobs
    c.close()
