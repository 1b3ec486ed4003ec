"""The OpenMP build of the oracle (its independent loops on all host cores)
gives the serial build's results bit for bit: particles, node charges,
potentials and step statistics over several full PIC steps with injection,
walk, wrap and absorption, on a plate and a tip, with several thread counts."""
import numpy as np
import pytest

from paper_1906_08125_gb300 import configs as K
from paper_1906_08125_gb300 import inputs


def _stats(st):
    return [tuple(getattr(s, f) for f, _ in type(s)._fields_) for s in st]


@pytest.mark.parametrize("meshname", ["plate_small", "tip_small"])
def test_parallel_oracle_is_bit_identical(oracle_mod, meshname, request):
    mesh = request.getfixturevalue(meshname)
    p = K.params(E0=1e10, w_sp=0.05, pcg_rtol=1e-12, capacity=200_000)
    parts = inputs.random_particles(mesh, 20_000, seed=8, v_scale=4e6, v_up=6e6)
    runs = {}
    for threads in (None, 1, 3, 8):
        o = oracle_mod.Oracle(mesh, p, parallel=threads is not None)
        if threads is not None:
            assert oracle_mod.set_threads(threads) == threads
        o.init_potential()
        o.set_particles(*parts)
        st = o.step(6)
        runs[threads] = (o.particles(), o.charge(), o.potential(), _stats(st), o.field())
    ref = runs[None]
    assert ref[3][-1][0] > 0 and sum(s[1] + s[2] for s in ref[3]) > 0   # injected, removed
    for threads, got in runs.items():
        for a, b in zip(got[0], ref[0]):
            assert np.array_equal(a, b), threads
        for a, b in zip(got[1:], ref[1:]):
            assert np.array_equal(np.asarray(a), np.asarray(b)), threads
