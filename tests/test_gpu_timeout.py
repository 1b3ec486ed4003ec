"""The failure path of the solver's device-side waits.  Every grid barrier and
every tagged halo word of the Poisson solve polls a bounded number of times;
pic_tuning.wait_limit lowers that bound so that the waits run out on purpose.
The solve must then return PIC_ERR_TIMEOUT (the kernel records the status
and returns; nothing traps or hangs), and once the limit is restored the
same context must solve again to the usual accuracy.  Covered: the resident
FP64 and FP32+IR solvers (grid barriers and, for FP32, the tagged exchange)
and the grouped general solver of a batch."""
import numpy as np
import pytest

from paper_1906_08125_gb300 import configs as K
from paper_1906_08125_gb300 import inputs

pytestmark = pytest.mark.gpu

PIC_ERR_TIMEOUT = -8


@pytest.fixture(scope="module")
def picfem():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_08125_gb300 import picfem as P
    P.load()
    return P


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _timeout_then_recover(P, ctx, ref, tol):
    assert ctx.info()["pcg_grid"] > 1          # blocks that wait for one another
    assert ctx.tuning()["wait_limit"] == 0
    zero = np.zeros_like(ref)
    ctx.set_potential(zero)
    ctx.set_tuning(wait_limit=1)               # no barrier can be met in one poll
    with pytest.raises(P.PicError) as e:
        ctx.poisson_solve()
    assert e.value.code == PIC_ERR_TIMEOUT
    assert "timed out" in str(e.value)
    ctx.set_tuning(wait_limit=0)
    ctx.set_potential(zero)
    it, rr = ctx.poisson_solve()
    assert it > 0 and rr <= ctx.params["pcg_rtol"]
    assert rel(ctx.potential(), ref) <= tol
    # a full step on the same context runs as well
    ctx.step(1)


@pytest.mark.parametrize("prec", [K.PREC_FP64, K.PREC_FP32_IR])
def test_resident_solver_wait_limit(picfem, prec):
    mesh, p, _ = K.workload("plate_96k")
    pp = dict(p, precision=prec, pcg_rtol=1e-12 if prec == K.PREC_FP64 else 1e-8,
              pcg_cheb_degree=0 if prec == K.PREC_FP64 else 6)
    ctx = picfem.Context(pp).mesh_load(mesh)
    assert ctx.info()["pcg_resident"] == 1
    if prec == K.PREC_FP32_IR:
        assert ctx.tuning()["pcg_halo_sync"] == 1   # the tagged exchange is in use
    ctx.init_potential()
    ref = ctx.potential()
    _timeout_then_recover(picfem, ctx, ref, 1e-9 if prec == K.PREC_FP64 else 1e-6)
    ctx.close()


def test_grouped_solver_wait_limit(picfem, plate_small, tip_small):
    batch = inputs.batch_meshes([tip_small, plate_small], [1.0e10, 9.0e9])
    p = K.params(w_sp=0.5, pcg_rtol=1e-12, capacity=200_000, precision=K.PREC_FP64,
                 pcg_cheb_degree=0)
    ctx = picfem.Context(p).mesh_load_batch(batch)
    assert ctx.info()["pcg_resident"] == 0
    ctx.init_potential()
    ref = ctx.potential()
    _timeout_then_recover(picfem, ctx, ref, 1e-9)
    ctx.close()


def test_wait_limit_range(picfem, plate_small):
    ctx = picfem.Context(K.params()).mesh_load(plate_small)
    for bad in (-1, (1 << 30) + 1):
        with pytest.raises(picfem.PicError) as e:
            ctx.set_tuning(wait_limit=bad)
        assert e.value.code == -1
    ctx.close()
