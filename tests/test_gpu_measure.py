"""The FP64 rate probe (pic_measure_fp64_rate) that the FP64 form's roofline is
set against: a finite rate of the right order for a GB300 (its FP64 FMA
rate is a small fraction of the FP32 one), repeatable, and argument errors
refused on the host."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def picfem():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_08125_gb300 import picfem as P
    P.load()
    return P


def test_fp64_rate_probe(picfem):
    a = picfem.measure_fp64_rate(iters=1 << 12)
    b = picfem.measure_fp64_rate(iters=1 << 13)
    print(f"FP64 FMA rate: {a:.3f} / {b:.3f} TFLOP/s")
    assert 0.05 < a < 200.0 and 0.05 < b < 200.0
    assert abs(a - b) <= 0.25 * max(a, b)
    with pytest.raises(picfem.PicError) as e:
        picfem.measure_fp64_rate(iters=0)
    assert e.value.code == -1
