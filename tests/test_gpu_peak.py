"""The measured FP32 FMA throughput (kpx_fp32_fma_rate), the reference the
bench reports beside the FP32 peak derived from unit counts and the clock:
it must be positive, below the derived peak at the maximum SM clock (with a
little headroom for clock reporting), and scale with the work (twice the
chain length, about twice the time)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kpx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_02846_gb300 as k
    k.load()
    return k


def test_fma_rate_is_plausible(kpx):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    derived = sms * 128 * 2 * 2.07e9 / 1e12  # TFLOP/s at the maximum SM clock
    r1 = kpx.fp32_fma_rate(1024)
    r2 = kpx.fp32_fma_rate(2048)
    print("FP32 FMA rate: %.1f and %.1f TFLOP/s (derived peak %.1f)" % (r1, r2, derived))
    for r in (r1, r2):
        assert 0.25 * derived < r < 1.05 * derived
    assert abs(r2 / r1 - 1.0) < 0.25


def test_fma_rate_rejects_bad_arguments(kpx):
    import ctypes as C
    out = C.c_double()
    L = kpx.load()
    assert L.kpx_fp32_fma_rate(0, C.byref(out), None) == kpx.KPX_E_INVALID
    assert L.kpx_fp32_fma_rate(16, None, None) == kpx.KPX_E_INVALID
