"""pp_fma_rate, the measured denominator of the ALU roofline fractions: the FP32 rate
of a kernel of FMA chains only must come close to (and not above) SMs x 128 lanes x
2 flop x the maximum SM clock, and the FP64 rate must be far below it (GB300)."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_08919_gb300 import build
    build.build()
    import paper_1704_08919_gb300 as pp
    pp.lib()
    return pp


def test_fma_rates_against_the_derived_fp32_peak(pp):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    derived = sms * 128 * 2 * 2.07e9  # the part's maximum SM clock, 2070 MHz
    r32 = pp.fma_rate("fp32")
    r64 = pp.fma_rate("fp64")
    assert pp.fma_rate("fp32fast") > 0.9 * r32
    assert 0.7 * derived < r32 < 1.03 * derived, (r32, derived)
    assert 0 < r64 < 0.1 * r32, (r64, r32)
