"""reloc_measure_peaks: the measured FP32 and exponential throughput used as
roofline denominators.  Bounds: a GB300 has 152 SMs x 128 FP32 lanes at up
to 2.07 GHz, 80.5 TFLOP/s nominal for scalar FMAs; a measurement is expected
within a factor of two below that (clock under load) and not above the
nominal figure of the packed form (2x), and the exponential unit runs at a
fraction of the FMA rate."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_11367_gb300.build import build
    build()
    from paper_2403_11367_gb300 import reloc
    return reloc


def test_measured_peaks_are_plausible(R):
    p = R.reloc_measure_peaks(0)
    print(p)
    assert 30.0 < p["fp32_scalar_tflops"] < 90.0
    assert 30.0 < p["fp32_packed_tflops"] < 180.0
    ex2_per_s = p["ex2_gops"] * 1e9
    assert 1e11 < ex2_per_s < p["fp32_scalar_tflops"] * 1e12 / 2


def test_measure_peaks_rejects_missing_device(R):
    with pytest.raises(R.RelocError):
        R.reloc_measure_peaks(10_000)
