"""On-chip throughput microbenchmarks (the denominators of the on-chip
rooflines): each figure is positive and within a factor of a few of what the
SM count and clock allow (FP32: 128 FMA lanes per SM; L1 and shared memory:
128 bytes per clock per SM)."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2202_08627_gb300 import build
    build.build()


def test_measured_peaks_are_plausible():
    from paper_2202_08627_gb300 import ei
    p = ei.ei_measure_peaks()
    sms = p["num_sms"]
    assert sms == torch.cuda.get_device_properties(0).multi_processor_count
    ghz_hi = 2.5                                   # above any shipping SM clock
    assert 0.25 * sms * 128 * 2 * 1.0 * 1e-3 < p["fp32_tflops"] < sms * 128 * 2 * ghz_hi * 1e-3
    for k in ("l1_load_tbs", "smem_load_tbs"):
        assert 0.25 * sms * 128 * 1.0 * 1e-3 < p[k] < 2 * sms * 128 * ghz_hi * 1e-3, (k, p[k])
