"""GPU: the arithmetic-throughput microbenchmark returns plausible rates.

The FP32 FMA rate must lie between half and 1.1 times the rate derived from
the unit counts (128 FP32 lanes per SM) at the maximum SM clock the device
reports, and the other rates must be positive."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_measured_peaks():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_01521_gb300 as qslab
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    clock_hz = None
    try:
        import subprocess
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits",
                              "-i", "0"], capture_output=True, text=True, timeout=30)
        clock_hz = float(out.stdout.strip().splitlines()[0]) * 1e6
    except Exception:
        pytest.skip("no SM clock reading")
    p = qslab.qslab_measure_peaks(0)
    derived = sms * 128 * clock_hz
    assert 0.5 * derived < p["fp32_fma"] < 1.1 * derived, (p, derived)
    assert p["fp32_ffma2"] > 0.5 * derived
    assert p["fp64_fma"] > 0 and p["ex2"] > 0
