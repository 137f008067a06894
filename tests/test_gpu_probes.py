"""The pipe probes the roofline denominators and the precision choices rest on
(spike_measure_fp64_peak, spike_measure_pipes): positive rates, the DFMA figure of both
entry points agreeing, the lower-precision pipes faster than FP64, and the mixed-warp run
taking at least as long as either solo run."""
import pytest

from paper_1811_03559_gb300 import spike

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    spike.lib()


def test_pipe_probes_are_consistent():
    peak = spike.measure_fp64_peak()
    p = spike.measure_pipes()
    assert all(v > 0 for v in p.values()), p
    assert abs(p["dfma_tflops"] - peak) <= 0.2 * peak, (p, peak)
    assert p["fp32_fma_tflops"] > p["dfma_tflops"]
    assert p["bf16_mma_sync_tflops"] > p["fp32_fma_tflops"]
    solo = max(p["dfma_even_warps_ms"], p["dmma_odd_warps_ms"])
    assert p["both_alternate_warps_ms"] >= 0.9 * solo, p


def test_pipe_probe_arguments():
    import ctypes
    import numpy as np
    L = spike.lib()
    assert L.spike_measure_pipes(None, None, 7) == -2
    out = np.zeros(2)
    assert L.spike_measure_pipes(None, out.ctypes.data_as(ctypes.c_void_p), 0) == -3
    # a short output array receives the leading entries only
    assert L.spike_measure_pipes(None, out.ctypes.data_as(ctypes.c_void_p), 2) == 0
    assert out[0] > 0 and out[1] > 0
