"""The unit-peak microbenchmarks used by the benchmark's rooflines return figures of the right
order for a Blackwell GPU (152 SMs at about 2 GHz: 128 FP32 lanes, 16 special-function lanes
per SM; FP64 a small fraction of FP32), so a broken timing or a kernel the compiler emptied
would show."""
import pytest

pytestmark = pytest.mark.gpu


def test_measure_peaks_plausible():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_06736_gb300 import build
    build.build()
    import paper_1808_06736_gb300 as pkg
    st, pk = pkg.nufft_measure_peaks(torch.cuda.current_stream().cuda_stream)
    assert st == 0
    assert 20.0 < pk["fp32_tflops"] < 120.0, pk
    assert 0.2 < pk["fp64_tflops"] < 10.0, pk
    assert pk["fp64_tflops"] < pk["fp32_tflops"] / 4, pk
    assert 500.0 < pk["sfu_gops"] < 20000.0, pk
    assert 1e12 < pk["smem_atomics_per_s"] < 3e13, pk
    assert pkg.nufft_measure_peaks.__doc__
