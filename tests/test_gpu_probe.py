"""se_probe_peak: the measured unit rates that bench.py uses as roofline
denominators are positive and of the right order for a GB300 class GPU."""
import pytest
import torch

from paper_1712_04718_gb300 import se

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def test_probe_rates():
    fp32 = se.probe_peak("fp32_fma")
    fp64 = se.probe_peak("fp64_fma")
    au = se.probe_peak("smem_atomic_u32")
    af = se.probe_peak("smem_atomic_f32")
    assert 1e13 < fp32 < 2e14          # FP32 FMA: tens of TFLOP/s
    assert 1e11 < fp64 < fp32          # FP64 well below FP32 on this part
    # conflict-free shared atomics: up to one warp instruction per clock per SM
    assert 1e11 < au < 3e13
    assert 1e11 < af < 3e13
