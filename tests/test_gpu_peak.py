"""The FMA rate micro-benchmark that the ALU rooflines are quoted against: it runs, and
its FP32 rate lies below the lane-count bound (SMs x 128 FP32 lanes x 2 flop x the
maximum SM clock) and well above half of it; FP64 runs far below FP32 on this part."""
import pytest
import torch

pytestmark = pytest.mark.gpu

MAX_SM_MHZ = 2070   # GB300's maximum SM clock


@pytest.fixture(scope="module")
def G():
    from conftest import build_libhmc
    build_libhmc()
    import paper_1009_0457_gb300 as G
    return G


def test_fma_peak_within_the_lane_count_bound(G):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    bound = sms * 128 * 2 * MAX_SM_MHZ * 1e6 / 1e12
    f32 = G.hmc_fma_peak(G.HMC_FP32, 1024)
    f64 = G.hmc_fma_peak(G.HMC_FP64, 64)
    assert 0.5 * bound < f32 <= 1.02 * bound, (f32, bound)
    assert 0.0 < f64 < 0.25 * f32, (f64, f32)
