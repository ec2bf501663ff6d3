"""The FMA-throughput probe that the arithmetic rooflines divide by."""
import pytest

from paper_1911_10747_gb300 import lbm

pytestmark = pytest.mark.gpu


def test_fma_probe_measures_a_plausible_rate_and_restores_the_device():
    import torch
    dev = torch.cuda.current_device()
    props = torch.cuda.get_device_properties(dev)
    f32 = lbm.peak_fma(32, iters=2048)
    f64 = lbm.peak_fma(64, iters=256)
    # 128 FP32 lanes per SM at no more than 3 GHz bounds the FP32 rate from
    # above; FP64 runs at a fraction of FP32 on this part
    assert 0.2 * props.multi_processor_count * 128 * 2 * 1.0e9 / 1e12 < f32 < \
        props.multi_processor_count * 128 * 2 * 3.0e9 / 1e12
    assert 0.0 < f64 < f32
    assert torch.cuda.current_device() == dev
