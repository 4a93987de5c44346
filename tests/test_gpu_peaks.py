"""The pipe-rate microbenchmarks behind the roofline fractions run and give
plausible rates (bounded by the nominal unit counts at the device's clock)."""
import pytest

import gpu_util as G

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_plausible():
    torch = G.torch_cuda()
    _lib = G.lib()
    pk = _lib.petfmm_measure_peaks()
    sms = pk["sms"]
    assert sms == torch.cuda.get_device_properties(0).multi_processor_count
    # 128 FP32 lanes per SM at no more than 2.2 GHz; at least a third of that
    fp32_max = sms * 128 * 2.2e9
    assert fp32_max / 3 < pk["fp32_ops"] <= fp32_max * 1.01
    assert 0 < pk["fp64_ops"] < pk["fp32_ops"]
    assert 0 < pk["mufu_rcp_ops"] < pk["fp32_ops"]
    assert 0 < pk["mufu_ex2_ops"] < pk["fp32_ops"]
    # dense TF32 on the tensor cores: far above the SIMT FP32 rate
    assert pk["tf32_flops"] > 2 * 2 * pk["fp32_ops"]
