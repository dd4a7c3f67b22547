"""The roofline ceilings the library measures (ceiling_measure) are positive and ordered as the
hardware orders them.

Bounds are loose on purpose, since the clock varies from box to box. Packed and scalar FP32 FMAs
each reach at least a quarter of the nominal FP32 rate (SMs x 128 lanes x 2 flops x 2.07 GHz)
and at most 1.5 times it. L1-resident 8-byte loads are at least as fast as L2-resident ones,
and L2-resident loads move at least 1 TB/s. Each kind also runs through the Python binding.
"""
import pytest
import torch

import paper_1403_4209_gb300 as wg

pytestmark = pytest.mark.gpu


def test_ceilings_plausible():
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sms * 128 * 2 * 2.07e9
    c = {k: wg.ceiling(k) for k in ("fp32_fma2", "fp32_fma", "fetch_l1", "fetch_l2", "shared")}
    print("\nceilings:", {k: "%.3g" % v for k, v in c.items()})
    for k in ("fp32_fma2", "fp32_fma"):
        assert 0.25 * nominal < c[k] < 1.5 * nominal, (k, c[k], nominal)
    assert c["fetch_l2"] > 1e12
    assert c["fetch_l1"] >= 0.9 * c["fetch_l2"]
    assert c["shared"] > 1e12
