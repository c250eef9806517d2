"""og_measure_fp32_peak: the measured FP32 rate is positive and cannot exceed
the unit-count ceiling (SMs x 128 FP32 lanes x 2 flops x the highest SM
clock, 2070 MHz on GB300) by more than timing noise."""
from __future__ import annotations

import pytest

from paper_2609_17658_gb300 import build as B
from paper_2609_17658_gb300 import og

pytestmark = pytest.mark.gpu

MAX_SM_MHZ = 2070.0


def test_fp32_rate_is_below_the_unit_ceiling():
    torch = pytest.importorskip("torch")
    B.build()
    ctx = og.Context(0)
    try:
        r = og.og_measure_fp32_peak(ctx.h)
    finally:
        ctx.close()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ceiling = sms * 128 * 2 * MAX_SM_MHZ * 1e6 / 1e12
    for k in ("fma", "fma2"):
        assert 0.25 * ceiling < r[k] <= 1.03 * ceiling, (k, r[k], ceiling)


def test_fp32_rate_rejects_null():
    B.build()
    with pytest.raises(og.OGError) as e:
        og._check(og.lib().og_measure_fp32_peak(None, None, None))
    assert e.value.status == og.OG_ERR_ARG
