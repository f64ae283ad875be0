"""The latency probe the ring's hop time is compared with, and the multiply
rate probe the factor roofline uses: both run, finish and give values in the
range the hardware allows (a GPU clock is near 2 GHz: one L2 round trip is
hundreds of cycles, not single cycles nor milliseconds)."""
import pytest

from paper_1505_07368_gb300 import cafgpu as C

pytestmark = pytest.mark.gpu


def test_latency_probe_values_are_plausible():
    import torch
    torch.cuda.set_device(0)
    lat = C.measure_latency()
    for k in ("atomic_ns", "load_acquire_ns", "store_fence_sc_ns", "handoff_ns"):
        assert 20.0 < lat[k] < 20000.0, (k, lat)
    # a flag handoff between SMs needs at least one L2 round trip
    assert lat["handoff_ns"] >= 0.5 * lat["load_acquire_ns"], lat
    print("\nLATENCY", lat)


def test_mul_rate_probe_orders():
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    r = C.measure_mul_rates()
    per_sm_clk = {k: v / sms / 2.07e9 for k, v in r.items()}
    # 32-bit multiplies: at most 64 per SM per clock; the high multiply is slower
    assert 8 < per_sm_clk["mul_lo_per_s"] <= 70, per_sm_clk
    assert per_sm_clk["mul_hi_per_s"] < per_sm_clk["mul_lo_per_s"], per_sm_clk
