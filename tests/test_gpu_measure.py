"""The roofline denominators the library measures itself: each microbenchmark runs on every SM
and returns a rate within the range the B300's unit counts and clocks allow (148 SMs at up to
2,032 MHz: one 128-byte shared-memory wavefront, 128 fp32 fused multiply-adds and 16 population
counts per SM per clock)."""
import pytest

pytestmark = pytest.mark.gpu


def _ct():
    from paper_2606_28372_b300 import build as B
    B.build()
    from paper_2606_28372_b300 import catune as ct
    return ct


def _sms():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


CLOCK_MAX = 2.032e9


def test_smem_peak_is_one_wavefront_per_sm_clock_at_most():
    v = _ct().measure_smem_peak()
    top = _sms() * CLOCK_MAX
    assert 0.4 * top < v < 1.05 * top, v


def test_fp32_peak_is_within_the_fma_units():
    v = _ct().measure_fp32_peak()
    top = _sms() * 128 * 2 * CLOCK_MAX
    assert 0.4 * top < v < 1.05 * top, v


def test_int_peak_is_within_the_popc_units():
    v = _ct().measure_int_peak()
    top = _sms() * 16 * CLOCK_MAX
    assert 0.3 * top < v < 1.05 * top, v
