"""hf_measure_unit_rates: the measured MUFU ex2 and FP32 FMA rates that the
benchmark reports beside its derived peaks.  Checked against the device's SM
count and the unit counts per SM (32 ex2 lanes -- GB300 doubles the 16 of
earlier parts -- and 128 FMA lanes) at its clock range: a measured rate may
not exceed the derived one at the maximum clock by more than rounding, nor
fall far below it."""

import pytest

pytestmark = pytest.mark.gpu


def test_unit_rates_match_the_unit_counts():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2201_10887_gb300 import hf
    props = torch.cuda.get_device_properties(0)
    r = hf.hf_measure_unit_rates()
    assert r["sms"] == props.multi_processor_count
    max_hz = 2.2e9  # above the part's maximum SM clock (2070 MHz)
    for key, lanes in (("ex2_per_s", 32), ("ffma_per_s", 128)):
        derived = lanes * r["sms"] * max_hz
        assert 0.3 * derived < r[key] <= 1.01 * derived, (key, r[key], derived)
