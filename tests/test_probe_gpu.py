"""The widening-multiply throughput probe (the measured denominator of the
forest fire's multiply roofline) returns a rate inside what the GPU can do:
between 0.1 and 4 warp instructions per SM-clock (the issue limit) at the
clocks this GPU reports, and about the same rate twice in a row."""
import pytest

pytestmark = pytest.mark.gpu


def test_mul_wide_probe_rate_is_plausible_and_repeatable():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1501_01405_gb300 as eng
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    max_hz = 2.2e9  # above any SM clock of this part
    a = eng.mrip_probe_mul_wide()
    b = eng.mrip_probe_mul_wide()
    assert 0.1 * sms * 1.0e9 < a < 4.0 * sms * max_hz
    assert abs(a - b) < 0.2 * a
