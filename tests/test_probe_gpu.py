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


def test_forest_fire_multiply_count_stays_under_the_measured_rate():
    """The bench's multiply roofline for the 256^2 forest fire counts 137
    widening multiplies per lattice word and step; over a timed launch that
    count must come out below the probe's measured rate (a count too high, or
    a kernel not doing the work, would show above it) and not far below it."""
    import numpy as np
    import torch
    import mrip_inputs
    import paper_1501_01405_gb300 as eng
    w = mrip_inputs.workload("ff256_cv")
    dps = torch.tensor(w["dps"], device="cuda")
    n_reps, L, T = 16, 256, 2000
    counts = torch.empty(64 * n_reps * T, dtype=torch.int32, device="cuda")
    run = lambda: eng.mrip_forest_fire_simulate(dps, n_reps, L, T, w["density"], 42,  # noqa: E731
                                                counts=counts)
    run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    run()
    e1.record()
    torch.cuda.synchronize()
    seconds = e0.elapsed_time(e1) / 1e3
    words = 64 * n_reps * (L * L // 32) * T
    achieved = 137 * words / 32 / seconds
    peak = eng.mrip_probe_mul_wide()
    assert 0.4 < achieved / peak < 1.02, (achieved, peak)
    assert np.all(counts.cpu().numpy() >= 0)
