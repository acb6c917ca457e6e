"""The walk entry point that allocates nothing (GPU).

Some callers cannot call cudaMalloc -- a host framework or memory pool owns
every device allocation, or a latency-critical loop forbids an allocation
that may synchronize the device.  mrip_walk_simulate_noalloc serves them:
its scratch is a fixed array inside the library.  These checks call it
through the C ABI and compare it, twice in a row (the second call finds the
first call's leftovers in the shared array), with mrip_walk_simulate, which
allocates its scratch; walk times are integers, so the match is bit-exact.
The file sorts last so that a first-failure run has already run the rest.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_walk_matches_allocating_entry_point_twice():
    import torch
    assert torch.cuda.is_available(), "needs CUDA"
    import paper_1501_01405_gb300 as eng
    lib = eng.lib()
    stream = torch.cuda.current_stream()
    radii = np.array([16.0, 5.0, 33.0, 1.0, 64.0, 2.0])
    n_reps = 777
    n = radii.size * n_reps
    rp = radii.ctypes.data_as(ctypes.c_void_p)
    for seed, mapping in ((42, eng.MRIP_MAP_PERSISTENT), (43, eng.MRIP_MAP_PERSISTENT),
                          (44, eng.MRIP_MAP_WARP_COOP)):
        ref = torch.full((n,), -7, dtype=torch.int64, device="cuda")
        got = torch.full((n,), -9, dtype=torch.int64, device="cuda")
        eng.mrip_walk_simulate(radii, n_reps, seed, 1 << 38, mapping, ref, chunk=29)
        rc = lib.mrip_walk_simulate_noalloc(rp, radii.size, 0, n_reps, seed, 1 << 38, mapping, 0,
                                            0, 29, ctypes.c_void_p(got.data_ptr()),
                                            ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.mrip_last_error()
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
        assert int(got.min()) >= 1


def test_noalloc_walk_step_cap_then_reset():
    """A small step cap: capped replications read -1 exactly where the
    allocating entry point writes -1; the next call (no cap in reach) starts
    from a cleared ticket and flag and matches again."""
    import torch
    import paper_1501_01405_gb300 as eng
    lib = eng.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    radii = np.array([64.0, 8.0])
    rp = radii.ctypes.data_as(ctypes.c_void_p)
    n_reps = 300
    n = radii.size * n_reps
    for max_steps, rep0 in ((50, 0), (1 << 38, 1000)):
        ref = torch.full((n,), -7, dtype=torch.int64, device="cuda")
        got = torch.full((n,), -9, dtype=torch.int64, device="cuda")
        eng.mrip_walk_simulate(radii, n_reps, 42, max_steps, eng.MRIP_MAP_PERSISTENT, ref,
                               chunk=16, rep0=rep0)
        torch.cuda.synchronize()
        capped = max_steps < 1000
        if capped:  # the allocating path reports the cap through its flag
            with pytest.raises(eng.MripError) as e:
                eng.mrip_check_device_flags()
            assert e.value.code == 4
        rc = lib.mrip_walk_simulate_noalloc(rp, radii.size, rep0, n_reps, 42, max_steps,
                                            eng.MRIP_MAP_PERSISTENT, 0, 0, 16,
                                            ctypes.c_void_p(got.data_ptr()), stream)
        assert rc == 0, lib.mrip_last_error()
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
        g = got.cpu().numpy().reshape(2, n_reps)
        if capped:
            assert (g[0] == -1).all()  # R = 64 needs at least 64 moves
            assert ((g[1] == -1) | ((g[1] >= 8) & (g[1] <= 50))).all()
            assert (g[1] > 0).any()
        else:
            assert g.min() >= 8


def test_noalloc_walk_rejects_too_many_design_points():
    import torch
    import paper_1501_01405_gb300 as eng
    lib = eng.lib()
    radii = np.full(1025, 8.0)
    tau = torch.empty(1025, dtype=torch.int64, device="cuda")
    rc = lib.mrip_walk_simulate_noalloc(radii.ctypes.data_as(ctypes.c_void_p), 1025, 0, 1, 1, 100,
                                        0, 0, 0, 0, ctypes.c_void_p(tau.data_ptr()), None)
    assert rc == 1
    assert b"1024" in lib.mrip_last_error()
