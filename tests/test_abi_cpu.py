"""The engine library loads and exports every entry point of include/mrip.h,
and its host-only entry points behave (CPU only; no kernel is launched).

* every function declared in the header is exported by libmrip.so;
* the host Student-t critical value equals the oracle's;
* mrip_stats_finalize (host) turns (n, mean, M2) into the oracle's interval;
* argument validation returns MRIP_EINVAL before any CUDA work.
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
import oracle.stats as ostats

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mrip.h")


def _engine():
    eng = pytest.importorskip("paper_1501_01405_gb300")
    try:
        eng.lib()
    except eng.MripLibraryMissing:
        from paper_1501_01405_gb300 import build
        build.build()
        eng.lib()
    return eng


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mrip_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("mrip_create_model", "mrip_run", "mrip_stats", "mrip_destroy",
                     "mrip_last_error", "mrip_mm1_simulate", "mrip_forest_fire_simulate",
                     "mrip_walk_simulate", "mrip_tandem3_simulate", "mrip_stats_reduce",
                     "mrip_mlp_loss_grad", "mrip_adam_step", "mrip_cv_reduce", "mrip_run_cv"):
        assert required in names


def test_library_exports_every_declared_symbol():
    eng = _engine()
    out = subprocess.run(["nm", "-D", "--defined-only", eng.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if " T " in l)
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    # the binding declares a signature for each of them
    from paper_1501_01405_gb300._abi import SIGNATURES
    assert sorted(SIGNATURES) == _declared()


@pytest.mark.parametrize("df", [1, 2, 3, 4, 9, 31, 127, 229, 255, 1023, 4095, 2**17 - 1])
@pytest.mark.parametrize("conf", [0.9, 0.95, 0.99])
def test_t_crit_matches_oracle(df, conf):
    eng = _engine()
    got = eng.mrip_t_crit(conf, df)
    ref = oracle.t_crit(conf, df)
    assert got == pytest.approx(ref, rel=2e-15)


def test_stats_finalize_matches_oracle():
    eng = _engine()
    rng = np.random.default_rng(3)
    rows = [rng.normal(5, 2, size=n) for n in (2, 3, 32, 256)]
    nmm2 = []
    for r in rows:
        m = r.mean()
        nmm2 += [len(r), m, float(((r - m) ** 2).sum())]
    got = eng.mrip_stats_finalize(np.array(nmm2), 0.95)
    for g, r in zip(got, rows):
        ref = ostats.ci(r, 0.95)
        assert g["n"] == ref["n"]
        assert g["half_width"] == pytest.approx(ref["half_width"], rel=1e-13)
        assert g["t_crit"] == pytest.approx(ref["t_crit"], rel=1e-14)
    one = eng.mrip_stats_finalize(np.array([1.0, 7.0, 0.0]), 0.95)[0]
    assert one["n"] == 1 and one["mean"] == 7.0 and np.isnan(one["half_width"])


def test_invalid_arguments_rejected_on_host():
    eng = _engine()
    with pytest.raises(eng.MripError) as e:
        eng.mrip_create_model(eng.MRIP_FOREST_FIRE, L=100, n_steps=10, density=0.5, window=5)
    assert e.value.code == 1
    with pytest.raises(eng.MripError):
        eng.mrip_create_model(eng.MRIP_MM1, n_clients=0)
    with pytest.raises(eng.MripError):
        eng.mrip_create_model(eng.MRIP_WALK_L1_EXIT, max_steps=1 << 40)
    with pytest.raises(eng.MripError):
        eng.mrip_t_crit(1.5, 3)
    L = eng.lib()
    # stage entry points validate sizes before touching the device
    assert L.mrip_mm1_simulate(None, -1, 0, 1, 1, 0, 0, None, None, None, None) == 1
    assert L.mrip_forest_fire_simulate(None, 1, 0, 1, 100, 10, 0.5, 0, None, None, None, None,
                                       None) == 1
    r = (ctypes.c_double * 1)(2.5)
    assert L.mrip_walk_simulate(r, 1, 0, 4, 0, 100, 0, 0, 0, 0, ctypes.c_void_p(16), None) == 1
    assert b"integer" in L.mrip_last_error()
    # replication ranges: indices must stay below 2^32, rep0 >= 0
    assert L.mrip_mm1_simulate(None, 1, (1 << 32) - 1, 2, 10, 0, 0, None, None, None, None) == 1
    assert b"2^32" in L.mrip_last_error()
    assert L.mrip_pi_simulate(-1, 1, 10, 0, None, None) == 1
    assert L.mrip_area_walk_simulate(1 << 32, 1, 10, 0, 0, None, None, None) == 1
    assert L.mrip_forest_fire_skip_simulate(None, 1, -3, 1, 32, 10, 0.5, 0, None, None, None,
                                            None, None) == 1
    assert L.mrip_walk_simulate_noalloc(r, 1, 1 << 32, 4, 0, 100, 0, 0, 0, 0,
                                        ctypes.c_void_p(16), None) == 1
    m = eng.Model(eng.MRIP_MM1, n_clients=10)
    for lo, hi in ((5, 5), (7, 3), (-1, 4), (0, (1 << 32) + 1)):
        with pytest.raises(eng.MripError) as e:
            m.run_range([[0.5, 1.0]], lo, hi, 42)
        assert e.value.code == 1
    m.close()


def test_plan_json_round_trip_and_rejection():
    eng = _engine()
    m = eng.Model(eng.MRIP_WALK_L1_EXIT, max_steps=1 << 30)
    m.set_plan('{"mapping": 5, "warps_per_cta": 8, "ctas_per_sm": 2, "chunk": 64}')
    assert m.get_plan() == '{"mapping": 5, "warps_per_cta": 8, "ctas_per_sm": 2, "chunk": 64}'
    with pytest.raises(eng.MripError):
        m.set_plan('{"mapping": 5, "bogus": 1}')
    with pytest.raises(eng.MripError):
        m.set_plan('{"mapping": 4}')  # CTA mapping is for lattices
    q = eng.Model(eng.MRIP_MM1, n_clients=10)
    with pytest.raises(eng.MripError):
        q.stats()
    m.close()
    q.close()


def test_cv_and_training_arguments_rejected_on_host():
    """mrip_run_cv and mrip_mlp_train validate their parameters before any
    device work: a bad training fraction, validation fraction, patience or
    control-run count, too few held-out or fit replications, a model kind
    without a control variate; a bad network size, minibatch or resume
    epoch."""
    eng = _engine()
    dps = [[0.9, 1.0, 1.1, 1.2]]
    m = eng.Model(eng.MRIP_TANDEM3, n_clients=50, window=10)
    bad = [dict(train_frac=0.0), dict(train_frac=1.0), dict(val_frac=1.0), dict(val_frac=-0.1),
           dict(patience=-1), dict(m_ctrl=1), dict(epochs=0), dict(batch=0), dict(conf=1.0)]
    for kw in bad:
        with pytest.raises(eng.MripError) as e:
            m.run_cv(dps, 40, 7, **kw)
        assert e.value.code == 1, kw
    with pytest.raises(eng.MripError) as e:  # 4 replications: 1 training, 3 held-out, 0 fit left
        m.run_cv(dps, 4, 7, train_frac=0.25, val_frac=0.5)
    assert e.value.code == 1 and b"fit" in eng.lib().mrip_last_error()
    with pytest.raises(eng.MripError) as e:
        m.cv_network()
    assert e.value.code == 5  # no control-variate run yet
    m.close()
    w = eng.Model(eng.MRIP_WALK_L1_EXIT, max_steps=1 << 20)
    with pytest.raises(eng.MripError) as e:
        w.run_cv([[8.0]], 40, 7)
    assert e.value.code == 6
    w.close()
    L = eng.lib()
    from paper_1501_01405_gb300 import _abi
    prm = _abi.mrip_train_params(batch=64, epochs=1, patience=0, max_steps=0, lr=1e-3, beta1=0.9,
                                 beta2=0.999, eps=1e-8, order_seed=1, epoch0=0)
    p16 = ctypes.c_void_p(16)
    assert L.mrip_mlp_train(9, p16, p16, 10, None, None, 0, ctypes.byref(prm), p16, None, None,
                            None, None, None, None, None, None, None) == 1
    for field, value in (("batch", 0), ("epochs", 0), ("epoch0", -1), ("lr", 0.0), ("beta2", 1.0)):
        q = _abi.mrip_train_params.from_buffer_copy(prm)
        setattr(q, field, value)
        assert L.mrip_mlp_train(8, p16, p16, 10, None, None, 0, ctypes.byref(q), p16, None, None,
                                None, None, None, None, None, None, None) == 1, field
    # a validation set needs its pointers
    assert L.mrip_mlp_train(8, p16, p16, 10, None, None, 5, ctypes.byref(prm), p16, None, None,
                            None, None, None, None, None, None, None) == 1


def test_release_library_has_no_debug_checks():
    eng = _engine()
    assert eng.mrip_debug_checks() == (False, None)
    assert eng.lib().mrip_debug_selftest() == 1  # MRIP_EINVAL: not a debug build


def test_debug_variant_builds_and_exports_every_symbol():
    """The bounds-checked variant (-DMRIP_DEBUG) compiles for sm_103a and
    exports the same entry points; it is only run on a GPU."""
    eng = _engine()
    from paper_1501_01405_gb300 import build
    path = build.build(variant="debug")
    assert path != eng.library_path() and os.path.exists(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if " T " in l)
    assert not [n for n in _declared() if n not in exported]
    eng.load_library(path)  # loads beside the release library
