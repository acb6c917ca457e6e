"""The oracle against its stored values (tests/golden/oracle_values.json,
written by tests/golden/make_golden.py from the oracle alone).

The paper prints no numbers to compare with, so these fixtures guard the
oracle itself: a change of its arithmetic, its build flags or its random
streams shows here, and must be justified before the fixtures are rewritten.
"""
import json
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_values.json")


def load():
    with open(GOLDEN) as fh:
        return json.load(fh)


def test_philox_and_variates():
    g = load()
    p = g["philox4x32_10"]
    words = oracle.philox4x32_10(np.array(p["counter"], dtype=np.uint32), np.array(p["key"], dtype=np.uint32))
    assert words.astype(np.int64).tolist() == p["words"]
    e = g["u53_expo"]
    u, x = oracle.u53_expo(np.array(e["lo"], dtype=np.uint32), np.array(e["hi"], dtype=np.uint32),
                           np.array(e["rate"]))
    assert u.tolist() == e["u"]
    np.testing.assert_allclose(x, e["e"], rtol=4e-16, atol=0)


def test_models():
    g = load()
    m = g["mm1"]
    w, i, v = oracle.mm1(np.array(m["dps"]), [0] * len(m["reps"]), m["reps"], m["n_clients"], m["seed"])
    for a, b in ((w, m["wait"]), (i, m["idle"]), (v, m["system"])):
        np.testing.assert_allclose(a, b, rtol=1e-14, atol=0)
    t = g["tandem3"]
    y, f = oracle.tandem3(np.array(t["dps"]), [0] * len(t["reps"]), t["reps"], t["n_clients"], t["seed"],
                          window=t["window"])
    np.testing.assert_allclose(y, t["y"], rtol=1e-14, atol=0)
    np.testing.assert_allclose(f, t["feat"], rtol=1e-14, atol=0)
    ff = g["forest_fire"]
    c, _ = oracle.forest_fire_rep(ff["L"], ff["n_steps"], *ff["p"], ff["density"], ff["seed"], ff["dp"], ff["rep"])
    assert c.tolist() == ff["counts"]
    fs = g["forest_fire_skip"]
    c, _, ties = oracle.forest_fire_skip_rep(fs["L"], fs["n_steps"], *fs["p"], fs["density"], fs["seed"],
                                             fs["dp"], fs["rep"])
    assert c.tolist() == fs["counts"] and ties == fs["near_ties"]
    wk = g["walk"]
    tau = oracle.walk(np.array(wk["radii"]), wk["dp"], wk["rep"], wk["seed"])
    assert tau.tolist() == wk["tau"]
    aw = g["area_walk"]
    fa, vis = oracle.area_walk(np.array(aw["reps"]), aw["n_steps"], aw["seed"])
    assert fa.tolist() == aw["final_area"] and vis.tolist() == aw["visits"]
    pi = g["pi"]
    assert oracle.pi_hits(np.array(pi["reps"]), pi["n_draws"], pi["seed"]).tolist() == pi["hits"]


def test_t_critical_values():
    g = load()["t_crit"]
    np.testing.assert_allclose([oracle.t_crit(g["conf"], d) for d in g["df"]], g["t"], rtol=1e-15, atol=0)
