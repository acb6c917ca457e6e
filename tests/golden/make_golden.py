"""Writes tests/golden/oracle_values.json from the oracle alone.

The paper prints no numeric results (its timing figures are not in the text),
so the stored values here are regression fixtures of the oracle: each entry
names the passage the oracle function follows.  tests/test_oracle_golden.py
recomputes them: integers bit for bit, floating point to a few ulps (the C
library's log may differ in the last bit between machines).  Regenerate only for a justified change of the oracle:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_values.json")


def build():
    g = {}
    ctr = np.array([[0, 0, 0, 0], [1, 2, 3, 4], [0xFFFFFFFF] * 4], dtype=np.uint32)
    key = np.array([[0, 0], [42, 0], [0xFFFFFFFF, 0xFFFFFFFF]], dtype=np.uint32)
    g["philox4x32_10"] = {
        "cite": "Salmon et al., SC'11 (Philox4x32-10); counter layout of the engine",
        "counter": ctr.tolist(), "key": key.tolist(),
        "words": oracle.philox4x32_10(ctr, key).astype(np.int64).tolist()}
    lo = np.array([0, 1, 0x12345678, 0xFFFFFFFF], dtype=np.uint32)
    hi = np.array([0, 0, 0x9ABCDEF0, 0xFFFFFFFF], dtype=np.uint32)
    rate = np.array([1.0, 0.9, 1.5, 2.0])
    u, e = oracle.u53_expo(lo, hi, rate)
    g["u53_expo"] = {"cite": "Section 5.1 (exponential arrival and service times), E = -log(1-u)/rate",
                     "lo": lo.tolist(), "hi": hi.tolist(), "rate": rate.tolist(),
                     "u": u.tolist(), "e": e.tolist()}
    w, i, v = oracle.mm1(np.array([[0.9, 1.0]]), [0, 0, 0], [0, 1, 31], 1000, 42)
    g["mm1"] = {"cite": "Section 5.1, second model (M/M/1 via the Lindley recurrence)",
                "dps": [[0.9, 1.0]], "reps": [0, 1, 31], "n_clients": 1000, "seed": 42,
                "wait": w.tolist(), "idle": i.tolist(), "system": v.tolist()}
    y, f = oracle.tandem3(np.array([[0.7, 1.1, 1.2, 1.3]]), [0, 0], [0, 5], 2000, 42, window=100)
    g["tandem3"] = {"cite": "three-station tandem of the engine's workloads (departure recurrence)",
                    "dps": [[0.7, 1.1, 1.2, 1.3]], "reps": [0, 5], "n_clients": 2000, "seed": 42,
                    "window": 100, "y": y.tolist(), "feat": f.tolist()}
    c, _ = oracle.forest_fire_rep(64, 100, 0.01, 1e-5, 0.5, 42, 0, 3)
    g["forest_fire"] = {"cite": "stochastic forest-fire automaton of the engine's workloads",
                        "L": 64, "n_steps": 100, "p": [0.01, 1e-5], "density": 0.5, "seed": 42,
                        "dp": 0, "rep": 3, "counts": c.tolist()}
    cs, _, ties = oracle.forest_fire_skip_rep(64, 100, 0.01, 1e-5, 0.5, 42, 0, 3)
    g["forest_fire_skip"] = {"cite": "skip-sampled variant (geometric gaps, tags 5 and 6)",
                             "L": 64, "n_steps": 100, "p": [0.01, 1e-5], "density": 0.5,
                             "seed": 42, "dp": 0, "rep": 3, "counts": cs.tolist(),
                             "near_ties": ties}
    tau = oracle.walk(np.array([16.0, 64.0]), [0, 1, 1], [0, 0, 7], 42)
    g["walk"] = {"cite": "Section 5.1, third model, adapted to an L1 exit time",
                 "radii": [16.0, 64.0], "dp": [0, 1, 1], "rep": [0, 0, 7], "seed": 42,
                 "tau": tau.tolist()}
    fa, vis = oracle.area_walk(np.array([0, 9]), 1000, 42)
    g["area_walk"] = {"cite": "Section 5.1, third model (30 areas), Section 5.3 (1,000 steps)",
                      "reps": [0, 9], "n_steps": 1000, "seed": 42, "final_area": fa.tolist(),
                      "visits": vis.tolist()}
    hits = oracle.pi_hits(np.array([0, 1]), 10**6, 42)
    g["pi"] = {"cite": "Section 5.1, first model (Monte Carlo pi)", "reps": [0, 1],
               "n_draws": 10**6, "seed": 42, "hits": hits.tolist()}
    g["t_crit"] = {"cite": "Section 1 (Student-t confidence interval); A&S 26.7.3/26.7.4",
                   "conf": 0.95, "df": [1, 2, 31, 255, 1023],
                   "t": [oracle.t_crit(0.95, d) for d in (1, 2, 31, 255, 1023)]}
    return g


if __name__ == "__main__":
    with open(OUT, "w") as fh:
        json.dump(build(), fh, indent=1)
        fh.write("\n")
    print(OUT)
