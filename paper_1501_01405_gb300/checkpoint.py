"""Checkpoint and resume of an experiment run in replication ranges.

Every replication is a pure function of (seed, design point, replication
index), and per-design-point (n, mean, M2) triples merge associatively
(mrip_stats_merge), so the whole state of an unfinished experiment is small:
the design points, the seed, the model's fixed parameters, the replication
ranges already run and their triples.  Resuming runs the missing ranges
(mrip_run_range) and merges; the result is the one run of all replications
up to the rounding of the merge.  The ranges are merged in replication
order, so the result does not depend on the order in which they ran.
"""
import json
import os

import numpy as np


class Checkpoint:
    """The state of one experiment: n_reps replications of every design
    point, run in ranges [lo, hi)."""

    def __init__(self, kind, params, design_points, n_reps, seed):
        self.kind = int(kind)
        self.params = dict(params)
        self.dps = np.ascontiguousarray(np.asarray(design_points, dtype=np.float64))
        self.n_dp = self.dps.shape[0] if self.dps.ndim > 1 else self.dps.size
        self.n_reps = int(n_reps)
        self.seed = int(seed)
        self.done = {}  # lo -> (hi, triples (n_dp, 3))

    def add(self, lo, hi, triples):
        """Record the (n, mean, M2) triples of replications [lo, hi)."""
        lo, hi = int(lo), int(hi)
        if not (0 <= lo < hi <= self.n_reps):
            raise ValueError("range [%d, %d) outside 0..%d" % (lo, hi, self.n_reps))
        for a, (b, _) in self.done.items():
            if lo < b and a < hi:
                raise ValueError("range [%d, %d) overlaps [%d, %d)" % (lo, hi, a, b))
        t = np.asarray(triples, dtype=np.float64).reshape(self.n_dp, 3)
        if not np.all(t[:, 0] == hi - lo):
            raise ValueError("triples do not count hi - lo replications per design point")
        self.done[lo] = (hi, t.copy())

    def missing(self):
        """The replication ranges not run yet, in order."""
        out, at = [], 0
        for lo in sorted(self.done):
            if lo > at:
                out.append((at, lo))
            at = self.done[lo][0]
        if at < self.n_reps:
            out.append((at, self.n_reps))
        return out

    def complete(self):
        return not self.missing()

    def merged(self):
        """(n_dp, 3) triples of all ranges run so far, merged in replication order."""
        from . import mrip_stats_merge
        if not self.done:
            return np.zeros((self.n_dp, 3))
        parts = np.stack([self.done[lo][1] for lo in sorted(self.done)])
        return mrip_stats_merge(parts)

    def save(self, path):
        """Write the state as JSON (atomically: a temporary file, then rename)."""
        state = {"kind": self.kind, "params": self.params, "design_points": self.dps.tolist(),
                 "n_reps": self.n_reps, "seed": self.seed,
                 "done": [[lo, hi, t.tolist()] for lo, (hi, t) in sorted(self.done.items())]}
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(state, f)
        os.replace(tmp, path)

    @classmethod
    def load(cls, path):
        with open(path) as f:
            s = json.load(f)
        c = cls(s["kind"], s["params"], s["design_points"], s["n_reps"], s["seed"])
        for lo, hi, t in s["done"]:
            c.add(lo, hi, t)
        return c


def run_resumable(ckpt, chunk, path=None, model=None, max_chunks=None):
    """Run the checkpoint's missing replications in ranges of at most `chunk`
    per design point, recording (and, with `path`, saving) the state after
    each; stop after `max_chunks` ranges if given.  Returns the merged
    triples so far."""
    from . import Model
    own = model is None
    if own:
        model = Model(ckpt.kind, **ckpt.params)
    ran = 0
    try:
        for lo, hi in ckpt.missing():
            for a in range(lo, hi, chunk):
                if max_chunks is not None and ran >= max_chunks:
                    return ckpt.merged()
                b = min(a + chunk, hi)
                model.run_range(ckpt.dps, a, b, ckpt.seed)
                ckpt.add(a, b, model.moments())
                if path:
                    ckpt.save(path)
                ran += 1
    finally:
        if own:
            model.close()
    return ckpt.merged()
