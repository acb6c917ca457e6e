"""The bench's JSON contract, checked on the CPU through its reference arm
(the oracle timed on the host cores; no GPU needed)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + list(args),
                          capture_output=True, text=True, cwd=ROOT, timeout=300)


def test_reference_arm_prints_one_contract_line():
    r = _run("--impl", "reference", "--workload", "mm1_32", "--steps", "1", "--warmup", "3",
             "--ref-seconds", "1")
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["unit"] == "replications/s" and d["n_gpus"] == 1
    assert d["steps"] == 1 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["vs_baseline"] is None and d["scaling"] == "weak"
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_fewer_than_three_warmup_steps_rejected():
    r = _run("--impl", "reference", "--workload", "mm1_32", "--steps", "1", "--warmup", "2")
    assert r.returncode != 0
    assert "warmup" in (r.stderr + r.stdout)


def test_shard_mode_splits_the_replications():
    """bench.py --shard: every rank runs its own contiguous replication range
    of the one experiment (same seed), the ranges cover every replication
    once, and the line's unit count is the whole experiment's."""
    sys.path.insert(0, ROOT)
    import bench
    for name in ("ff256", "ff128", "walk8", "tandem", "mm1_32"):
        world = 3
        ranges, full = [], None
        for r in range(world):
            wl = bench.make_workload(name, r)
            n_reps = wl.w["n_reps"]
            f = wl.shard(r, world)
            full = f if full is None else full
            assert f == wl.w["n_dp"] * n_reps
            assert wl.seed == wl.w["seed"]
            ranges.append((wl.rep0, wl.rep0 + wl.w["n_reps"]))
        assert ranges[0][0] == 0 and ranges[-1][1] == n_reps
        assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))


def test_multiply_count_per_lattice_word():
    """The forest-fire multiply roofline counts, per 32-cell lattice word and
    step, 8 Philox4x32-10 blocks of 20 widening multiplies less the 3 each
    that a step shares (round 1's product of the replication word, round 2's
    product of word 0) or a word shares (round 1's product of the block index,
    one per word for 8 blocks): 8 x 17 + 1."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.FF_MUL_WIDE_PER_WORD == 8 * (20 - 3) + 1
