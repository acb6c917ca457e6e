#!/usr/bin/env python
"""Benchmark of the MRIP engine: one JSON line on stdout (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--impl engine|reference]

A step is one pass of the hot path over one batch of synthetic input: all
replications of the workload simulated by the CUDA kernels and reduced to
per-design-point (n, mean, M2) on the device.  The default workload is the
largest configuration, the 256x256 forest fire with 64 design points
(ff256: 128 replications each x 2,000 steps); the line also carries the
replications/s of the other configurations (mm1_32, ff128, walk8, tandem;
"configs") and the plain-vs-control-variate time to the target half-width
on the tandem and ff256 workloads ("time_to_target").  Other workloads are
selectable: mm1_32 (latency; its step replays as one CUDA graph), mm1_64k
(throughput), walk8, tandem, ff128, ff128_skip / ff256_skip (skip-sampled
lattice events), area_walk and pi (the paper's own models; --sweep times
them against the replication count).

value   = replications / s over the K timed steps, inputs resident in HBM,
          device time from CUDA events on the launching stream, L2 flushed
          (256 MiB write) between steps outside the timed intervals.
e2e     = the same through the public model-handle API (mrip_run with the
          design points in pinned host memory + mrip_stats reading the
          intervals back), wall time.
roofline= the dominant kernel's algorithmic work per launch / its mean event
          time.  Lattices: integer instructions per cell-update against the
          issue rate (SMs x 4 warp instructions per clock x maximum SM clock),
          with the integer-multiply unit beside it ("alt"); the other models
          against the nominal integer-multiply rate: every model is bound by
          Philox's 32x32->64 products, not by HBM or the tensor cores.
cpu_baseline = the oracle (plain C) on a bounded sample of the same workload
          on all host cores (rank 0, N = 1 only).

With --impl reference the oracle itself is timed as the reference arm.
Under torchrun (N > 1) every rank runs its own batch (seed + rank: weak
scaling, no collective on the data path); the time is the max over ranks.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import mrip_inputs  # noqa: E402

METRIC = ("replications/sec and time to target 95% CI half-width, plain vs control-variate")
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")

# Nominal unit counts (per SM per clock) used for the ALU rooflines.
SMS = 152
SM_MAX_MHZ = 2070.0
IMUL_PER_CLK_SM = 64      # 32-bit integer multiply / multiply-add results
DFMA_PER_CLK_SM = 2       # FP64 fused multiply-add results (1.25 TFLOP/s nominal)
INT_MULS_PER_PHILOX = 40  # 10 rounds x 2 products x (low + high half)
# one gap of the skip-sampled lattice: half a Philox block (20) + the
# fixed-point log's seven 64x64-bit products, each four 32-bit products (28)
MULS_PER_GAP = 48
# one exponential variate in 48-bit fixed point: the log's products (26: the
# 64x64-bit m * 1/c and r^2, the 32-bit tail, n ln 2) + the 64x64-bit scaling
# by 2^-9 / rate (8)
MULS_PER_FIXED_VARIATE = 34


# DRAM bytes (read + write) per launch of a dominant kernel, from the ncu
# capture summarised in profiles/ (None once the kernel changes).  The 256^2
# kernel was captured on 4 of its 128 replications per design point (256 of
# 8,192 CTAs: 37,888 B read, 0 written during the launch -- per-CTA design
# points, constants and code; the counts stay in L2) and is scaled by the
# replications of a full launch (x32).
PROFILED_TRAFFIC = {"forest_fire_kernel<8>": 399360 * 32}


# Issue slots: 4 schedulers per SM, one warp instruction each per clock.
ISSUE_PER_CLK_SM = 4
# Integer instructions per forest-fire cell-update: a quarter of a
# Philox4x32-10 block (15-20 integer instructions) plus the bit-parallel
# rule (32 cells per word); the midpoint 17.5 is the algorithmic figure.
FF_INSTR_PER_CELL = 17.5
FF_MUL_WIDE_PER_WORD = 137  # widening multiplies per 32-cell lattice word and step


def issue_peak_g():
    """Warp instructions per second (G) at the maximum SM clock."""
    return SMS * ISSUE_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e9


def imul_peak_gops():
    return SMS * IMUL_PER_CLK_SM * SM_MAX_MHZ * 1e6 / 1e9


# ---------------------------------------------------------------------------
# workloads: device state, one step, the dominant kernel, the oracle sample
# ---------------------------------------------------------------------------
class Workload:
    name = ""
    units_name = "replications"
    dtype = ""
    rep0 = 0  # first replication of this rank's shard (sharded mode)

    def __init__(self, rank):
        self.rank = rank

    def config(self):
        raise NotImplementedError

    def shard(self, rank, world):
        """Run only this rank's replication range of the one experiment
        (same seed on every rank); returns the experiment's replication
        count over all design points."""
        from paper_1501_01405_gb300.distributed import shard_range
        full = self.units()
        lo, hi = shard_range(self.w["n_reps"], rank, world)
        if hi <= lo:
            raise SystemExit("--shard: more ranks than replications")
        self.w["n_reps"] = hi - lo
        self.rep0 = lo
        self.seed = self.w["seed"]
        return full


class ForestFire(Workload):
    dtype = "u32"

    def __init__(self, rank, key="ff128"):
        super().__init__(rank)
        self.key = key
        self.w = mrip_inputs.workload(key)
        self.name = key
        self.seed = self.w["seed"] + rank

    def units(self):
        return self.w["n_dp"] * self.w["n_reps"]

    def config(self):
        w = self.w
        return {"workload": "%s: forest fire %dx%d, %d steps, %d design point(s) x %d "
                            "replications, density %.2f" % (self.key, w["L"], w["L"], w["n_steps"],
                                                             w["n_dp"], w["n_reps"], w["density"]),
                "L": w["L"], "n_steps": w["n_steps"], "n_dp": w["n_dp"], "n_reps": w["n_reps"],
                "p_grow": float(w["dps"][0, 0]), "p_lightning": float(w["dps"][0, 1]),
                "seed": self.seed, "mapping": "CTA per replication, bit-packed rows"}

    def setup(self, eng, torch):
        w = self.w
        self.eng, self.torch = eng, torch
        self.d_dps = torch.tensor(w["dps"], dtype=torch.float64, device="cuda")
        n = self.units()
        self.counts = torch.empty(n * w["n_steps"], dtype=torch.int32, device="cuda")
        self.scalar = torch.empty(n, dtype=torch.float64, device="cuda")
        self.nmm2 = torch.empty(w["n_dp"] * 3, dtype=torch.float64, device="cuda")

    def step(self, k_start=None, k_end=None):
        w = self.w
        if k_start is not None:
            k_start.record()
        self.eng.mrip_forest_fire_simulate(self.d_dps, w["n_reps"], w["L"], w["n_steps"],
                                           w["density"], self.seed, None, self.counts,
                                           self.scalar, rep0=self.rep0)
        if k_end is not None:
            k_end.record()
        self.eng.mrip_stats_reduce(self.scalar.view(w["n_dp"], w["n_reps"]), self.nmm2)

    launches_per_step = 2

    def roofline_work(self):
        w = self.w
        cells = w["L"] * w["L"] * w["n_steps"] * self.units()
        alt = dict(unit="Gop/s (32-bit integer multiply)",
                   work=cells * INT_MULS_PER_PHILOX / 4.0, peak=imul_peak_gops(),
                   peak_source="nominal: %d SMs x %d int-mul/clk x %.0f MHz" % (
                       SMS, IMUL_PER_CLK_SM, SM_MAX_MHZ),
                   per_unit="10 int multiplies per cell-update (1/4 Philox block)")
        return dict(kernel="forest_fire_kernel<%d>" % (w["L"] // 32), bound="alu",
                    unit="G warp-instructions/s",
                    work=cells * FF_INSTR_PER_CELL / 32.0, peak=issue_peak_g(),
                    peak_source="issue slots: %d SMs x %d warp-instr/clk x %.0f MHz" % (
                        SMS, ISSUE_PER_CLK_SM, SM_MAX_MHZ),
                    per_unit="%.1f integer instructions per cell-update (1/4 Philox4x32-10 "
                             "block + the bit-parallel rule), 32 per warp instruction"
                             % FF_INSTR_PER_CELL, alt=alt,
                    mul_wide=dict(work=cells * FF_MUL_WIDE_PER_WORD / 32.0 / 32.0,
                                  per_unit="%d widening multiplies per 32-cell word and step (8 "
                                           "Philox blocks x 17, two per-step products shared, "
                                           "+ 1), 32 per warp instruction" % FF_MUL_WIDE_PER_WORD))

    def extra_rates(self, reps_per_s, torch):
        w = self.w
        cells = float(w["L"] * w["L"] * w["n_steps"])
        # algorithmic HBM traffic: the int32 burning count of every step and the
        # FP64 scalar per replication written, the design points read
        bytes_per_rep = 4.0 * w["n_steps"] + 8.0 + 16.0 / w["n_reps"]
        return {"cell_updates_per_s": reps_per_s * cells,
                "hbm_gbs_algorithmic": reps_per_s * bytes_per_rep / 1e9,
                "hbm_note": "low by construction: the lattice lives in shared memory"}

    def make_model(self):
        w = self.w
        m = self.eng.Model(self.eng.MRIP_FOREST_FIRE, L=w["L"], n_steps=w["n_steps"],
                           density=w["density"], window=min(100, w["n_steps"]))
        return m

    def e2e_inputs(self):
        return self.w["dps"], self.w["n_reps"]

    def oracle_sample(self, n_items, threads):
        import oracle
        w = self.w
        rep = np.arange(n_items) % w["n_reps"]
        dp = (np.arange(n_items) // w["n_reps"]) % w["n_dp"]
        oracle.forest_fire(w["L"], w["n_steps"], w["dps"], w["density"], dp.astype(np.int32),
                           rep, self.seed, threads=threads)


class ForestFireSkip(ForestFire):
    """The forest-fire workload with skip-sampled events (same rules, same
    initial state; each step draws p L^2 gaps instead of L^2 words)."""

    def config(self):
        c = super().config()
        c["workload"] = c["workload"].replace("forest fire", "forest fire, skip-sampled events")
        c["mapping"] = "CTA per replication, bit-packed rows, all warps draw the event gaps"
        return c

    def step(self, k_start=None, k_end=None):
        w = self.w
        if k_start is not None:
            k_start.record()
        self.eng.mrip_forest_fire_skip_simulate(self.d_dps, w["n_reps"], w["L"], w["n_steps"],
                                                w["density"], self.seed, None, self.counts,
                                                self.scalar, rep0=self.rep0)
        if k_end is not None:
            k_end.record()
        self.eng.mrip_stats_reduce(self.scalar.view(w["n_dp"], w["n_reps"]), self.nmm2)

    def roofline_work(self):
        w = self.w
        cells = float(w["L"] * w["L"])
        p = np.asarray(w["dps"], dtype=np.float64)
        gaps_per_step = (p[:, 0] + p[:, 1]).mean() * cells + 2.0
        gaps = gaps_per_step * w["n_steps"] * self.units()
        return dict(kernel="forest_fire_skip_kernel<%d>" % (w["L"] // 32), bound="alu",
                    unit="Gop/s (32-bit integer multiply)",
                    work=gaps * MULS_PER_GAP, peak=imul_peak_gops(),
                    peak_source="nominal: %d SMs x %d int-mul/clk x %.0f MHz" % (
                        SMS, IMUL_PER_CLK_SM, SM_MAX_MHZ),
                    per_unit="%d int multiplies per gap (half a Philox block + the fixed-point log); "
                             "(p_grow + p_light) L^2 + 2 gaps per step" % MULS_PER_GAP)

    def make_model(self):
        return None

    def outputs(self):
        return [self.counts, self.scalar]

    def oracle_sample(self, n_items, threads):
        import oracle
        w = self.w
        rep = np.arange(n_items) % w["n_reps"]
        dp = (np.arange(n_items) // w["n_reps"]) % w["n_dp"]
        oracle.forest_fire_skip(w["L"], w["n_steps"], w["dps"], w["density"], dp.astype(np.int32),
                                rep, self.seed, threads=threads)


class Walk(Workload):
    dtype = "i32"

    def __init__(self, rank):
        super().__init__(rank)
        self.w = mrip_inputs.workload("walk8")
        self.name = "walk8"
        self.seed = self.w["seed"] + rank
        self.radii = self.w["dps"][:, 0].copy()

    def units(self):
        return self.w["n_dp"] * self.w["n_reps"]

    def config(self):
        w = self.w
        return {"workload": "walk8: L1-exit walk, R in %s, %d replications each" % (
            list(mrip_inputs.WALK_RADII), w["n_reps"]), "n_dp": w["n_dp"], "n_reps": w["n_reps"],
                "seed": self.seed, "mapping": "persistent work stealing, lane refill"}

    def setup(self, eng, torch):
        self.eng, self.torch = eng, torch
        n = self.units()
        self.tau = torch.empty(n, dtype=torch.int64, device="cuda")
        self.nmm2 = torch.empty(len(self.radii) * 3, dtype=torch.float64, device="cuda")

    def step(self, k_start=None, k_end=None):
        if k_start is not None:
            k_start.record()
        self.eng.mrip_walk_simulate(self.radii, self.w["n_reps"], self.seed, 1 << 38,
                                    self.eng.MRIP_MAP_PERSISTENT, self.tau, rep0=self.rep0)
        if k_end is not None:
            k_end.record()
        self.eng.mrip_stats_reduce_i64(self.tau.view(len(self.radii), self.w["n_reps"]), self.nmm2)

    launches_per_step = 3  # walk, statistics over slices, slice merge

    def extra_rates(self, reps_per_s, torch):
        moves = float(self.tau.double().sum().item())  # every replication's exit time
        return {"moves_per_s": reps_per_s * moves / self.units(), "moves_per_step": moves}

    def roofline_work(self):
        moves = 0.0
        for R in mrip_inputs.WALK_RADII:
            moves += self.w["n_reps"] * (2.0 / 3.0) * R * R
        return dict(kernel="walk_persistent_kernel", bound="alu",
                    unit="Gop/s (32-bit integer multiply)", work=moves / 64.0 * INT_MULS_PER_PHILOX,
                    peak=imul_peak_gops(), peak_source="nominal int-mul rate",
                    per_unit="40 int multiplies per 64 moves (one Philox block); E[tau] ~ 2R^2/3")

    def make_model(self):
        return self.eng.Model(self.eng.MRIP_WALK_L1_EXIT, max_steps=1 << 38)

    def e2e_inputs(self):
        return self.w["dps"], self.w["n_reps"]

    def oracle_sample(self, n_items, threads):
        import oracle
        w = self.w
        g = np.arange(n_items)
        dp = (g % w["n_dp"]).astype(np.int32)
        rep = g // w["n_dp"]
        oracle.walk(self.radii, dp, rep, self.seed, threads=threads)


def stats_launches(n_reps):
    """Kernels of one statistics reduction: slices of 4,096 replications are
    merged by a second kernel."""
    return 2 if n_reps > 4096 else 1


class Queue(Workload):
    dtype = "f64"

    def __init__(self, rank, key):
        super().__init__(rank)
        self.key = key
        if key in ("mm1_32", "mm1_64k"):
            self.w = mrip_inputs.workload(key)
        else:
            self.w = mrip_inputs.workload("tandem_cv")
        self.name = key
        self.seed = self.w["seed"] + rank

    def units(self):
        return self.w["n_dp"] * self.w["n_reps"]

    def config(self):
        w = self.w
        if self.key == "mm1_64k":
            return {"workload": "mm1_64k: M/M/1 Lindley, lambda 0.9, mu 1, 1000 clients, 65536 "
                                "replications", "n_reps": w["n_reps"], "n_clients": w["n_clients"],
                    "seed": self.seed, "mapping": "thread per replication, 48-bit fixed-point times"}
        if self.key == "mm1_32":
            return {"workload": "mm1_32: M/M/1 Lindley, lambda 0.9, mu 1, 1000 clients, 32 "
                                "replications", "n_reps": w["n_reps"], "n_clients": w["n_clients"],
                    "seed": self.seed, "mapping": "CTA per replication, block scan of max-plus "
                                                  "maps, 48-bit fixed-point times",
                    "launch": "each step (simulate + statistics) replayed as one CUDA graph"}
        return {"workload": "tandem: 3-station tandem, %d design points x %d replications x %d "
                            "clients (plain estimator)" % (w["n_dp"], w["n_reps"], w["n_clients"]),
                "n_dp": w["n_dp"], "n_reps": w["n_reps"], "n_clients": w["n_clients"],
                "seed": self.seed, "mapping": "thread per replication"}

    def setup(self, eng, torch):
        self.eng, self.torch = eng, torch
        w = self.w
        n = self.units()
        self.d_dps = torch.tensor(w["dps"], dtype=torch.float64, device="cuda")
        self.y = torch.empty(n, dtype=torch.float64, device="cuda")
        self.feat = torch.empty(8 * n, dtype=torch.float64, device="cuda") \
            if self.key == "tandem" else None
        self.nmm2 = torch.empty(w["n_dp"] * 3, dtype=torch.float64, device="cuda")

    def step(self, k_start=None, k_end=None):
        w = self.w
        if k_start is not None:
            k_start.record()
        if self.key in ("mm1_32", "mm1_64k"):
            mapping = self.eng.MRIP_MAP_CTA if self.key == "mm1_32" else self.eng.MRIP_MAP_THREAD
            self.eng.mrip_mm1_simulate(self.d_dps, w["n_reps"], w["n_clients"], self.seed,
                                       mapping, self.y, rep0=self.rep0)
        else:
            self.eng.mrip_tandem3_simulate(self.d_dps, self.rep0, w["n_reps"], w["n_clients"],
                                           w["window"], self.seed, 0, self.eng.MRIP_MAP_THREAD,
                                           self.y, self.feat)
        if k_end is not None:
            k_end.record()
        self.eng.mrip_stats_reduce(self.y.view(w["n_dp"], w["n_reps"]), self.nmm2)

    @property
    def launches_per_step(self):
        return 1 + stats_launches(self.w["n_reps"])

    def extra_rates(self, reps_per_s, torch):
        clients = reps_per_s * self.w["n_clients"]
        return {"clients_per_s": clients,
                "exponential_variates_per_s": clients * (4 if self.key == "tandem" else 2)}

    @property
    def graph_step(self):
        return self.key == "mm1_32"

    def roofline_work(self):
        w = self.w
        clients = self.units() * w["n_clients"]
        blocks = 2 if self.key == "tandem" else 1
        logs = 4 if self.key == "tandem" else 2
        per_client = blocks * INT_MULS_PER_PHILOX + logs * MULS_PER_FIXED_VARIATE
        kernel = {"mm1_32": "mm1_cta_kernel (graph with the statistics kernel)",
                  "mm1_64k": "mm1_serial_kernel", "tandem": "tandem3_serial_kernel"}[self.key]
        return dict(kernel=kernel, bound="alu",
                    unit="Gop/s (32-bit integer multiply)", work=clients * per_client,
                    peak=imul_peak_gops(),
                    peak_source="nominal: %d SMs x %d int-mul/clk x %.0f MHz" % (
                        SMS, IMUL_PER_CLK_SM, SM_MAX_MHZ),
                    per_unit="%d int multiplies per client: %d Philox block(s) (40 each) + %d "
                             "fixed-point variates (%d each: log 26, scaling 8)" % (
                                 per_client, blocks, logs, MULS_PER_FIXED_VARIATE))

    def make_model(self):
        w = self.w
        if self.key in ("mm1_32", "mm1_64k"):
            m = self.eng.Model(self.eng.MRIP_MM1, n_clients=w["n_clients"])
            mapping = self.eng.MRIP_MAP_CTA if self.key == "mm1_32" else self.eng.MRIP_MAP_THREAD
            m.set_plan('{"mapping": %d}' % mapping)
            return m
        return self.eng.Model(self.eng.MRIP_TANDEM3, n_clients=w["n_clients"],
                              window=w["window"])

    def e2e_inputs(self):
        return self.w["dps"], self.w["n_reps"]

    def oracle_sample(self, n_items, threads):
        import oracle
        w = self.w
        g = np.arange(n_items)
        dp = (g % w["n_dp"]).astype(np.int32)
        rep = (g // w["n_dp"]) % w["n_reps"]
        if self.key in ("mm1_32", "mm1_64k"):
            oracle.mm1(w["dps"], dp, rep, w["n_clients"], self.seed, threads=threads)
        else:
            oracle.tandem3(w["dps"], dp, rep, w["n_clients"], self.seed, window=w["window"],
                           threads=threads)


class AreaWalk(Workload):
    """The paper's walk (30 areas, 1,000 moves) mapped one replication per thread."""
    dtype = "i32"

    def __init__(self, rank, n_reps=1 << 16, n_steps=1000, mapping="THREAD"):
        super().__init__(rank)
        self.w = dict(n_reps=n_reps, n_steps=n_steps, n_dp=1, dps=np.zeros((1, 1)), kind="area_walk")
        self.name = "area_walk"
        self.seed = mrip_inputs.SEED + rank
        self.mapping = mapping

    def units(self):
        return self.w["n_reps"]

    def config(self):
        return {"workload": "area_walk: the paper's 30-area random walk (60x50 periodic map, "
                            "10x10 areas), %d moves, %d replications" % (self.w["n_steps"], self.w["n_reps"]),
                "n_reps": self.w["n_reps"], "n_steps": self.w["n_steps"], "seed": self.seed,
                "mapping": self.mapping}

    def setup(self, eng, torch):
        self.eng, self.torch = eng, torch
        n = self.w["n_reps"]
        self.fa = torch.empty(n, dtype=torch.int32, device="cuda")
        self.vis = torch.empty(30 * n, dtype=torch.int32, device="cuda")

    def step(self, k_start=None, k_end=None):
        if k_start is not None:
            k_start.record()
        self.eng.mrip_area_walk_simulate(self.w["n_reps"], self.w["n_steps"], self.seed,
                                         getattr(self.eng, "MRIP_MAP_" + self.mapping), self.fa, self.vis)
        if k_end is not None:
            k_end.record()

    launches_per_step = 1

    def roofline_work(self):
        moves = float(self.w["n_reps"]) * self.w["n_steps"]
        return dict(kernel="area_walk_serial_kernel", bound="alu", unit="Gop/s (32-bit integer multiply)",
                    work=moves / 64.0 * INT_MULS_PER_PHILOX, peak=imul_peak_gops(),
                    peak_source="nominal int-mul rate",
                    per_unit="40 int multiplies per 64 moves (one Philox block)")

    def make_model(self):
        return None

    def outputs(self):
        return [self.fa, self.vis]

    def oracle_sample(self, n_items, threads):
        import oracle
        oracle.area_walk(np.arange(n_items) % self.w["n_reps"], self.w["n_steps"], self.seed,
                         threads=threads)


class MonteCarloPi(Workload):
    """The paper's first model: pi from the share of 10^7 random points per
    replication that fall in the quarter disc; 256 replications."""
    dtype = "u32"

    def __init__(self, rank, n_reps=256, n_draws=10**7):
        super().__init__(rank)
        self.w = dict(n_reps=n_reps, n_draws=n_draws, n_dp=1, dps=np.zeros((1, 1)), kind="pi")
        self.name = "pi"
        self.seed = mrip_inputs.SEED + rank

    def units(self):
        return self.w["n_reps"]

    def config(self):
        return {"workload": "pi: Monte Carlo pi, %d draws per replication, %d replications"
                            % (self.w["n_draws"], self.w["n_reps"]),
                "n_reps": self.w["n_reps"], "n_draws": self.w["n_draws"], "seed": self.seed}

    def setup(self, eng, torch):
        self.eng, self.torch = eng, torch
        self.hits = torch.empty(self.w["n_reps"], dtype=torch.int64, device="cuda")

    def step(self, k_start=None, k_end=None):
        if k_start is not None:
            k_start.record()
        self.eng.mrip_pi_simulate(self.w["n_reps"], self.w["n_draws"], self.seed, self.hits)
        if k_end is not None:
            k_end.record()

    launches_per_step = 1  # plus the clearing memset of the counters

    def roofline_work(self):
        draws = float(self.w["n_reps"]) * self.w["n_draws"]
        return dict(kernel="pi_kernel", bound="alu", unit="Gop/s (32-bit integer multiply)",
                    work=draws * (INT_MULS_PER_PHILOX + 4) / 2.0, peak=imul_peak_gops(),
                    peak_source="nominal int-mul rate",
                    per_unit="22 int multiplies per draw (half a Philox block + two 32x32->64 squares)")

    def make_model(self):
        return None

    def outputs(self):
        return [self.hits]

    def oracle_sample(self, n_items, threads):
        import oracle
        oracle.pi_hits(np.arange(n_items) % self.w["n_reps"], self.w["n_draws"], self.seed, threads=threads)


def pi_sweep(eng, torch, n_draws=10**7, runs=7):
    """Time per launch (median of `runs`, CUDA events) for 1 .. 256
    replications of 10^7 draws, and the oracle's time per replication on one
    core: the paper's GPU-versus-CPU curve for this model (Section 5.2)."""
    import oracle
    out = {"n_draws": n_draws, "reps": [], "ms": []}
    for n in list(range(1, 9)) + [16, 32, 64, 65, 128, 152, 153, 256]:
        hits = torch.empty(n, dtype=torch.int64, device="cuda")
        times = []
        for r in range(runs + 1):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            eng.mrip_pi_simulate(n, n_draws, 42, hits)
            e1.record()
            torch.cuda.synchronize()
            if r:
                times.append(e0.elapsed_time(e1))
        out["reps"].append(n)
        out["ms"].append(float(np.median(times)))
    t0 = time.perf_counter()
    oracle.pi_hits(np.arange(4), n_draws, 42, threads=1)
    out["cpu_ms_per_rep_one_core"] = (time.perf_counter() - t0) / 4 * 1e3
    return out


def mm1_sweep(eng, torch, runs=5):
    """M/M/1 (lambda 0.9, mu 1) mappings against the replication count and
    length: time per launch (median of `runs`, CUDA events)."""
    d = torch.tensor([[0.9, 1.0]], dtype=torch.float64, device="cuda")
    out = {"cases": [], "ms": {"THREAD": [], "WARP_1LANE": [], "WARP_COOP": [], "CTA": []}}
    for n_reps, n_clients in ((1, 10**5), (32, 1000), (32, 10**4), (1024, 1000), (1 << 16, 1000)):
        w = torch.empty(n_reps, dtype=torch.float64, device="cuda")
        out["cases"].append([n_reps, n_clients])
        for mp in out["ms"]:
            if mp == "WARP_1LANE" and n_reps > 1024:
                out["ms"][mp].append(None)
                continue
            times = []
            for r in range(runs + 1):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                eng.mrip_mm1_simulate(d, n_reps, n_clients, 42, getattr(eng, "MRIP_MAP_" + mp), w)
                e1.record()
                torch.cuda.synchronize()
                if r:
                    times.append(e0.elapsed_time(e1))
            out["ms"][mp].append(float(np.median(times)))
    return out


def tandem_sweep(eng, torch, n_clients=10**5, runs=5):
    """Few replications of a long horizon: time per launch (median of `runs`,
    CUDA events) of each tandem mapping for 1 .. 16,384 replications of
    10^5 clients at one design point (lambda 0.9, mu 1.0, 1.1, 1.2)."""
    out = {"n_clients": n_clients, "reps": [],
           "ms": {"THREAD": [], "WARP_1LANE": [], "WARP_COOP": [], "CTA": []}}
    dps = torch.tensor([[0.9, 1.0, 1.1, 1.2]], dtype=torch.float64, device="cuda")
    for k in range(0, 15, 2):
        n = 1 << k
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        out["reps"].append(n)
        for mp in out["ms"]:
            if mp == "WARP_1LANE" and n > 1024:
                out["ms"][mp].append(None)
                continue
            times = []
            for r in range(runs + 1):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                eng.mrip_tandem3_simulate(dps, 0, n, n_clients, 100, 42, 0, getattr(eng, "MRIP_MAP_" + mp),
                                          y, None)
                e1.record()
                torch.cuda.synchronize()
                if r:
                    times.append(e0.elapsed_time(e1))
            out["ms"][mp].append(float(np.median(times)))
    return out


def area_walk_sweep(eng, torch, n_steps=1000, runs=7):
    """Time per launch (median of `runs`, CUDA events) of each mapping for
    1 .. 2^16 replications, and the oracle's time per replication on one
    core: the GPU-versus-CPU and WLP-versus-TLP comparisons of the paper
    (Section 5.2-5.3), re-measured."""
    import oracle
    out = {"n_steps": n_steps, "reps": [], "ms": {"THREAD": [], "WARP_1LANE": [], "WARP_COOP": []}}
    maps = list(out["ms"])
    for k in range(17):
        n = 1 << k
        fa = torch.empty(n, dtype=torch.int32, device="cuda")
        vis = torch.empty(30 * n, dtype=torch.int32, device="cuda")
        out["reps"].append(n)
        for mp in maps:
            times = []
            for r in range(runs + 1):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                eng.mrip_area_walk_simulate(n, n_steps, 42, getattr(eng, "MRIP_MAP_" + mp), fa, vis)
                e1.record()
                torch.cuda.synchronize()
                if r:
                    times.append(e0.elapsed_time(e1))
            out["ms"][mp].append(float(np.median(times)))
    t0 = time.perf_counter()
    oracle.area_walk(np.arange(2000), n_steps, 42, threads=1)
    out["cpu_ms_per_rep_one_core"] = (time.perf_counter() - t0) / 2000 * 1e3
    i64 = out["reps"].index(64)
    out["wlp_over_tlp_time_at_64"] = out["ms"]["WARP_1LANE"][i64] / out["ms"]["THREAD"][i64]
    return out


def shrink(wl, n):
    """A smaller case of the same kernel for profiling captures."""
    w = wl.w
    if w["dps"].shape[0] > 1 and w.get("kind") == "tandem3":
        w["dps"] = np.ascontiguousarray(w["dps"][:n])
        w["n_dp"] = w["dps"].shape[0]
    else:
        w["n_reps"] = n
    wl.w = w


def make_workload(name, rank):
    if name in ("ff128", "ff256"):
        return ForestFire(rank, "ff128" if name == "ff128" else "ff256_cv")
    if name in ("ff128_skip", "ff256_skip"):
        return ForestFireSkip(rank, "ff128" if name == "ff128_skip" else "ff256_cv")
    if name == "walk8":
        return Walk(rank)
    if name in ("mm1_32", "mm1_64k", "tandem"):
        return Queue(rank, name)
    if name == "area_walk":
        return AreaWalk(rank)
    if name == "pi":
        return MonteCarloPi(rank)
    raise SystemExit("unknown workload %s" % name)


# ---------------------------------------------------------------------------
# time to a target interval half-width, plain vs learned control variate
# ---------------------------------------------------------------------------
CV_DEFAULTS = dict(train_frac=0.1, val_frac=0.1, epochs=20, patience=3, batch=1024, lr=1e-3,
                   gate=True, m_ctrl=0)
PHASES = ("ms_simulate", "ms_train", "ms_control", "ms_infer", "ms_estimate")


def _median_hw(stats):
    return float(np.median([s["half_width"] for s in stats]))


def time_to_target(eng, torch, stream, seed, which="tandem_cv"):
    """Tandem workload (4,096 design points x 10,000 clients, 256
    replications) or the 256x256 forest fire (64 design points x 2,000 steps,
    128 replications): the target is the median plain 95 % half-width at
    n_reps replications, which the plain estimator reaches by definition in
    the time of that run.  The control-variate estimator (mrip_run_cv:
    network on 10 % of the replications with a 10 % validation split and
    early stopping, control runs sized from the validation rho^2, the gate
    on) is run at n_reps; if it declines, its result is the plain interval
    and its time that of the whole call; otherwise its replication count is
    scaled by (half-width ratio)^2 and it is run again at that count.  Every
    run is timed end to end (wall clock around the synchronous call) and
    carries the library's CUDA-event breakdown of its phases."""
    w = mrip_inputs.workload(which)
    n_reps = w["n_reps"]
    if which == "tandem_cv":
        model = eng.Model(eng.MRIP_TANDEM3, n_clients=w["n_clients"], window=w["window"])
        label = ("tandem_cv: 3-station tandem, 4096 design points, 10000 clients, %d replications, "
                 "network 8-64-64-1 on 10 percent of replications" % n_reps)
    else:
        model = eng.Model(eng.MRIP_FOREST_FIRE, L=w["L"], n_steps=w["n_steps"], density=w["density"],
                          window=w["window"])
        label = ("ff256_cv: forest fire 256x256, 64 design points, 2000 steps, %d replications, "
                 "network 6-64-64-1 on 10 percent of replications" % n_reps)
    model.set_stream(stream)

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    def cv_run(n):
        return model.run_cv(w["dps"], n, seed, **CV_DEFAULTS)

    def summary(n, secs, cv, rep):
        d = {"replications": n, "seconds": secs, "median_half_width": _median_hw(cv),
             "declined": rep["declined"], "val_rho2": rep["val_rho2"],
             "var_ratio_predicted": rep["var_ratio"], "control_runs_per_dp": rep["m_ctrl"],
             "epochs_run": rep["epochs_run"], "best_epoch": rep["best_epoch"],
             "train_loss": rep["train_loss"], "val_loss": rep["val_loss"]}
        d["phases_ms"] = {k[3:]: rep[k] for k in PHASES}
        return d

    model.run(w["dps"], n_reps, seed)  # warm (graph capture, allocations)
    model.stats()
    _, t_plain = timed(lambda: (model.run(w["dps"], n_reps, seed), model.stats()))
    plain = model.stats()
    target = _median_hw(plain)
    cv_run(n_reps)  # warm
    (pl, cv, rep), t_cv0 = timed(lambda: cv_run(n_reps))
    at_n = summary(n_reps, t_cv0, cv, rep)
    if rep["declined"]:
        final, t_cv, n_need = at_n, t_cv0, n_reps
    else:
        hw0 = _median_hw(cv)
        n_held0 = cv[0]["n"]
        n_need = max(n_reps // 8, int(math.ceil(n_held0 * (hw0 / target) ** 2
                                                 / (1 - CV_DEFAULTS["train_frac"]))))
        (pl2, cv2, rep2), t_cv = timed(lambda: cv_run(n_need))
        final = summary(n_need, t_cv, cv2, rep2)
    # the break-even rho^2: with this run's overhead (everything but the
    # plain simulation), M sized for a tenth of the residual variance and
    # 10 % of the replications spent on training, the control variate reaches
    # the plain half-width in the plain time when (1 - rho^2) 1.1 / 0.9 =
    # 1 - overhead / simulation
    ph = at_n["phases_ms"]
    t_sim = ph["simulate"]
    over = sum(v for k, v in ph.items() if k != "simulate")
    rho2_be = 1.0 - (1.0 - over / t_sim) * (1 - CV_DEFAULTS["train_frac"]) / 1.1 if t_sim > 0 else None
    model.close()
    return {"workload": label,
            "target_half_width": target,
            "plain": {"replications": n_reps, "seconds": t_plain, "median_half_width": target},
            "cv_at_same_replications": at_n,
            "cv": final,
            "cv_over_plain_time": t_cv / t_plain,
            "break_even_val_rho2": rho2_be,
            "note": "declined: the gate returned the plain interval (the plain estimator is the "
                    "fallback), so the time above is the plain run plus training and validation"
            if final["declined"] else "accepted: control runs and inference included"}


def config_rates(eng, torch, steps=5, warmup=3):
    """replications/s of the other configurations (device time, CUDA events,
    L2 flushed between steps): M/M/1 (32 replications, one CUDA graph per
    step; and 2^16 replications, the throughput row), the 128^2 forest fire,
    the walk batch and the plain tandem, each with its dominant kernel's
    roofline fraction over the whole step's time."""
    out = {}
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    for name in ("mm1_32", "mm1_64k", "ff128", "walk8", "tandem"):
        wl = make_workload(name, 0)
        wl.setup(eng, torch)
        step = wl.step
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        graph = None
        if getattr(wl, "graph_step", False):
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                wl.step()
            torch.cuda.synchronize()
            step = graph.replay
            for _ in range(warmup):
                step()
            torch.cuda.synchronize()
        n = steps if name != "mm1_32" else 50
        ms = []
        for i in range(n):
            flush.fill_(float(i))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            step()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        t = sum(ms) / len(ms)
        rw = wl.roofline_work()
        ach = rw["work"] / (t / 1e3) / 1e9  # the whole step's time: a lower bound
        out[name] = {"replications_per_s": wl.units() / (t / 1e3), "ms_per_step": t,
                     "steps": n, "workload": wl.config()["workload"],
                     "roofline": {"kernel": rw["kernel"], "bound": rw["bound"], "unit": rw["unit"],
                                  "achieved": ach, "peak": rw["peak"], "frac": ach / rw["peak"],
                                  "per_unit": rw["per_unit"], "timed": "whole step"}}
        del graph
    return out


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def time_oracle(wl, target_s, threads):
    """Run the oracle on a sample sized to about target_s seconds on `threads`
    cores; returns (items, seconds)."""
    import oracle
    oracle.lib()
    n = threads
    t0 = time.perf_counter()
    wl.oracle_sample(n, threads)
    dt = time.perf_counter() - t0
    while dt < 0.5 and n < 10**7:  # calibrate on cheap workloads
        n *= 4
        t0 = time.perf_counter()
        wl.oracle_sample(n, threads)
        dt = time.perf_counter() - t0
    per_item = dt / n
    m = max(threads, int(target_s / per_item) // threads * threads)
    t0 = time.perf_counter()
    wl.oracle_sample(m, threads)
    return m, time.perf_counter() - t0


def reference_arm(args, wl, rank, world):
    import oracle
    if rank != 0:
        return
    threads = oracle.host_threads()
    oracle.lib()
    # size each step so the whole run stays within about three minutes (--ref-seconds)
    per_step = max(0.2, min(8.0, args.ref_seconds / max(1, args.steps + args.warmup)))
    n_cal = threads
    t0 = time.perf_counter()
    wl.oracle_sample(n_cal, threads)
    dt = time.perf_counter() - t0
    while dt < 0.3 and n_cal < 10**7:
        n_cal *= 4
        t0 = time.perf_counter()
        wl.oracle_sample(n_cal, threads)
        dt = time.perf_counter() - t0
    m = max(threads, int(per_step / (dt / n_cal)) // threads * threads)
    for _ in range(args.warmup):
        wl.oracle_sample(m, threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        wl.oracle_sample(m, threads)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = m * len(times) / total
    sample = "%d replications per step of %s (the workload has %d)" % (m, wl.name, wl.units())
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": "replications/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": wl.dtype, "data": "synthetic", "config": wl.config(),
            "cpu_baseline": {"value": value, "unit": "replications/s", "cores": threads,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "replications/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def e2e_model(wl, model, stream, torch, steps, barrier, world, total_units, sharded=False):
    """mrip_run with host design points + mrip_stats reading the intervals back;
    sharded: mrip_run_range over this rank's replications, mrip_moments, and
    the triples all-gathered and merged (every rank gets the intervals of the
    whole experiment)."""
    import torch.distributed as dist
    from paper_1501_01405_gb300.distributed import gather_merge_stats
    model.set_stream(stream)
    dps, n_reps = wl.e2e_inputs()
    # the step's inputs live in pinned host memory (a numpy view of it: the
    # C ABI takes a plain host pointer)
    dps = torch.tensor(np.ascontiguousarray(dps, dtype=np.float64)).pin_memory().numpy()

    def one():
        if sharded:
            model.run_range(dps, wl.rep0, wl.rep0 + n_reps, wl.seed)
            return gather_merge_stats(model.moments(), device="cuda")
        model.run(dps, n_reps, wl.seed)
        return model.stats(0.95)
    for _ in range(3):
        one()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize()
    barrier()
    e2e_s = time.perf_counter() - t0
    if world > 1:
        tt = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_s = float(tt.item())
    model.close()
    return {"value": total_units / e2e_s, "unit": "replications/s",
            "h2d_bytes_per_step": int(np.asarray(dps).nbytes),
            "d2h_bytes_per_step": int(np.asarray(dps).shape[0] * 3 * 8)}


def e2e_stage(wl, torch, steps, barrier, world):
    """Stage entry point per step, then a device-to-host copy of its outputs
    into pinned memory (the step's result)."""
    import torch.distributed as dist
    dev = wl.outputs()
    host = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in dev]
    for _ in range(3):
        wl.step()
        for h, d in zip(host, dev):
            h.copy_(d)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        wl.step()
        for h, d in zip(host, dev):
            h.copy_(d)
    torch.cuda.synchronize()
    barrier()
    e2e_s = time.perf_counter() - t0
    if world > 1:
        tt = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_s = float(tt.item())
    return {"seconds": e2e_s, "unit": "replications/s", "h2d_bytes_per_step": 0,
            "d2h_bytes_per_step": int(sum(h.numel() * h.element_size() for h in host))}


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="ff256",
                    choices=["ff128", "ff256", "ff128_skip", "ff256_skip", "walk8", "mm1_32", "mm1_64k", "tandem",
                             "area_walk", "pi"])
    ap.add_argument("--sweep", action="store_true",
                    help="area_walk: time every mapping for 1 .. 2^16 replications; "
                         "pi: time 1 .. 256 replications; tandem: mappings for 1 .. 16,384 "
                         "replications of 10^5 clients; mm1_32: M/M/1 mappings")
    ap.add_argument("--impl", default="engine", choices=["engine", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-dp", type=int, default=0,
                    help="profiling only: keep the first N design points (tandem) or use N "
                         "replications per design point (other workloads)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=150.0,
                    help="--impl reference: host seconds for the whole run (each step 0.2 .. 8 s)")
    ap.add_argument("--no-cv", action="store_true",
                    help="skip the plain-vs-control-variate time-to-target measurement")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the replications/s of the other configurations")
    ap.add_argument("--shard", action="store_true",
                    help="under torchrun: split the replications of one experiment across the "
                         "ranks (strong scaling) instead of one batch per rank")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    wl = make_workload(args.workload, rank)
    if args.n_dp > 0:
        shrink(wl, args.n_dp)
    full_units = wl.shard(rank, world) if args.shard else None

    if args.impl == "reference":
        reference_arm(args, wl, rank, world)
        return

    import torch
    import torch.distributed as dist
    import paper_1501_01405_gb300 as eng
    eng.lib()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    if args.sweep:
        sweeps = {"area_walk": area_walk_sweep, "pi": pi_sweep, "tandem": tandem_sweep,
                  "mm1_32": mm1_sweep}
        if args.workload not in sweeps:
            raise SystemExit("--sweep applies to --workload area_walk, pi, tandem or mm1_32")
        if rank == 0:
            print(json.dumps({"metric": METRIC, "sweep": sweeps[args.workload](eng, torch),
                              "config": wl.config()}), flush=True)
        return
    wl.setup(eng, torch)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")  # 256 MiB > L2
    for _ in range(args.warmup):
        wl.step()
    torch.cuda.synchronize()
    if getattr(wl, "graph_step", False):
        # latency-bound steps: replay the step's launches as one CUDA graph, so
        # the device time is not the host's launch rate
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            wl.step()
        torch.cuda.synchronize()

        def graph_step_fn(k_start=None, k_end=None):
            if k_start is not None:
                k_start.record()
            graph.replay()
            if k_end is not None:
                k_end.record()
        wl.step = graph_step_fn
        for _ in range(args.warmup):
            wl.step()
        torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ke = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))  # outside the timed interval
        starts[i].record(stream)
        wl.step(ks[i], ke[i])
        ends[i].record(stream)
    torch.cuda.synchronize()
    barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    dev_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    kern_ms = [s.elapsed_time(e) for s, e in zip(ks, ke)]
    if world > 1:
        tt = torch.tensor([dev_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        dev_ms = float(tt.item())
    total_units = (full_units if args.shard else wl.units() * world) * args.steps
    value = total_units / (dev_ms / 1e3)

    # ---- end to end through the public API, host buffers
    model = wl.make_model()
    if model is None:  # stage entry point: launch, then read the outputs back
        e2e = e2e_stage(wl, torch, args.steps, barrier, world)
    else:
        e2e = e2e_model(wl, model, stream, torch, args.steps, barrier, world, total_units,
                        sharded=args.shard)
    if model is None:
        e2e["value"] = total_units / e2e.pop("seconds")
    # ---- roofline of the dominant kernel
    rw = wl.roofline_work()
    kmean = sum(kern_ms) / len(kern_ms)
    achieved = rw["work"] / (kmean / 1e3) / 1e9
    roof = {"bound": rw["bound"], "kernel": rw["kernel"], "achieved": achieved,
            "peak": rw["peak"], "unit": rw["unit"],
            "frac": (achieved / rw["peak"]) if rw["peak"] else None,
            "traffic": PROFILED_TRAFFIC.get(rw["kernel"]) if args.n_dp == 0 else None,
            "kernel_ms": kmean, "per_unit": rw["per_unit"],
            "peak_source": rw["peak_source"]}
    if "mul_wide" in rw:  # the binding unit against its rate measured on this GPU, now
        mw = rw["mul_wide"]
        m_ach = mw["work"] / (kmean / 1e3) / 1e9
        m_peak = wl.eng.mrip_probe_mul_wide() / 1e9
        roof["measured_unit"] = {"unit": "G warp widening-multiplies/s", "achieved": m_ach,
                                 "peak": m_peak, "frac": m_ach / m_peak,
                                 "per_unit": mw["per_unit"],
                                 "peak_source": "measured by mrip_probe_mul_wide after the timed "
                                                "steps (every SM full of independent chains)"}
    if "alt" in rw:
        alt = rw["alt"]
        a_ach = alt["work"] / (kmean / 1e3) / 1e9
        roof["alt"] = {"achieved": a_ach, "peak": alt["peak"], "unit": alt["unit"],
                       "frac": a_ach / alt["peak"], "per_unit": alt["per_unit"],
                       "peak_source": alt["peak_source"]}

    line = {"metric": METRIC, "value": value, "unit": "replications/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dev_ms / args.steps,
            "higher_is_better": True, "scaling": "strong" if args.shard else "weak",
            "vs_baseline": None,
            "dtype": wl.dtype, "data": "synthetic (seeded Philox streams)",
            "config": dict(wl.config(), l2="flushed between timed steps (256 MiB write)",
                           parallelism=("one experiment, replications split over %d ranks "
                                        "(mrip_run_range shards, triples merged)" % world)
                           if args.shard else "replicas x%d (independent seeds)" % world),
            "roofline": roof, "e2e": e2e, "clocks": clk,
            "gpu_launches": wl.launches_per_step * args.steps,
            "wall_s": t_wall}

    extra = wl.extra_rates(value, torch) if hasattr(wl, "extra_rates") else None
    if extra:
        line["rates"] = extra
    if rank == 0 and world == 1 and not args.no_cv:
        line["time_to_target"] = {
            "tandem_cv": time_to_target(eng, torch, stream, 42, which="tandem_cv"),
            "ff256_cv": time_to_target(eng, torch, stream, 42, which="ff256_cv")}
    if rank == 0 and world == 1 and not args.no_configs and args.workload == "ff256":
        line["configs"] = config_rates(eng, torch)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        threads = oracle.host_threads()
        n, s = time_oracle(wl, args.cpu_seconds, threads)
        n1, s1 = time_oracle(wl, max(1.0, args.cpu_seconds / 4), 1)
        line["cpu_baseline"] = {"value": n / s, "unit": "replications/s", "cores": threads,
                                "kind": "oracle",
                                "sample": "%d replications of %s in %.1f s" % (n, wl.name, s),
                                "single_thread": {"value": n1 / s1, "unit": "replications/s",
                                                  "sample": "%d replications in %.1f s" % (n1, s1)}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
