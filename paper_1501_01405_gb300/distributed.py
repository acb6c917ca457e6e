"""Host-side helpers for running the engine on several GPUs, one process each.

Every replication is a pure function of (seed, design point, replication),
so ranks need no collective on the data path.  Two layouts are supported:

* independent batches (weak scaling): rank r runs the whole workload with
  seed + r; the only cross-rank operation is the max of the timed seconds;
* shards of one experiment: rank r runs the contiguous replication range
  shard_range(n_reps, r, world) through mrip_run_range (run_shard,
  sharded_stats); its per-design-point (n, mean, M2) triples
  are all-gathered (n_dp x 24 bytes per rank) and merged in rank order by
  mrip_stats_merge, which gives the same interval on every rank.

torch.distributed is the transport (NCCL on GPUs, gloo on CPUs).
"""
import numpy as np


def shard_range(n_reps, rank, world):
    """[lo, hi) replication range of `rank` (sizes differ by at most one)."""
    base, extra = divmod(int(n_reps), int(world))
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def max_over_ranks(value, device=None):
    """Max of a float over all ranks (the timing rule of the benchmark)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_merge_stats(nmm2, device=None):
    """All-gather each rank's (n_dp, 3) triples and merge them in rank order."""
    import torch
    import torch.distributed as dist
    from . import mrip_stats_merge
    local = np.ascontiguousarray(np.asarray(nmm2, dtype=np.float64).reshape(-1, 3))
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return mrip_stats_merge(local[None])
    t = torch.tensor(local, dtype=torch.float64, device=device)
    parts = [torch.empty_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, t)
    stacked = np.stack([p.cpu().numpy() for p in parts])
    return mrip_stats_merge(stacked)


def run_shard(model, design_points, n_reps, seed, rank, world):
    """Run this rank's replication range of one experiment through the engine
    (mrip_run_range) and return its per-design-point (n, mean, M2) triples."""
    lo, hi = shard_range(n_reps, rank, world)
    if hi <= lo:  # more ranks than replications: an empty part
        n_dp = np.asarray(design_points).shape[0]
        return np.zeros((n_dp, 3))
    model.run_range(design_points, lo, hi, seed)
    return model.moments()


def sharded_stats(model, design_points, n_reps, seed, conf=0.95, device=None):
    """Intervals of one experiment whose replications are split across the
    ranks of the process group: each rank runs its shard, the triples are
    all-gathered and merged in rank order, and every rank gets the same
    intervals (those of one run of all n_reps replications, up to the
    rounding of the merge)."""
    from . import mrip_stats_finalize
    rank, world = 0, 1
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        rank, world = dist.get_rank(), dist.get_world_size()
    local = run_shard(model, design_points, n_reps, seed, rank, world)
    merged = gather_merge_stats(local, device)
    return mrip_stats_finalize(merged, conf), merged


def collect_with_recovery(store, rank, world, local_nmm2, recompute, timeout_s=5.0):
    """Rank 0 collects every rank's triples from a key-value store
    (torch.distributed.Store) and merges them in rank order; a rank whose key
    has not appeared within `timeout_s` is treated as failed and its shard is
    recomputed locally with recompute(rank) -> (n_dp, 3) triples.  Other ranks
    only publish.  Returns (merged triples or None, list of failed ranks)."""
    import datetime
    local = np.ascontiguousarray(np.asarray(local_nmm2, dtype=np.float64).reshape(-1, 3))
    store.set("mrip/stats/%d" % rank, local.tobytes())
    if rank != 0:
        return None, []
    from . import mrip_stats_merge
    parts, failed = [], []
    for r in range(world):
        key = "mrip/stats/%d" % r
        try:
            store.wait([key], datetime.timedelta(seconds=timeout_s))
            parts.append(np.frombuffer(store.get(key), dtype=np.float64).reshape(-1, 3))
        except Exception:
            failed.append(r)
            parts.append(np.asarray(recompute(r), dtype=np.float64).reshape(-1, 3))
    return mrip_stats_merge(np.stack(parts)), failed
