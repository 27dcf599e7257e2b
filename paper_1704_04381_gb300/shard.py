"""Ensembles split over GPUs (one process per GPU).

Chains are independent and each chain's random numbers depend only on its
global index (Philox keyed by seed, chain, ensemble, step).  An ensemble can
therefore be split into contiguous chain ranges, one per rank, and grown with
no communication.  Only the statistics are exchanged at the end: the
rosen_stats of each rank (18 numbers), gathered and merged on the host in
fixed rank order.

The merge is the library's own (rosen_stats_merge, the reduction's tile
merge run on the host): the largest log W maximum M, each weighted sum
rescaled by exp(M_r - M) and each squared-weight sum by exp(2 (M_r - M)),
counts added, then Eq. 9's log Z, Eq. 2's means, their standard errors and
the ESS formed as rosen_reduce forms them.  The result equals a single
reduction over all chains up to FP64 rounding order.
"""
STAT_KEYS = ["n", "n_alive", "log_max", "S0", "S1", "S2", "Q0", "Q1_r2", "Q2_r2", "Q1_rg2",
             "Q2_rg2", "logZ", "logZ_norm", "mean_r2", "se_r2", "mean_rg2", "se_rg2", "ess"]


def chain_range(rank, world, C):
    """Contiguous chain range [chain0, chain0 + count) of `rank` out of `world`."""
    lo = C * rank // world
    hi = C * (rank + 1) // world
    return lo, hi - lo


def merge_stats(parts, N, k=0):
    """Merge rosen_stats dicts of disjoint chain sets (in the given order).

    N and k are the ensemble's monomers and trials per step (for logZ_norm).
    """
    from . import rosen
    return rosen.rosen_stats_merge(parts, N, k)


def gather_stats(stats, N, k=0, group=None):
    """All-gather every rank's statistics (a dict or 18-element sequence in
    STAT_KEYS order) and return their merge, identical on every rank."""
    import torch
    import torch.distributed as dist

    vec = [stats[key] for key in STAT_KEYS] if isinstance(stats, dict) else list(stats)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else "cpu"
    mine = torch.tensor(vec, dtype=torch.float64, device=dev)
    world = dist.get_world_size(group)
    got = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(got, mine, group=group)
    parts = [dict(zip(STAT_KEYS, t.cpu().tolist())) for t in got]
    return merge_stats(parts, N, k)


def max_over_ranks(value, group=None):
    """The largest of every rank's value (the job time of a weak-scaling step)."""
    import torch
    import torch.distributed as dist

    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
