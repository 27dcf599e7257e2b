"""Ensembles split over GPUs (one process per GPU).

Chains are independent and each chain's random numbers depend only on its
global index (Philox keyed by seed, chain, ensemble, step).  An ensemble can
therefore be split into contiguous chain ranges, one per rank, and grown with
no communication.  Only the statistics are exchanged at the end: the
rosen_stats of each rank (18 numbers), gathered and merged on the host in
fixed rank order.

The merge is the reduction's own tile merge:
- M = max of the ranks' log W maxima;
- each weighted sum is rescaled by exp(M_r - M), and each squared-weight sum
  by exp(2 (M_r - M));
- counts add.
The derived quantities (Eq. 9's log Z, Eq. 2's means, their standard errors
and the ESS) are then formed as rosen_reduce forms them.  The result equals a
single reduction over all chains up to FP64 rounding order.
"""
import math

STAT_KEYS = ["n", "n_alive", "log_max", "S0", "S1", "S2", "Q0", "Q1_r2", "Q2_r2", "Q1_rg2",
             "Q2_rg2", "logZ", "logZ_norm", "mean_r2", "se_r2", "mean_rg2", "se_rg2", "ess"]
_FIRST = ("S0", "S1", "S2")
_SECOND = ("Q0", "Q1_r2", "Q2_r2", "Q1_rg2", "Q2_rg2")


def chain_range(rank, world, C):
    """Contiguous chain range [chain0, chain0 + count) of `rank` out of `world`."""
    lo = C * rank // world
    hi = C * (rank + 1) // world
    return lo, hi - lo


def merge_stats(parts, N, k=0):
    """Merge rosen_stats dicts of disjoint chain sets (in the given order).

    N and k are the ensemble's monomers and trials per step (for logZ_norm).
    """
    M = max(p["log_max"] for p in parts)
    out = {"n": sum(p["n"] for p in parts), "n_alive": sum(p["n_alive"] for p in parts),
           "log_max": M}
    for key in _FIRST + _SECOND:
        out[key] = 0.0
    if M == -math.inf:
        out.update(logZ=-math.inf, logZ_norm=-math.inf, mean_r2=math.nan, se_r2=math.nan,
                   mean_rg2=math.nan, se_rg2=math.nan, ess=0.0)
        return out
    for p in parts:
        if p["log_max"] == -math.inf:
            continue
        f = math.exp(p["log_max"] - M)
        for key in _FIRST:
            out[key] += p[key] * f
        for key in _SECOND:
            out[key] += p[key] * f * f
    S0 = out["S0"]
    out["logZ"] = M + math.log(S0 / out["n"])
    out["logZ_norm"] = out["logZ"] - (N - 1) * math.log(k) if k > 0 else out["logZ"]
    for m, q1, q2, sk, mk, sek in (("S1", "Q1_r2", "Q2_r2", "S1", "mean_r2", "se_r2"),
                                  ("S2", "Q1_rg2", "Q2_rg2", "S2", "mean_rg2", "se_rg2")):
        mean = out[sk] / S0
        var = out[q2] - 2.0 * mean * out[q1] + mean * mean * out["Q0"]
        out[mk] = mean
        out[sek] = math.sqrt(var if var > 0.0 else 0.0) / S0
    out["ess"] = S0 * S0 / out["Q0"]
    return out


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
