"""Multi-GPU layout of the estimator: one process per GPU, weak scaling.

Every probe of every noise set is an independent right-hand side (Eq. (5)), so
ranks split the work by noise set: rank r solves sets [r n, (r + 1) n) of the
same colourings and the same operator.  Nothing on the data path crosses
ranks; the only collective is the end-of-run reduction of the timing (the
slowest rank) and of the work done (summed over ranks).  The per-set
estimates of all ranks together are the estimates of world x n sets.
"""


def rank_sets(rank, sets_per_rank):
    """(first set, number of sets) of this rank."""
    if rank < 0 or sets_per_rank < 1:
        raise ValueError("rank must be >= 0 and sets_per_rank >= 1")
    return rank * sets_per_rank, sets_per_rank


def reduce_timing(t_ms, units, device=None):
    """(max over ranks of t_ms, sum over ranks of units) via torch.distributed;
    returns the inputs unchanged when no process group is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(t_ms), float(units)
    t = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def gather_estimates(est, device=None):
    """Concatenate the per-set estimates (numpy complex [..., n_sets, n_p] with
    sets on axis -2) of all ranks in rank order; identity without a group."""
    import numpy as np
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return est
    t = torch.view_as_real(torch.as_tensor(np.ascontiguousarray(est))).to(device)
    parts = [torch.empty_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, t)
    return np.concatenate([torch.view_as_complex(p.cpu()).numpy() for p in parts], axis=-2)
