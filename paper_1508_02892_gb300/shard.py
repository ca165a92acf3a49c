"""Host logic of the multi-GPU runs: independent discharges are partitioned
over ranks (one process per GPU) with no exchange on the data path; the only
collectives are the timing barrier and the reduction of the measured time
(max over ranks) and work (sum over ranks)."""


def instance_seed(rank: int, base: int = 2026) -> int:
    """Seed of the batched workload drawn by `rank`: every rank simulates its
    own set of discharges (weak scaling)."""
    return base + 7919 * int(rank)


def rank_share(items, rank: int, world: int):
    """Requests dealt round-robin: item k goes to rank k mod world."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    return [x for k, x in enumerate(items) if k % world == rank]


def aggregate(ms_local: float, n_local: float, device=None):
    """(max over ranks of the timed milliseconds, sum over ranks of the work);
    with no process group initialised, the local values."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms_local), float(n_local)
    t = torch.tensor([float(ms_local), float(n_local)], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return mx[0].item(), sm[1].item()
