"""Multi-GPU harness: one independent replica of the workload per rank.

The force evaluation of one box is not sharded across GPUs here, so ranks
exchange nothing on the data path; they only agree on the timing of the
measured region (max over ranks) and on the work done (sum over ranks).
Replica r draws its random batches from its own key, base seed + 1000 r.
"""
from __future__ import annotations


def replica_seed(base_seed: int, rank: int) -> int:
    """Philox key of replica ``rank`` (independent batch sequences)."""
    return int(base_seed) + 1000 * int(rank)


def aggregate(local_ms: float, local_units: float, dist=None, device=None):
    """Whole-job throughput of the replicas: (units summed over ranks) /
    (max over ranks of the measured time).  Returns (units per second,
    max milliseconds, total units).  ``dist`` is ``torch.distributed`` with an
    initialised process group, or None for one process."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return local_units / (local_ms / 1000.0), float(local_ms), float(local_units)
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    ms, units = float(t.item()), float(u.item())
    return units / (ms / 1000.0), ms, units
