"""Multi-GPU runs as independent replicas (one lattice per rank).

The lattice evolution needs no exchange between ranks here: every rank
advances its own lattice (seeded by rank), so the only collectives are the
benchmark's barrier and the maximum of the per-rank timed regions.  These
helpers are shared by the benchmark (NCCL on GPUs) and the gloo tests on CPU.
"""
from __future__ import annotations


def replica_seed(base_seed: int, rank: int) -> int:
    return base_seed + rank


def barrier(dist=None):
    if dist is not None and dist.is_initialized():
        dist.barrier()


def max_over_ranks(value: float, dist=None, device: str = "cpu") -> float:
    """Largest value over all ranks (the slowest rank's time bounds the job)."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(world_size: int, units_per_rank: float, seconds: float) -> float:
    """Units processed by all ranks per second of the slowest rank."""
    return world_size * units_per_rank / seconds
