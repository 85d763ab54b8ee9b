"""Wavelength sharding across ranks.

The field solves, Born rows and J x of different wavelengths are independent (the per-
wavelength loop of the recycled solver "can be executed in parallel", Section 3.2), so ranks
take disjoint wavelength chunks with no exchange. J^T y is a sum over wavelengths: each
rank accumulates the contribution of its own chunks, and one sum of n_chrom*N values over
the ranks completes the gradient.
"""
from __future__ import annotations


def chunk_of_step(step: int, rank: int, world: int, n_chunks: int) -> int:
    """Chunk processed by `rank` at `step`: ranks interleave, so one step of all ranks covers
    `world` distinct chunks."""
    return (step * world + rank) % n_chunks


def chunks_of_rank(rank: int, world: int, n_chunks: int):
    """Chunks a rank owns when the chunks are split once over the ranks."""
    return list(range(rank, n_chunks, world))


def allreduce_gradient(g):
    """Sum the per-rank J^T y contributions (torch.distributed, in place); a no-op for one rank."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(g, op=dist.ReduceOp.SUM)
    return g
