"""Partition of the work across ranks (one process per GPU) and the one exchange it needs.

The energies of a scan are independent problems (each is a separate QEP, Eq. (4)), so
splitting them needs no communication at all.  Within one energy the quadrature points
of the ring (§3.2) and the right-hand-side columns are independent solves (§3.3, top
layer); their only coupling is the moment sum S_k = sum_j w_j z_j^k Y_j over the points
(Algorithm 1, first step), so splitting the points needs one sum reduction of the partial
moments S_k and mu_k before the extraction.
"""
from __future__ import annotations


def block_range(n: int, rank: int, world: int) -> range:
    """Contiguous share of n items for `rank` of `world`; the first n % world ranks take
    one extra item, so shares differ by at most one and cover 0..n-1 exactly once."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, n >= 0")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def energies_for_rank(energies, rank: int, world: int):
    """The energies this rank solves when a scan is split across ranks."""
    r = block_range(len(energies), rank, world)
    return [energies[i] for i in r]


def points_for_rank(n_int: int, rank: int, world: int) -> range:
    """Quadrature points j (of each circle) whose shifted systems this rank solves."""
    return block_range(n_int, rank, world)


def reduce_moments(S, mu, group=None):
    """Sum the partial moments of every rank in place (torch.distributed all-reduce on
    the tensors' own device; host tensors with the gloo backend).  Returns (S, mu)."""
    import torch.distributed as dist
    dist.all_reduce(S, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(mu, op=dist.ReduceOp.SUM, group=group)
    return S, mu
