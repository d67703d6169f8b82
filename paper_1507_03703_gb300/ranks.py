"""Independent chains sharded over ranks (one process per GPU).

Replica-exchange chains are independent Markov chains, so the sampling loop has no data-path
exchange between ranks: each rank runs its own block of chains.  Every random number of the method
is a Philox draw named by a global replica index (HMC momenta, Metropolis tests, learned moves) or a
global ladder index (exchange sweeps).  With the offsets below a rank's block of chains keeps the
global indices that the same chains have in a one-process run, so a single ladder sharded over any
number of ranks samples exactly the chains one GPU would.  The one collective is after sampling:
the recorded samples meet for the free-energy estimate (MBAR needs every sample at every state).
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class Shard:
    rank: int
    world: int
    chain_begin: int   # global index of the rank's first chain
    n_chains: int      # chains on this rank

    def rep_offset(self, k_total: int) -> int:
        """Global index of the rank's first replica slot, slots numbered chain-major over all the
        chains' k_total states (the sum of the legs' ladder lengths)."""
        return self.chain_begin * k_total

    def ladder_offset(self, n_legs: int) -> int:
        """Global index of the rank's first ladder (n_legs ladders per chain)."""
        return self.chain_begin * n_legs


def shard(n_chains: int, world: int, rank: int) -> Shard:
    """Contiguous blocks of chains, the remainder going one each to the first ranks (strong
    scaling: a fixed total of chains)."""
    if world < 1 or not 0 <= rank < world or n_chains < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, n_chains >= 0")
    base, extra = divmod(n_chains, world)
    begin = rank * base + min(rank, extra)
    return Shard(rank, world, begin, base + (1 if rank < extra else 0))


def shard_per_rank(n_chains_per_rank: int, world: int, rank: int) -> Shard:
    """The same number of chains on every rank (weak scaling)."""
    if world < 1 or not 0 <= rank < world or n_chains_per_rank < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, n_chains_per_rank >= 0")
    return Shard(rank, world, rank * n_chains_per_rank, n_chains_per_rank)


def gather_rows(t, group=None):
    """All ranks' row blocks of t ([n_r, ...], n_r may differ by rank) concatenated in rank order,
    on every rank.  One all_gather of the row counts, one of the rows (padded to the longest)."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized():
        return t
    world = dist.get_world_size(group)
    n = torch.tensor([t.shape[0]], dtype=torch.int64, device=t.device)
    counts = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(counts, n, group=group)
    counts = [int(c.item()) for c in counts]
    m = max(counts) if counts else 0
    pad = t.new_zeros((m,) + tuple(t.shape[1:]))
    pad[: t.shape[0]] = t
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad.contiguous(), group=group)
    return torch.cat([p[:c] for p, c in zip(parts, counts)], 0)


def max_over_ranks(value: float, device=None, group=None) -> float:
    """The largest of the ranks' values (the step time of the slowest rank), on every rank."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sum_over_ranks(value: float, device=None, group=None) -> float:
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())
