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

import numpy as np


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


def mbar_sharded(ctx, u_local, N_k, tol=1e-10, max_iter=10000, precision_mode=0, partials=None, group=None):
    """MBAR ("Estimation") over samples spread across the ranks: each rank holds the columns of u_kn
    of its own samples.  Per iteration: this rank's (max, sum) pair per state
    (algdock_mbar_partials on its GPU, or ``partials(f)`` if given), one all_gather of the K pairs,
    and algdock_mbar_update over the pairs in rank order, so that every rank holds the same f.
    N_k are the counts over all ranks.  Returns (f [K], iterations); raises if max_iter is reached."""
    import torch
    import torch.distributed as dist
    from .algdock import AlgdockError, E_NOT_CONVERGED, mbar_update

    K = len(N_k)
    on = dist.is_available() and dist.is_initialized()
    world = dist.get_world_size(group) if on else 1
    dev = None
    if on and dist.get_backend(group) == "nccl":
        dev = torch.device("cuda", torch.cuda.current_device())
    f = np.zeros(K)
    for it in range(1, max_iter + 1):
        p = partials(f) if partials is not None else ctx.mbar_partials(u_local, N_k, f, precision_mode)
        p = np.ascontiguousarray(p, dtype=np.float64).reshape(K, 2)
        if world > 1:
            t = torch.from_numpy(p.ravel().copy())
            if dev is not None:
                t = t.to(dev)
            parts = [torch.empty_like(t) for _ in range(world)]
            dist.all_gather(parts, t, group=group)
            allp = np.stack([q.cpu().numpy().reshape(K, 2) for q in parts])
        else:
            allp = p[None]
        f, delta = mbar_update(allp, f)
        if delta < tol:
            return f, it
    raise AlgdockError(E_NOT_CONVERGED, "mbar_sharded: max_iter reached")
