"""Worker of the multi-rank tests: one gloo rank (CPU) running its shard of a replica-exchange ladder
with the oracle, then the collectives the multi-GPU path uses."""
import os

import numpy as np

import oracle
from paper_1507_03703_gb300 import ranks
from paper_1507_03703_gb300 import synthetic as S

N_CYCLES, N_STEPS, SEED = 3, 5, 31


def small_ladder():
    """A 6-atom ligand on smooth synthetic grids, a 4-state ladder, and one start pose per slot
    for up to 8 chains (deterministic)."""
    lig = S.make_ligand(6, seed=3)
    grid = S.cube_grid(np.zeros(3), 0.5, 17)
    ax = grid.origin[0] + grid.spacing * np.arange(17)
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    r2 = X ** 2 + Y ** 2 + Z ** 2
    ljr = (50.0 * np.exp(-r2 / 20.0)).astype(np.float64)
    lja = (-5.0 * np.exp(-r2 / 30.0)).astype(np.float64)
    elec = (2.0 * np.sin(X / 2.0) * np.cos(Y / 3.0)).astype(np.float64)
    leg = S.cd_ladder(4, dt_fs=2.0)
    osys = oracle.OracleSystem(grid, ljr, lja, elec, lig, leg.T, leg.alpha, leg.dt_fs, site=np.zeros(3))
    rng = np.random.default_rng(4)
    base = lig.x0
    x0 = np.stack([base + rng.normal(scale=0.5, size=3) for _ in range(8 * leg.K)])
    return osys, x0


def run_shard(osys, x0, sh: ranks.Shard):
    """The shard's chains with their global Philox offsets; samples as [chains, cycles, K, 4]."""
    K = osys.K
    xs = x0[sh.chain_begin * K:(sh.chain_begin + sh.n_chains) * K]
    comps, st, _, _, x = oracle.run_ladder(osys, xs, sh.n_chains, N_CYCLES, N_STEPS, SEED,
                                           rep_offset=sh.rep_offset(K), ladder_offset=sh.ladder_offset(1))
    c = comps.reshape(N_CYCLES, sh.n_chains, K, 4).transpose(1, 0, 2, 3)
    s = st.reshape(N_CYCLES, sh.n_chains, K).transpose(1, 0, 2)
    return np.ascontiguousarray(c), np.ascontiguousarray(s), x.reshape(sh.n_chains, K, -1, 3)


def ladder_worker(rank, world, port, n_chains, out):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        osys, x0 = small_ladder()
        sh = ranks.shard(n_chains, world, rank)
        c, s, x = run_shard(osys, x0, sh)
        gc = ranks.gather_rows(torch.from_numpy(c))
        gs = ranks.gather_rows(torch.from_numpy(s))
        gx = ranks.gather_rows(torch.from_numpy(x))
        slowest = ranks.max_over_ranks(10.0 + rank)
        total = ranks.sum_over_ranks(float(sh.n_chains))
        if rank == 0:
            np.savez(out, comps=gc.numpy(), states=gs.numpy(), x=gx.numpy(), slowest=slowest, total=total)
    finally:
        dist.destroy_process_group()


def harmonic_ukn(K=6, n_per=700, seed=8):
    """u_kn of exact samples of K harmonic wells (deterministic), with N_k."""
    bk, mu, x, N_k = S.harmonic_oscillator_samples(K, n_per, seed=seed, D=2)
    return 0.5 * bk[:, None] * ((x[None, :, :] - mu[:, None, :]) ** 2).sum(-1), N_k


def mbar_split(N, world, rank):
    """Uneven contiguous column blocks: rank r holds a block proportional to r + 1."""
    w = np.arange(1, world + 1, dtype=np.float64)
    edges = np.concatenate([[0], np.round(np.cumsum(w) / w.sum() * N)]).astype(int)
    return edges[rank], edges[rank + 1]


def mbar_worker(rank, world, port, out):
    """MBAR sharded over samples: each rank's pairs from the oracle's FP64 state sums of its own
    columns, one all_gather per iteration, the library's update on every rank."""
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        u, N_k = harmonic_ukn()
        a, b = mbar_split(u.shape[1], world, rank)
        ul = u[:, a:b]
        f, it = ranks.mbar_sharded(None, None, N_k, tol=1e-12, partials=lambda f: oracle.mbar_partials(ul, N_k, f))
        np.savez(out + ".%d.npz" % rank, f=f, it=it)
    finally:
        dist.destroy_process_group()
