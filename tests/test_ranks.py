"""The multi-rank path on CPU: chains sharded over two gloo ranks with global Philox offsets sample
exactly the chains of a one-process run (replica exchange, "Sampling": chains are independent, so
sharding them needs no data exchange), and the collectives after sampling (gathering the samples
for MBAR, the slowest rank's time) give what one process would."""
import socket

import numpy as np
import pytest

import oracle
from paper_1507_03703_gb300 import ranks

import rank_worker as W

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n,world", [(0, 1), (1, 3), (5, 2), (8, 4), (13, 5), (100, 8)])
def test_shards_partition_the_chains(n, world):
    sh = [ranks.shard(n, world, r) for r in range(world)]
    assert sh[0].chain_begin == 0
    for a, b in zip(sh, sh[1:]):
        assert b.chain_begin == a.chain_begin + a.n_chains
    assert sum(s.n_chains for s in sh) == n
    assert max(s.n_chains for s in sh) - min(s.n_chains for s in sh) <= 1


def test_global_offsets_give_disjoint_streams():
    """Replica slots and ladders of different ranks never share a Philox index."""
    K_total, n_legs = 128, 2
    seen_r, seen_l = set(), set()
    for r in range(4):
        sh = ranks.shard_per_rank(64, 4, r)
        rr = set(range(sh.rep_offset(K_total), sh.rep_offset(K_total) + sh.n_chains * K_total))
        ll = set(range(sh.ladder_offset(n_legs), sh.ladder_offset(n_legs) + sh.n_chains * n_legs))
        assert not (rr & seen_r) and not (ll & seen_l)
        seen_r |= rr
        seen_l |= ll
    with pytest.raises(ValueError):
        ranks.shard(4, 2, 2)


@pytest.mark.parametrize("n_chains", [6, 5])
def test_two_gloo_ranks_sample_the_one_process_chains(tmp_path, n_chains):
    import torch.multiprocessing as mp

    out = str(tmp_path / "r.npz")
    mp.spawn(W.ladder_worker, args=(2, _free_port(), n_chains, out), nprocs=2, join=True)
    got = np.load(out)
    osys, x0 = W.small_ladder()
    c, s, x = W.run_shard(osys, x0, ranks.shard(n_chains, 1, 0))
    assert np.array_equal(got["comps"], c)
    assert np.array_equal(got["states"], s)
    assert np.array_equal(got["x"], x)
    assert float(got["slowest"]) == 11.0 and float(got["total"]) == n_chains
    # the pooled free energies (MBAR over every rank's samples) are the one-process ones
    T, alpha = osys.T, osys.alpha
    f1, _ = oracle.ladder_free_energies(T, alpha, got["comps"].reshape(-1, 4), got["states"].reshape(-1))
    f2, _ = oracle.ladder_free_energies(T, alpha, c.reshape(-1, 4), s.reshape(-1))
    assert np.array_equal(f1, f2)


def test_collectives_without_a_process_group_are_identities():
    t = torch.arange(6.0).reshape(3, 2)
    assert ranks.gather_rows(t) is t
    assert ranks.max_over_ranks(2.5) == 2.5
    assert ranks.sum_over_ranks(2.5) == 2.5


@pytest.mark.parametrize("world", [2, 3])
def test_mbar_sharded_over_gloo_ranks_matches_the_one_process_solve(tmp_path, world):
    """MBAR over samples split unevenly over the ranks ("Estimation"): every rank ends with the same
    free energies, and they equal the oracle's one-process solve within 1e-10 kT."""
    import torch.multiprocessing as mp

    out = str(tmp_path / "m")
    mp.spawn(W.mbar_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    fs = [np.load(out + ".%d.npz" % r)["f"] for r in range(world)]
    for f in fs[1:]:
        assert np.array_equal(f, fs[0])
    u, N_k = W.harmonic_ukn()
    f_ref, _ = oracle.mbar(u, N_k, tol=1e-12)
    assert np.max(np.abs(fs[0] - f_ref)) < 1e-10


def test_mbar_partials_of_a_partition_merge_to_the_whole():
    """The oracle's per-subset state sums (the sharded MBAR's unit of work) merged over a partition
    of the samples equal the sums over all samples, and a solve iterating the library's update on
    the whole set reproduces the oracle's MBAR."""
    from paper_1507_03703_gb300.algdock import mbar_update
    u, N_k = W.harmonic_ukn(K=4, n_per=300, seed=3)
    f = np.array([0.0, 0.3, -0.2, 1.1])
    whole = oracle.mbar_partials(u, N_k, f)
    parts = np.stack([oracle.mbar_partials(u[:, a:b], N_k, f) for a, b in [(0, 100), (100, 101), (101, 1200)]])
    f1, _ = mbar_update(whole[None], f)
    f3, _ = mbar_update(parts, f)
    assert np.max(np.abs(f1 - f3)) < 1e-12
    empty = oracle.mbar_partials(u[:, :0], N_k, f)
    f4, _ = mbar_update(np.concatenate([parts, empty[None]]), f)
    assert np.max(np.abs(f4 - f3)) == 0.0
    g = np.zeros(4)
    for _ in range(2000):
        g, d = mbar_update(oracle.mbar_partials(u, N_k, g)[None], g)
        if d < 1e-12:
            break
    f_ref, _ = oracle.mbar(u, N_k, tol=1e-12)
    assert np.max(np.abs(g - f_ref)) < 1e-10
