"""GPU parity of replica exchange ("Sampling", Eq. (repXacc)): permutations, per-slot states and
attempt/accept counts are bit-exact against the oracle given identical components and Philox
counters, for ladder sizes spanning one warp, several warps and a ragged tail."""
import numpy as np
import pytest

import oracle
from paper_1507_03703_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _ctx(T, alpha):
    from paper_1507_03703_gb300.algdock import Context
    ctx = Context(0)
    ctx.states_set(T, alpha, np.full(len(T), 2.0))
    return ctx


def _comps(rng, L, K, spread=1.0):
    c = np.zeros((L, K, 4))
    c[..., 0] = rng.normal(0, 3, size=(L, K)) * spread
    c[..., 1] = rng.uniform(0, 2, size=(L, K)) * spread
    c[..., 2] = rng.normal(0, 4, size=(L, K)) * spread
    c[..., 3] = rng.normal(-5, 4, size=(L, K)) * spread
    return c


@pytest.mark.parametrize("K,L,max_sep,n_sweeps", [(2, 3, 5, 25), (8, 64, 5, 25), (32, 4, 8, 10), (33, 5, 5, 25),
                                                  (64, 3, 5, 25), (65, 3, 7, 10), (96, 64, 5, 25), (127, 2, 8, 6),
                                                  (128, 4, 5, 25), (130, 2, 3, 7), (200, 3, 5, 4), (1, 4, 5, 3)])
def test_exchange_bit_exact(K, L, max_sep, n_sweeps):
    rng = np.random.default_rng(K * 1000 + L)
    # a table with a warming leg (alpha NaN) first, then the coupling leg under test
    Kbc = 4
    T = np.concatenate([S.geometric_temperatures(Kbc, 300, 600), np.linspace(600, 300, K)])
    alpha = np.concatenate([np.full(Kbc, np.nan), np.linspace(0, 1, K)])
    ctx = _ctx(T, alpha)
    comps = _comps(rng, L, K, spread=0.3)
    cfg0 = np.stack([rng.permutation(K) for _ in range(L)]).astype(np.int32)
    seed, cycle, loff = 0xDEADBEEF01, 17, 9
    cfg_o, att_o, acc_o = oracle.exchange(T[Kbc:], alpha[Kbc:], comps, cfg0, n_sweeps, max_sep, seed, cycle,
                                          ladder_offset=loff)
    cd = torch.from_numpy(comps).cuda()
    cfg = torch.from_numpy(cfg0.copy()).cuda()
    st = torch.full((L, K), -1, dtype=torch.int32, device="cuda")
    att = torch.zeros((max_sep, K), dtype=torch.int64, device="cuda")
    acc = torch.zeros((max_sep, K), dtype=torch.int64, device="cuda")
    ctx.exchange(K, Kbc, cd, cfg, st, n_sweeps=n_sweeps, max_sep=max_sep, seed=seed, cycle=cycle,
                 ladder_offset=loff, attempts=att, accepts=acc)
    torch.cuda.synchronize()
    assert np.array_equal(cfg.cpu().numpy(), cfg_o)
    assert np.array_equal(att.cpu().numpy(), att_o)
    assert np.array_equal(acc.cpu().numpy(), acc_o)
    s = st.cpu().numpy()
    for l in range(L):
        for k in range(K):
            assert s[l, cfg_o[l, k]] == Kbc + k
    if K > 1:
        assert acc_o.sum() > 0 and acc_o.sum() < att_o.sum()


def test_exchange_warming_leg_alpha_nan():
    rng = np.random.default_rng(3)
    K, L = 16, 10
    T = S.geometric_temperatures(K, 300, 600)
    alpha = np.full(K, np.nan)
    ctx = _ctx(T, alpha)
    comps = _comps(rng, L, K, spread=0.05)
    cfg0 = np.tile(np.arange(K, dtype=np.int32), (L, 1))
    cfg_o, att_o, acc_o = oracle.exchange(T, alpha, comps, cfg0, 25, 5, 77, 1)
    cfg = torch.from_numpy(cfg0.copy()).cuda()
    acc = torch.zeros((5, K), dtype=torch.int64, device="cuda")
    ctx.exchange(K, 0, torch.from_numpy(comps).cuda(), cfg, None, n_sweeps=25, max_sep=5, seed=77, cycle=1,
                 accepts=acc)
    assert np.array_equal(cfg.cpu().numpy(), cfg_o)
    assert np.array_equal(acc.cpu().numpy(), acc_o)


def test_exchange_bit_exact_cancelling_components():
    """A temperature ladder at full coupling (w_sg = 0, w_g = 1) whose slots carry U_L of +-1e4
    kcal/mol cancelled by Psi_g to within a few kcal/mol: the FP32 estimate's error bound is then
    wide, so most attempts take the FP64 test, which must still give the oracle's decisions."""
    rng = np.random.default_rng(29)
    K, L = 48, 8
    T = np.geomspace(300, 600, K)
    alpha = np.ones(K)
    ctx = _ctx(T, alpha)
    big = rng.normal(0, 1e4, size=(L, K))
    comps = np.zeros((L, K, 4))
    comps[..., 0] = big
    comps[..., 1] = rng.uniform(0, 2, size=(L, K))
    comps[..., 2] = rng.normal(0, 1e3, size=(L, K))  # soft grid: weight zero at alpha = 1
    comps[..., 3] = -big + rng.normal(0, 2, size=(L, K))
    cfg0 = np.stack([rng.permutation(K) for _ in range(L)]).astype(np.int32)
    cfg_o, att_o, acc_o = oracle.exchange(T, alpha, comps, cfg0, 25, 5, 1234, 3)
    cfg = torch.from_numpy(cfg0.copy()).cuda()
    att = torch.zeros((5, K), dtype=torch.int64, device="cuda")
    acc = torch.zeros((5, K), dtype=torch.int64, device="cuda")
    ctx.exchange(K, 0, torch.from_numpy(comps).cuda(), cfg, None, n_sweeps=25, max_sep=5, seed=1234, cycle=3,
                 attempts=att, accepts=acc)
    assert np.array_equal(cfg.cpu().numpy(), cfg_o)
    assert np.array_equal(att.cpu().numpy(), att_o)
    assert np.array_equal(acc.cpu().numpy(), acc_o)
    assert 0 < acc_o.sum() < att_o.sum()
