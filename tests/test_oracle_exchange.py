"""Oracle pins for Hamiltonian replica exchange (Eq. (repXacc); sweeps over pairs 1..min(5, K-1)
states apart): permutations stay permutations, identical states always swap, and the stationary
distribution over permutations is the exact product of Boltzmann factors (detailed balance)."""
import itertools

import numpy as np

import oracle


def _comps(rng, L, K):
    c = np.zeros((L, K, 4))
    c[..., 0] = rng.normal(0, 3, size=(L, K))
    c[..., 1] = rng.uniform(0, 2, size=(L, K))
    c[..., 2] = rng.normal(0, 4, size=(L, K))
    c[..., 3] = rng.normal(-5, 4, size=(L, K))
    return c


def test_exchange_keeps_permutations_and_counts():
    rng = np.random.default_rng(0)
    L, K = 7, 12
    T = np.linspace(600, 300, K)
    alpha = np.linspace(0, 1, K)
    cfg = np.tile(np.arange(K, dtype=np.int32), (L, 1))
    comps = _comps(rng, L, K)
    cfg2, att, acc = oracle.exchange(T, alpha, comps, cfg, n_sweeps=25, max_sep=5, seed=1, cycle=2)
    for l in range(L):
        assert sorted(cfg2[l]) == list(range(K))
    # every sweep attempts each pair (a, a+s) exactly once per ladder
    for s in range(1, 6):
        for a in range(K):
            assert att[s - 1, a] == (25 * L if a + s < K else 0)
    assert np.all(acc <= att)


def test_identical_states_always_exchange():
    rng = np.random.default_rng(1)
    K = 9
    T = np.full(K, 450.0)
    alpha = np.full(K, 0.3)
    comps = _comps(rng, 3, K)
    _, att, acc = oracle.exchange(T, alpha, comps, np.tile(np.arange(K, dtype=np.int32), (3, 1)), 5, 5, 2, 0)
    assert np.array_equal(att, acc) and att.sum() > 0


def test_exchange_stationary_distribution_is_boltzmann_over_permutations():
    rng = np.random.default_rng(2)
    K, L = 3, 40000
    T = np.array([300.0, 420.0, 600.0])
    alpha = np.array([1.0, 0.6, 0.2])
    base = _comps(rng, 1, K)[0] * 0.3
    comps = np.repeat(base[None], L, 0)
    u = oracle.ukn_from_comps(T, alpha, base)  # u[k, i]
    perms = list(itertools.permutations(range(K)))
    logw = np.array([-sum(u[k, p[k]] for k in range(K)) for p in perms])
    p_exact = np.exp(logw - logw.max())
    p_exact /= p_exact.sum()
    cfg = np.tile(np.arange(K, dtype=np.int32), (L, 1))
    cfg, _, _ = oracle.exchange(T, alpha, comps, cfg, n_sweeps=12, max_sep=5, seed=3, cycle=0)
    counts = np.array([np.sum(np.all(cfg == np.array(p), axis=1)) for p in perms])
    se = np.sqrt(L * p_exact * (1 - p_exact))
    assert np.all(np.abs(counts - L * p_exact) < 5 * se + 1), (counts, L * p_exact)
