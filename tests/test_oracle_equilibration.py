"""Oracle pins for automated equilibration detection ("Equilibration and production"; Chodera 2016:
discard the start t0 that maximises N_eff = (T - t0) / g of the remaining series):

- a stationary series keeps (almost) all of its samples;
- a series with a decaying transient discards about the transient and no more, and the kept tail's
  mean is the stationary mean (the full series' mean is not);
- the detection is invariant under an affine change of the series;
- each candidate's g is the statistical inefficiency (pinned on AR(1) series elsewhere) of its tail."""
import numpy as np

import oracle


def _ar1(n, phi, rng):
    e = rng.normal(size=n)
    x = np.empty(n)
    x[0] = e[0] / np.sqrt(1 - phi ** 2)
    for i in range(1, n):
        x[i] = phi * x[i - 1] + e[i]
    return x


def test_stationary_series_keeps_its_samples():
    rng = np.random.default_rng(1)
    a = _ar1(3000, 0.5, rng)
    g, t0, neff = oracle.detect_equilibration(a, stride=10)
    assert t0 <= 300
    assert 0.5 * 3000 / 3.0 < neff <= 3000


def test_transient_is_discarded():
    rng = np.random.default_rng(2)
    tau, T = 100.0, 2000
    t = np.arange(T)
    a = 8.0 * np.exp(-t / tau) + _ar1(T, 0.5, rng)
    g, t0, neff = oracle.detect_equilibration(a, stride=10)
    assert tau <= t0 <= 10 * tau, t0
    tail = a[t0:]
    se = tail.std() * np.sqrt(g[t0 // 10] / tail.size)
    assert abs(tail.mean()) < 4 * se
    assert abs(a.mean()) > 4 * se  # the transient biases the full series


def test_affine_invariance():
    rng = np.random.default_rng(3)
    a = 3.0 * np.exp(-np.arange(2000) / 30.0) + _ar1(2000, 0.7, rng)
    g1, t1, n1 = oracle.detect_equilibration(a, stride=20)
    g2, t2, n2 = oracle.detect_equilibration(3.0 * a + 7.0, stride=20)
    assert t1 == t2
    assert np.allclose(g1, g2, rtol=1e-9) and abs(n1 - n2) < 1e-9 * n1


def test_candidate_g_is_the_tail_statistical_inefficiency():
    rng = np.random.default_rng(4)
    a = _ar1(500, 0.8, rng)
    g, _, _ = oracle.detect_equilibration(a, stride=7, n_cand=50)
    for c in (0, 13, 49):
        assert g[c] == oracle.statistical_inefficiency(a[7 * c:])
