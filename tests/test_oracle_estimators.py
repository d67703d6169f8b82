"""Oracle pins for estimation ("Estimation"; "Equilibration and production"): MBAR against
closed-form harmonic free energies, its two-state reduction to BAR, identical states, the
reduced potential of the protocol at its milestones, and the statistical inefficiency of an AR(1)
series."""
import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
from paper_1507_03703_gb300 import synthetic as S


def _ukn_harmonic(bk, mu, x):
    return 0.5 * bk[:, None] * ((x[None, :, :] - mu[:, None, :]) ** 2).sum(-1)


def test_mbar_recovers_harmonic_oscillator_free_energies():
    bk, mu, x, N_k = S.harmonic_oscillator_samples(5, 20000, seed=0, D=2)
    u = _ukn_harmonic(bk, mu, x)
    f, it = oracle.mbar(u, N_k, tol=1e-10)
    assert it > 0
    exact = -(2 / 2.0) * np.log(2 * np.pi / bk)
    exact -= exact[0]
    assert np.max(np.abs(f - exact)) < 0.04, (f, exact)


def test_mbar_two_states_is_bar():
    bk, mu, x, N_k = S.harmonic_oscillator_samples(2, 3000, seed=1, D=1)
    u = _ukn_harmonic(bk, mu, x)
    f, it = oracle.mbar(u, N_k, tol=1e-13)
    du = u[1] - u[0]
    n0 = N_k[0]
    w0, w1 = du[:n0], du[n0:]
    M = np.log(N_k[0] / N_k[1])

    def bar(df):
        return (np.sum(1.0 / (1.0 + np.exp(M + w0 - df)))
                - np.sum(1.0 / (1.0 + np.exp(-M - w1 + df))))

    df = brentq(bar, -20, 20, xtol=1e-14)
    assert f[1] == pytest.approx(df, abs=1e-9)


def test_mbar_identical_states_and_nonconvergence():
    rng = np.random.default_rng(2)
    row = rng.normal(size=500)
    u = np.tile(row, (4, 1))
    f, it = oracle.mbar(u, np.array([100, 200, 0, 200]), tol=1e-12)
    assert np.allclose(f, 0.0, atol=1e-12) and it >= 1
    bk, mu, x, N_k = S.harmonic_oscillator_samples(4, 500, seed=3)
    f, it = oracle.mbar(_ukn_harmonic(bk, mu, x), N_k, tol=1e-14, max_iter=2)
    assert it == -1


def test_reduced_potential_at_milestones():
    sys_ = S.config_small(1)
    ljr, lja, elec = oracle.grid_direct_sum(sys_.receptor, sys_.grid)
    cd = sys_.legs[1]
    osys = oracle.OracleSystem(sys_.grid, ljr, lja, elec, sys_.ligand, cd.T, cd.alpha, cd.dt_fs)
    x = S.place_ligand(sys_.ligand, sys_.receptor, sys_.site, 4, seed=1, n_tries=8).astype(np.float64)
    u, comps = osys.reduced_energies(x)
    assert np.allclose(u, oracle.ukn_from_comps(cd.T, cd.alpha, comps), rtol=0, atol=0)
    bH, bT = oracle.beta(600.0), oracle.beta(300.0)
    # alpha = 0 is milestone C (ligand alone at T_H), alpha = 1 is milestone D (grids at T_T)
    assert np.allclose(u[0], bH * (comps[:, 0] + comps[:, 1]), rtol=1e-14)
    assert np.allclose(u[-1], bT * (comps[:, 0] + comps[:, 1] + comps[:, 3]), rtol=1e-14)
    # a warming-leg state (alpha = NaN) has no grid term
    unan = oracle.ukn_from_comps([450.0], [np.nan], comps)
    assert np.allclose(unan[0], oracle.beta(450.0) * (comps[:, 0] + comps[:, 1]), rtol=1e-14)


def test_statistical_inefficiency_of_ar1_series():
    rng = np.random.default_rng(4)
    rho, N = 0.8, 200000
    e = rng.normal(size=N)
    a = np.empty(N)
    a[0] = e[0]
    for i in range(1, N):
        a[i] = rho * a[i - 1] + np.sqrt(1 - rho * rho) * e[i]
    g = oracle.statistical_inefficiency(a)
    assert abs(g - (1 + rho) / (1 - rho)) < 0.1 * (1 + rho) / (1 - rho)
    assert oracle.statistical_inefficiency(rng.normal(size=20000)) < 1.2
