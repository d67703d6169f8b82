"""Oracle pins for protocol initialization ("Initialization": thermodynamic-length state placement,
importance-resampled seeds, time-step adaptation, the mean exchange probability check):

- the alpha step uses the exact derivatives of the protocol weights of Eq. (protocol): each term,
  isolated, matches a central difference of alpha_sg, alpha_g or T(alpha);
- resampled seeds follow their weights (chi-square);
- the mean exchange probability is 1 between a state and itself, and between two temperatures of a
  harmonic well it matches the closed-form expectation over Gamma-distributed energies;
- the time-step rule, including the order of its thresholds and the [0.1, 5] fs clamp;
- on a harmonic well (3 degrees of freedom, sigma[U] = k_B T sqrt(3/2)) the warming leg is
  geometric, T_{k+1}/T_k = 1 + s sqrt(2/3), spans 300 -> 600 K, and every neighbour pair passes the
  check; on a coupling leg that starts too fast the check shrinks the speed until neighbours
  overlap."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle
from paper_1507_03703_gb300 import synthetic as S


def test_alpha_step_uses_the_exact_weight_derivatives():
    s, T_T, T_H, h = 0.2, 300.0, 600.0, 1e-6
    for a in (0.1, 0.3, 0.49, 0.51, 0.7, 0.9):
        T = (T_T - T_H) * a + T_H
        sig = 200.0
        an = oracle.next_alpha(a, sig, 0.0, 0.0, s)  # the soft-grid term alone
        dsg = (oracle.alpha_sg(a + h) - oracle.alpha_sg(a - h)) / (2 * h)
        assert an - a == pytest.approx(min(1.0 - a, s / (abs(dsg) * sig / (oracle.KB * T))), rel=1e-6)
        an = oracle.next_alpha(a, 0.0, sig, 0.0, s)  # the full-grid term alone
        dg = (oracle.alpha_g(a + h) - oracle.alpha_g(a - h)) / (2 * h)
        if abs(dg) > 1e-6:
            assert an - a == pytest.approx(min(1.0 - a, s / (abs(dg) * sig / (oracle.KB * T))), rel=1e-5)
        an = oracle.next_alpha(a, 0.0, 0.0, 2.0, s)  # the temperature term alone
        assert an - a == pytest.approx(min(1.0 - a, s * T / (abs(T_T - T_H) * 2.0)), rel=1e-12)
    assert oracle.next_alpha(0.95, 0.0, 0.0, 1e-9, 1.0) == 1.0
    assert oracle.next_temperature(590.0, 0.1, 5.0) == 600.0


def test_resampled_seeds_follow_their_weights():
    w = np.array([1.0, 2.0, 3.0, 4.0, 0.0])
    logw = np.log(np.where(w > 0, w, 1e-300)) + 17.0  # a constant shift changes nothing
    picks = np.concatenate([oracle.resample(logw, 2000, 5, ctr) for ctr in range(4)])
    counts = np.bincount(picks, minlength=5)
    assert counts[4] == 0
    p = w[:4] / w[:4].sum()
    chi2 = (((counts[:4] - p * picks.size) ** 2) / (p * picks.size)).sum()
    assert chi2 < stats.chi2.ppf(0.999, 3)
    assert np.array_equal(oracle.resample(logw, 50, 5, 9), oracle.resample(logw, 50, 5, 9))


def _harmonic(k=5.0, T=(300.0,)):
    lig = S.one_atom_ligand(charge=0.0)
    grid = S.cube_grid(np.zeros(3), 0.5, 17)
    zero = np.zeros((17, 17, 17))
    return oracle.OracleSystem(grid, zero, zero, zero, lig, np.array(T), np.full(len(T), np.nan),
                               np.full(len(T), 2.0), site=np.zeros(3), k_rest=k, d0=0.0)


def test_mean_exchange_probability():
    osys = _harmonic(T=(300.0, 420.0))
    rng = np.random.default_rng(3)
    n = 40000
    Ua = rng.gamma(1.5, oracle.KB * 300.0, size=n)  # U = k r^2 / 2 in 3-D: Gamma(3/2, k_B T)
    Ub = rng.gamma(1.5, oracle.KB * 420.0, size=n)
    ca, cb = np.zeros((n, 4)), np.zeros((n, 4))
    ca[:, 1], cb[:, 1] = Ua, Ub
    assert osys.mean_pacc(ca, ca, 0, 0) == 1.0
    got = osys.mean_pacc(ca, cb, 0, 1)
    ba, bb = 1 / (oracle.KB * 300.0), 1 / (oracle.KB * 420.0)
    pa = lambda u: stats.gamma.pdf(u, 1.5, scale=1 / ba)
    pb = lambda u: stats.gamma.pdf(u, 1.5, scale=1 / bb)
    exact, _ = integrate.dblquad(lambda ub, ua: pa(ua) * pb(ub) * min(1.0, math.exp((ba - bb) * (ua - ub))),
                                 0, 30 / ba, 0, 30 / bb)
    assert abs(got - exact) < 0.01, (got, exact)


def test_time_step_rule():
    assert oracle.adapt_dt(2.0, 0.85) == 2.125
    assert oracle.adapt_dt(2.0, 0.6) == 2.0
    assert oracle.adapt_dt(2.0, 0.3) == 1.75
    assert oracle.adapt_dt(2.0, 0.05) == 1.5  # below 0.1 the larger cut applies
    assert oracle.adapt_dt(0.3, 0.05) == 0.1 and oracle.adapt_dt(4.95, 0.9) == 5.0


def test_warming_leg_is_geometric_on_a_harmonic_well():
    """Each step estimates sigma[U] from 2000 correlated samples (about 12 % scatter), so the
    ratios scatter by a few per cent about 1 + s sqrt(2/3); pooled over three protocols their mean
    is within 5 %."""
    s = 0.3
    # k = 1.13 kcal/mol/A^2 on a 12 amu atom: a period of ~1000 fs, so a 50-step trajectory at
    # 5 fs is a quarter period, which swaps potential and kinetic energy and decorrelates U
    # between trials (a half-period trajectory would leave U almost unchanged)
    ratios = []
    for sd in (6, 11, 12):
        osys = _harmonic(k=1.13)
        seeds = np.random.default_rng(sd).normal(scale=0.6, size=(50, 1, 3))
        r = oracle.build_leg(osys, "bc", seeds, seed=sd, speed=s, n_trials=40, dt0=5.0)
        T = r["T"]
        assert T[0] == 300.0 and T[-1] == 600.0 and np.all(np.diff(T) > 0)
        assert np.all(r["pacc"] >= 0.4) and r["speed"] == s
        assert np.all((r["dt"] >= 0.1) & (r["dt"] <= 5.0))
        ratios.extend(T[1:-1] / T[:-2])  # the last step is clipped at 600 K
    ratios = np.array(ratios)
    expect = 1 + s * math.sqrt(2 / 3)
    assert np.all(np.abs(ratios / expect - 1) < 0.12), ratios
    assert abs(ratios.mean() / expect - 1) < 0.05, ratios


def test_too_fast_a_protocol_is_slowed_until_neighbours_overlap():
    """Coupling leg of one charged atom in a strong uniform field (24 kcal/mol across the 6 A
    restraint sphere): from speed 5 the first step would jump from alpha = 0 to 1 with almost no
    overlap, so the check shrinks the speed (by 4/5 per try) until every neighbour pair has a mean
    exchange probability of at least 0.4, and the leg still ends at alpha = 1."""
    lig = S.one_atom_ligand(charge=1.0)
    grid = S.cube_grid(np.zeros(3), 0.5, 33)
    ax = grid.origin[2] + grid.spacing * np.arange(33)
    elec = np.broadcast_to(-2.0 * ax[:, None, None], (33, 33, 33)).copy()
    zero = np.zeros((33, 33, 33))
    osys = oracle.OracleSystem(grid, zero, zero, elec, lig, np.array([600.0]), np.array([0.0]), np.array([4.0]),
                               site=np.zeros(3))
    seeds = np.random.default_rng(5).uniform(-3, 3, size=(50, 1, 3))
    r = oracle.build_leg(osys, "cd", seeds, seed=7, speed=5.0, n_trials=20, dt0=4.0)
    assert r["speed"] < 5.0
    assert np.all(r["pacc"] >= 0.4)
    assert r["alpha"][0] == 0.0 and r["alpha"][-1] == 1.0 and np.all(np.diff(r["alpha"]) > 0)
    assert np.allclose(r["T"], 600.0 - 300.0 * r["alpha"])
