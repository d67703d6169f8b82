"""Oracle pins for the sampler ("Sampling": velocity Verlet inside HMC, Metropolis criterion):
time reversibility, energy error scaling as dt^2, and HMC reproducing closed-form equilibrium
averages of a harmonic and of the flat-bottom restraint (Eq. (binding_site))."""
import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_1507_03703_gb300 import synthetic as S


@pytest.fixture(scope="module")
def pocket():
    sys_ = S.config_small(1)
    ljr, lja, elec = oracle.grid_direct_sum(sys_.receptor, sys_.grid)
    leg = sys_.legs[1]
    osys = oracle.OracleSystem(sys_.grid, ljr, lja, elec, sys_.ligand, leg.T, leg.alpha, leg.dt_fs)
    x = S.place_ligand(sys_.ligand, sys_.receptor, sys_.site, 1, seed=0, n_tries=16)[0].astype(np.float64)
    return sys_, osys, x


def test_velocity_verlet_is_time_reversible(pocket):
    sys_, osys, x0 = pocket
    rng = np.random.default_rng(0)
    v0 = rng.normal(scale=0.005, size=x0.shape)
    x1, v1, _ = osys.vv(x0, v0, 0.3, 0.9, 1.0, 40)
    x2, v2, _ = osys.vv(x1, -v1, 0.3, 0.9, 1.0, 40)
    assert np.max(np.abs(x2 - x0)) < 1e-8
    assert np.max(np.abs(v2 + v0)) < 1e-10


def test_velocity_verlet_energy_error_scales_as_dt_squared(pocket):
    sys_, osys, x0 = pocket
    rng = np.random.default_rng(1)
    v0 = rng.normal(scale=0.004, size=x0.shape)
    dts = np.array([0.25, 0.5, 1.0, 2.0])
    errs = []
    for dt in dts:
        n = int(round(80.0 / dt))
        _, _, H = osys.vv(x0, v0, 0.0, 0.0, dt, n)
        errs.append(np.max(np.abs(H - H[0])))
    slope = np.polyfit(np.log(dts), np.log(errs), 1)[0]
    assert 1.8 < slope < 2.2, (errs, slope)


def _point_system(k_rest, d0, T=300.0):
    lig = S.one_atom_ligand(charge=0.0)
    g = S.cube_grid(np.zeros(3), 1.0, 3)
    z = np.zeros((3, 3, 3))
    return oracle.OracleSystem(g, z, z, z, lig, [T], [np.nan], [4.0], site=np.zeros(3), k_rest=k_rest, d0=d0)


def test_hmc_samples_harmonic_well_variance():
    k = 23.9
    osys = _point_system(k, 0.0)
    R = 512
    x = np.zeros((R, 1, 3))
    state = np.zeros(R, dtype=np.int32)
    vals = []
    for cyc in range(120):
        x, comps, dH, acc, _ = osys.hmc(x, state, 30, seed=5, cycle=cyc)
        if cyc >= 20:
            vals.append((x[:, 0, :] ** 2).sum(-1))
    vals = np.array(vals)  # [cycles, R]
    per_rep = vals.mean(0)
    mean, se = per_rep.mean(), per_rep.std(ddof=1) / np.sqrt(R)
    exact = 3 * oracle.KB * 300.0 / k
    assert abs(mean - exact) < 4 * se + 1e-12, (mean, exact, se)


def test_hmc_samples_flat_bottom_restraint():
    k, d0 = oracle.K_RESTRAINT, 2.0
    T = 600.0
    osys = _point_system(k, d0, T=T)
    b = oracle.beta(T)
    w = lambda r: r * r * np.exp(-0.5 * b * k * max(r - d0, 0.0) ** 2)
    Z = integrate.quad(w, 0, d0 + 3, points=[d0])[0]
    m2 = integrate.quad(lambda r: r * r * w(r), 0, d0 + 3, points=[d0])[0] / Z
    R = 512
    rng = np.random.default_rng(3)
    u = rng.normal(size=(R, 3))
    x = (u / np.linalg.norm(u, axis=1)[:, None] * d0 * rng.uniform(0, 1, (R, 1)) ** (1 / 3))[:, None, :]
    state = np.zeros(R, dtype=np.int32)
    vals = []
    for cyc in range(150):
        x, comps, dH, acc, _ = osys.hmc(x, state, 30, seed=6, cycle=cyc)
        if cyc >= 20:
            vals.append((x[:, 0, :] ** 2).sum(-1))
    per_rep = np.array(vals).mean(0)
    mean, se = per_rep.mean(), per_rep.std(ddof=1) / np.sqrt(R)
    assert abs(mean - m2) < 4 * se, (mean, m2, se)


def test_hmc_accept_rule_and_rejection_restores(pocket):
    sys_, osys, x0 = pocket
    R = 16
    x = np.repeat(x0[None], R, 0)
    state = np.arange(R, dtype=np.int32) % osys.K
    xn, comps, dH, acc, _ = osys.hmc(x, state, 10, seed=9, cycle=3)
    for r in range(R):
        if not acc[r]:
            assert np.array_equal(xn[r], x[r])
        c, _ = osys.energy_force(xn[r])
        assert np.allclose(c, comps[r], rtol=1e-12, atol=1e-12)
