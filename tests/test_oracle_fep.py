"""Oracle pins for the end-point corrections ("Estimation": f_AB and f_DE by free energy
perturbation, Zwanzig 1954; "Thermodynamic Cycle": the target force field computes the
receptor-ligand interaction directly, the sampling force field interpolates grids).

The estimator f = -ln <exp(-du)>:
- a constant du gives exactly that constant, with n_eff = N and no error;
- exact samples of a Gaussian du converge to mu - s^2/2 and of an exponential du to
  ln((lambda + 1) / lambda) (the cumulant generating functions);
- the sign convention: a harmonic well sampled at stiffness k_s and perturbed to k_t gives
  f = (D/2) ln(k_t / k_s), the exact free energy difference;
- shift and permutation invariance, min(du) <= f <= mean(du) (Jensen);
- the reported standard error matches the spread of f over independent batches.

The target interaction:
- one receptor and one ligand atom: the Lennard-Jones part has its minimum -sqrt(eps_i eps_j) at
  r = 2 sqrt(R*_i R*_j), crosses zero at 2^(-1/6) of that, and the electrostatic part falls as
  1/r^2 with the coefficient of a 4r dielectric and Coulomb's constant from CODATA, flat below 2 A;
- ligand atoms on lattice nodes give exactly the hard-grid energy of the sampling force field;
- off the nodes the grid energy converges to it at second order in the spacing;
- the interaction is additive over receptor atoms and invariant under a rigid motion of the whole
  complex."""
import math

import numpy as np
import pytest

import oracle
from paper_1507_03703_gb300 import synthetic as S


# ------------------------------------------------------------------ the estimator
def test_constant_difference_is_exact():
    for c in (-3.25, 0.0, 7.5):
        r = oracle.fep(np.full(17, c))
        assert r["f"] == c and r["n_eff"] == 17.0 and r["sigma"] == 0.0 and r["du_min"] == c


def test_gaussian_and_exponential_closed_forms():
    rng = np.random.default_rng(1)
    mu, s = 1.3, 1.0
    r = oracle.fep(rng.normal(mu, s, size=1_000_000))
    assert abs(r["f"] - (mu - 0.5 * s * s)) < 4 * r["sigma"], r
    lam = 2.0
    r = oracle.fep(rng.exponential(1.0 / lam, size=1_000_000))
    assert abs(r["f"] - math.log((lam + 1.0) / lam)) < 4 * r["sigma"], r


@pytest.mark.parametrize("D", [1, 3])
def test_harmonic_well_perturbation_gives_the_free_energy_difference(D):
    """Samples of u_s = k_s |x|^2 / 2 (beta = 1), target u_t = k_t |x|^2 / 2: the free energy of the
    target relative to the sampling state is (D/2) ln(k_t/k_s)."""
    rng = np.random.default_rng(2 + D)
    ks, kt = 1.0, 1.4
    x = rng.normal(scale=1.0 / math.sqrt(ks), size=(400_000, D))
    r2 = (x * x).sum(1)
    r = oracle.fep(0.5 * (kt - ks) * r2)
    exact = 0.5 * D * math.log(kt / ks)
    assert abs(r["f"] - exact) < 4 * r["sigma"], (r, exact)
    # the reverse direction: the sampling state seen from the target's samples
    y = rng.normal(scale=1.0 / math.sqrt(kt), size=(400_000, D))
    rb = oracle.fep(0.5 * (ks - kt) * (y * y).sum(1))
    assert abs(rb["f"] + exact) < 4 * rb["sigma"]


def test_invariances_and_bounds():
    rng = np.random.default_rng(4)
    du = rng.gamma(2.0, 1.5, size=5000) - 2.0
    r = oracle.fep(du)
    assert du.min() <= r["f"] <= du.mean()
    assert r["du_min"] == du.min()
    r2 = oracle.fep(du + 11.0)
    assert abs(r2["f"] - r["f"] - 11.0) < 1e-12 and abs(r2["n_eff"] - r["n_eff"]) < 1e-9 * r["n_eff"]
    r3 = oracle.fep(rng.permutation(du))
    assert abs(r3["f"] - r["f"]) < 1e-13 and abs(r3["sigma"] - r["sigma"]) < 1e-13
    # one sample dominating every other weight: n_eff -> 1, f -> that sample's du + ln N
    du1 = np.concatenate([[0.0], np.full(99, 50.0)])
    r1 = oracle.fep(du1)
    assert abs(r1["n_eff"] - 1.0) < 1e-12 and abs(r1["f"] - math.log(100.0)) < 1e-12
    assert math.isnan(oracle.fep([3.0])["sigma"]) and oracle.fep([3.0])["f"] == 3.0
    with pytest.raises(ValueError):
        oracle.fep([])


def test_reported_error_matches_the_spread_over_batches():
    rng = np.random.default_rng(5)
    fs, sig = [], []
    for _ in range(400):
        r = oracle.fep(rng.normal(0.0, 0.7, size=800))
        fs.append(r["f"])
        sig.append(r["sigma"])
    spread = np.std(fs, ddof=1)
    assert abs(np.mean(sig) / spread - 1.0) < 0.15, (np.mean(sig), spread)


# ------------------------------------------------------------------ the target interaction
def _atom_pair(ri, ei, qi, rj, ej, qj):
    rec = S.Receptor(xyz=np.zeros((1, 3)), rstar=np.array([rj]), eps=np.array([ej]), charge=np.array([qj]))
    lig = S.one_atom_ligand(rstar=ri, eps=ei, charge=qi)
    return rec, lig


def _psi_at(rec, lig, r):
    x = np.zeros((len(r), 1, 3))
    x[:, 0, 0] = r
    return oracle.target_interaction(rec, lig, x)


def test_pair_lennard_jones_minimum_and_zero_crossing():
    ri, ei, rj, ej = 1.7, 0.15, 1.9, 0.08
    rec, lig = _atom_pair(ri, ei, 0.0, rj, ej, 0.0)
    rho = 2.0 * math.sqrt(ri * rj)
    r = np.linspace(rho - 0.4, rho + 0.4, 8001)
    e = _psi_at(rec, lig, r)
    k = int(np.argmin(e))
    assert abs(r[k] - rho) <= 1e-4 + 0.5 * (r[1] - r[0])
    assert abs(e.min() + math.sqrt(ei * ej)) < 1e-6 * math.sqrt(ei * ej)
    # central differences vanish at rho; the energy crosses zero at 2^(-1/6) rho
    h = 1e-5
    d = _psi_at(rec, lig, np.array([rho + h, rho - h]))
    assert abs((d[0] - d[1]) / (2 * h)) < 1e-6
    r0 = rho * 2.0 ** (-1.0 / 6.0)
    assert abs(_psi_at(rec, lig, np.array([r0]))[0]) < 1e-10


def test_pair_electrostatics_coefficient_and_floor():
    # Coulomb's constant in kcal A / (mol e^2) from CODATA 2018 (exact SI e, N_A; measured eps0)
    e, eps0, NA = 1.602176634e-19, 8.8541878128e-12, 6.02214076e23
    k_e = e * e / (4 * math.pi * eps0) * NA / 4184.0 * 1e10
    qi, qj = 0.37, -0.81
    rec, lig = _atom_pair(1.8, 0.0, qi, 1.8, 0.0, qj)
    r = np.array([2.0, 2.5, 3.0, 5.0, 9.0, 17.0])
    v = _psi_at(rec, lig, r) * r * r / (qi * qj)
    # the 4r dielectric: E = k_e q_i q_j / (4 r^2)
    assert np.all(np.abs(v / (k_e / 4.0) - 1.0) < 2e-7), v
    below = _psi_at(rec, lig, np.array([0.5, 1.0, 1.99]))
    assert np.all(below == _psi_at(rec, lig, np.array([2.0]))[0])


@pytest.fixture(scope="module")
def pocket():
    sys_ = S.config_small(1)
    return sys_


def _node_positions(grid, lig, rng, n):
    """n configurations whose atoms sit on lattice nodes near the site (inside the pocket)."""
    c = (np.asarray(grid.n) - 1) // 2
    x = np.empty((n, lig.n_atoms, 3))
    for s in range(n):
        ijk = c + rng.integers(-6, 7, size=(lig.n_atoms, 3))
        x[s] = grid.origin + grid.spacing * ijk
    return x


def test_on_lattice_nodes_the_target_equals_the_hard_grid_energy(pocket):
    sys_ = pocket
    lig, rec, grid = sys_.ligand, sys_.receptor, sys_.grid
    ljr, lja, elec = oracle.grid_direct_sum(rec, grid)
    osys = oracle.OracleSystem(grid, ljr, lja, elec, lig, [300.0], [1.0], [2.0], site=sys_.site)
    x = _node_positions(grid, lig, np.random.default_rng(6), 12)
    want = np.array([osys.grid_terms(xi)[0][1] for xi in x])
    got = oracle.target_interaction(rec, lig, x)
    assert np.all(np.abs(got - want) <= 1e-11 * np.maximum(1.0, np.abs(want))), (got, want)


def test_grid_energy_converges_to_the_target_at_second_order():
    """Two receptor atoms 4-5 A from a probe region: the trilinear grid energy approaches the
    direct energy as h^2 at off-node points (log-log slope of the RMS error over four spacings)."""
    rec = S.Receptor(xyz=np.array([[0.0, 0.0, -4.0], [1.5, -0.5, -5.0]]), rstar=np.array([1.8, 1.6]),
                     eps=np.array([0.1, 0.15]), charge=np.array([0.5, -0.3]))
    lig = S.one_atom_ligand(rstar=1.7, eps=0.12, charge=0.6)
    pts = np.random.default_rng(7).uniform(-0.7, 0.7, size=(600, 1, 3))
    target = oracle.target_interaction(rec, lig, pts)
    errs = []
    hs = (0.2, 0.1, 0.05, 0.025)
    for h in hs:
        n = int(round(2.0 / h)) + 1
        grid = S.GridSpec(origin=np.full(3, -1.0), spacing=h, n=(n, n, n))
        lat = oracle.grid_direct_sum(rec, grid)
        osys = oracle.OracleSystem(grid, *lat, lig, [300.0], [1.0], [2.0], site=np.zeros(3))
        g = np.array([osys.grid_terms(p)[0][1] for p in pts])
        errs.append(np.sqrt(np.mean((g - target) ** 2)))
    order = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert abs(order - 2.0) < 0.15, (order, errs)


def test_additive_over_receptor_atoms_and_rigid_motion_invariant(pocket):
    sys_ = pocket
    lig, rec = sys_.ligand, sys_.receptor
    x = S.place_ligand(lig, rec, sys_.site, 6, seed=8).astype(np.float64)
    full = oracle.target_interaction(rec, lig, x)
    h = rec.n_atoms // 3
    parts = [S.Receptor(xyz=rec.xyz[sl], rstar=rec.rstar[sl], eps=rec.eps[sl], charge=rec.charge[sl])
             for sl in (slice(0, h), slice(h, None))]
    split = oracle.target_interaction(parts[0], lig, x) + oracle.target_interaction(parts[1], lig, x)
    assert np.allclose(split, full, rtol=1e-12, atol=1e-9)
    R = S.rotation_matrix(np.array([0.3, -0.5, 0.7, 0.4]) / np.linalg.norm([0.3, -0.5, 0.7, 0.4]))
    t = np.array([3.0, -7.0, 11.0])
    moved = S.Receptor(xyz=rec.xyz @ R.T + t, rstar=rec.rstar, eps=rec.eps, charge=rec.charge)
    got = oracle.target_interaction(moved, lig, x @ R.T + t)
    assert np.allclose(got, full, rtol=1e-10, atol=1e-8)
