"""Oracle pins for the external-coordinate moves ("Sampling": a random rotation about the centre of
mass from a random quaternion, a Gaussian translation of 0.6 A per dimension, the Metropolis
criterion; attempted at states with alpha < 0.01):

- the rotations are proper (orthonormal, det +1) and uniform over the rotation group: the mean of
  R is 0, E[(tr R)^2] = 1, and the rotation angle has the Haar density (1 - cos t)/pi;
- a move keeps every interatomic distance and the intramolecular energy;
- moves happen only at states below the alpha threshold (never on the warming leg);
- a one-atom ligand in a harmonic well has <|r - c|^2> = 3 kT / k;
- a dipole in a uniform field (linear electrostatic grid, exact under trilinear interpolation)
  has <cos theta> = coth(a) - 1/a, a = beta q d E (Langevin), which needs uniform rotations."""
import math

import numpy as np
import pytest

import oracle
from paper_1507_03703_gb300 import synthetic as S


def test_random_rotations_are_proper_and_uniform():
    rng = np.random.default_rng(1)
    n = 20000
    w = rng.integers(0, 2 ** 32, size=(n, 3), dtype=np.uint64)
    Rs = np.array([oracle.random_rotation(*row) for row in w])
    eye = np.einsum("nij,nkj->nik", Rs, Rs)
    assert np.max(np.abs(eye - np.eye(3))) < 1e-12
    assert np.max(np.abs(np.linalg.det(Rs) - 1.0)) < 1e-12
    # Haar measure on SO(3): every entry has mean 0 and variance 1/3; E[tr R] = 0, E[(tr R)^2] = 1
    se = math.sqrt(1.0 / 3.0 / n)
    assert np.max(np.abs(Rs.mean(0))) < 4.5 * se
    tr = np.trace(Rs, axis1=1, axis2=2)
    assert abs(tr.mean()) < 4.5 * tr.std() / math.sqrt(n)
    assert abs((tr ** 2).mean() - 1.0) < 4.5 * (tr ** 2).std() / math.sqrt(n)
    # rotation angle t from tr R = 1 + 2 cos t: CDF (t - sin t) / pi
    t = np.sort(np.arccos(np.clip((tr - 1.0) / 2.0, -1.0, 1.0)))
    cdf = (t - np.sin(t)) / math.pi
    ks = np.max(np.abs(cdf - np.arange(1, n + 1) / n))
    assert ks < 1.63 / math.sqrt(n)  # 1 % level of the Kolmogorov-Smirnov statistic


def _flat_system(lig, elec=None, T=(300.0,), alpha=(0.005,), k_rest=oracle.K_RESTRAINT, d0=oracle.D0):
    grid = S.cube_grid(np.zeros(3), 0.5, 33)
    zero = np.zeros((33, 33, 33))
    return oracle.OracleSystem(grid, zero, zero, zero if elec is None else elec, lig, np.array(T), np.array(alpha),
                               np.full(len(T), 2.0), site=np.zeros(3), k_rest=k_rest, d0=d0)


def test_moves_keep_internal_geometry_and_energy():
    lig = S.make_ligand(12, seed=4)
    osys = _flat_system(lig, d0=100.0)
    x0 = lig.x0[None] + 0.0
    c0 = np.array([osys.energy_force(x0[0])[0]])
    x, c, acc = osys.external_moves(x0, c0, np.zeros(1, np.int32), 30, seed=5, cycle=0)
    # zero grids and a restraint that never acts: the energy never changes, every move is accepted
    assert acc[0] == 30
    d0 = np.linalg.norm(x0[0][:, None] - x0[0][None], axis=-1)
    d1 = np.linalg.norm(x[0][:, None] - x[0][None], axis=-1)
    assert np.max(np.abs(d1 - d0)) < 1e-10
    assert abs(c[0, 0] - c0[0, 0]) < 1e-9 * max(1.0, abs(c0[0, 0]))
    assert np.linalg.norm(x[0].mean(0) - x0[0].mean(0)) > 0.1  # it did move


def test_moves_only_below_the_alpha_threshold():
    lig = S.make_ligand(5, seed=6)
    osys = _flat_system(lig, T=(300.0, 300.0, 300.0, 300.0), alpha=(np.nan, 0.0, 0.009, 0.5))
    x0 = np.repeat(lig.x0[None], 4, axis=0)
    c0 = np.array([osys.energy_force(xi)[0] for xi in x0])
    x, c, acc = osys.external_moves(x0, c0, np.arange(4, dtype=np.int32), 5, seed=7, cycle=1)
    assert acc[0] == 0 and acc[3] == 0 and acc[1] > 0 and acc[2] > 0
    assert np.array_equal(x[0], x0[0]) and np.array_equal(x[3], x0[3])
    assert not np.array_equal(x[1], x0[1])


def test_one_atom_in_a_harmonic_well():
    k = 5.0
    lig = S.one_atom_ligand(charge=0.0)
    osys = _flat_system(lig, k_rest=k, d0=0.0)
    R = 2000
    rng = np.random.default_rng(8)
    x = rng.normal(scale=0.3, size=(R, 1, 3))
    c = np.array([osys.energy_force(xi)[0] for xi in x])
    st = np.zeros(R, dtype=np.int32)
    vals = []
    for cyc in range(40):
        x, c, _ = osys.external_moves(x, c, st, 5, seed=9, cycle=cyc)
        if cyc >= 10:
            vals.append((x[:, 0, :] ** 2).sum(-1))
    per = np.array(vals).mean(0)
    exact = 3 * oracle.KB * 300.0 / k
    assert abs(per.mean() - exact) < 4 * per.std(ddof=1) / math.sqrt(R), (per.mean(), exact)


def test_dipole_in_a_uniform_field_follows_the_langevin_function():
    q, bond, E0, T = 0.5, 1.5, 1.2, 300.0  # e, A, kcal/(mol A e), K
    lig = S.Ligand(mass=np.array([12.0, 12.0]), charge=np.array([q, -q]), rstar=np.array([1.8, 1.8]),
                   eps=np.array([0.1, 0.1]), bonds=np.array([[0, 1]], dtype=np.int32), bond_k=np.array([400.0]),
                   bond_r0=np.array([bond]), angles=np.zeros((0, 3), dtype=np.int32), angle_k=np.zeros(0),
                   angle_theta0=np.zeros(0), torsions=np.zeros((0, 4), dtype=np.int32),
                   torsion_V=np.zeros((0, 3)), torsion_gamma=np.zeros((0, 3)),
                   x0=np.array([[0.0, 0.0, 0.5 * bond], [0.0, 0.0, -0.5 * bond]]))
    grid = S.cube_grid(np.zeros(3), 0.5, 33)
    ax = grid.origin[2] + grid.spacing * np.arange(33)
    elec = np.broadcast_to(-E0 * ax[:, None, None], (33, 33, 33)).copy()  # phi = -E0 z, [z][y][x]
    zero = np.zeros((33, 33, 33))
    # alpha = 1: only the hard grids (w_g = 1), whose electrostatic channel is linear in z
    osys = oracle.OracleSystem(grid, zero, zero, elec, lig, np.array([T]), np.array([1.0]), np.array([2.0]),
                               site=np.zeros(3))
    R = 1500
    x = np.repeat(lig.x0[None], R, axis=0)
    c = np.array([osys.energy_force(xi)[0] for xi in x[:1]] * R)
    st = np.zeros(R, dtype=np.int32)
    vals = []
    for cyc in range(30):
        x, c, _ = osys.external_moves(x, c, st, 4, seed=10, cycle=cyc, alpha_max=1.5)
        if cyc >= 5:
            u = x[:, 0] - x[:, 1]
            vals.append(u[:, 2] / np.linalg.norm(u, axis=1))
    per = np.array(vals).mean(0)
    a = q * bond * E0 / (oracle.KB * T)
    exact = 1.0 / math.tanh(a) - 1.0 / a
    assert abs(per.mean() - exact) < 4 * per.std(ddof=1) / math.sqrt(R), (per.mean(), exact)
