"""Oracle pins for the energy terms: analytic forces against central finite differences, and
hand values of each term on 2-5 atom molecules (sampling force field; Eq. (binding_site))."""
import numpy as np
import pytest

import oracle
from paper_1507_03703_gb300 import synthetic as S


@pytest.fixture(scope="module")
def small():
    sys_ = S.config_small(1)
    ljr, lja, elec = oracle.grid_direct_sum(sys_.receptor, sys_.grid)
    leg = sys_.legs[1]
    osys = oracle.OracleSystem(sys_.grid, ljr, lja, elec, sys_.ligand, leg.T, leg.alpha, leg.dt_fs)
    x = S.place_ligand(sys_.ligand, sys_.receptor, sys_.site, 3, seed=0, n_tries=8).astype(np.float64)
    return sys_, osys, x


def _fd(fun, x, h=1e-5):
    g = np.zeros_like(x)
    for i in range(x.shape[0]):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, d] += h
            xm[i, d] -= h
            g[i, d] = (fun(xp) - fun(xm)) / (2 * h)
    return g


@pytest.mark.parametrize("w", [(0.0, 0.0), (1.0, 0.0), (0.0, 1.0), (0.35, 0.8)])
def test_total_force_matches_finite_differences(small, w):
    _, osys, xs = small
    for x in xs:
        comps, F = osys.energy_force(x, *w)
        U = lambda y: (lambda c: c[0] + c[1] + w[0] * c[2] + w[1] * c[3])(osys.energy_force(y, *w)[0])
        Ffd = -_fd(U, x)
        assert np.linalg.norm(F - Ffd) / np.linalg.norm(F) < 1e-6


def test_restraint_force_matches_finite_differences(small):
    _, osys, xs = small
    x = xs[0] + np.array([7.5, 0.0, 0.0])  # push the centre of mass outside d0
    e, F = osys.restraint(x)
    assert e > 0
    Ffd = -_fd(lambda y: osys.restraint(y)[0], x)
    assert np.linalg.norm(F - Ffd) / np.linalg.norm(F) < 1e-7


def _chain(n, **kw):
    """A linear chain 0-1-...-(n-1) with chosen parameters (no grid contribution)."""
    z = S.one_atom_ligand()
    lig = S.Ligand(
        mass=np.full(n, 12.0), charge=kw.get("charge", np.zeros(n)), rstar=np.full(n, 1.7),
        eps=kw.get("eps", np.zeros(n)), bonds=np.array([[i, i + 1] for i in range(n - 1)], dtype=np.int32).reshape(-1, 2),
        bond_k=np.full(n - 1, 400.0), bond_r0=np.full(n - 1, 1.5),
        angles=np.array([[i, i + 1, i + 2] for i in range(n - 2)], dtype=np.int32).reshape(-1, 3),
        angle_k=np.full(max(n - 2, 0), 60.0), angle_theta0=np.full(max(n - 2, 0), np.radians(110.0)),
        torsions=np.array([[i, i + 1, i + 2, i + 3] for i in range(n - 3)], dtype=np.int32).reshape(-1, 4),
        torsion_V=kw.get("V", np.zeros((max(n - 3, 0), 3))),
        torsion_gamma=kw.get("gamma", np.zeros((max(n - 3, 0), 3))), x0=np.zeros((n, 3)))
    g = S.cube_grid(np.zeros(3), 1.0, 3)
    zero = np.zeros((3, 3, 3))
    return lig, oracle.OracleSystem(g, zero, zero, zero, lig, [300.0], [np.nan], [2.0], site=np.zeros(3))


def test_bond_hand_value():
    lig, osys = _chain(2)
    x = np.array([[0, 0, 0], [1.6, 0, 0]], dtype=float)
    e, F, terms = osys.ligand_ff(x)
    assert terms[0] == pytest.approx(400.0 * 0.1 ** 2, rel=1e-12)
    assert F[0, 0] == pytest.approx(2 * 400.0 * 0.1, rel=1e-12)  # pulled toward atom 1
    assert F[1, 0] == pytest.approx(-2 * 400.0 * 0.1, rel=1e-12)


def test_angle_hand_value():
    lig, osys = _chain(3)
    th = np.radians(110.0) + 0.1
    x = np.array([[1.5, 0, 0], [0, 0, 0], [1.5 * np.cos(th), 1.5 * np.sin(th), 0]])
    _, _, terms = osys.ligand_ff(x)
    assert terms[1] == pytest.approx(60.0 * 0.1 ** 2, rel=1e-10)
    assert terms[0] == pytest.approx(0.0, abs=1e-20)


@pytest.mark.parametrize("phi_deg", [0.0, 60.0, 180.0, -100.0])
def test_torsion_hand_value(phi_deg):
    V = np.array([[1.3, 0.7, 0.4]])
    gam = np.array([[0.0, np.pi, 0.0]])
    lig, osys = _chain(4, V=V, gamma=gam)
    phi = np.radians(phi_deg)
    th = np.radians(110.0)
    # i on the -x side, j at origin, k on +z axis, l rotated by phi about z (IUPAC sign)
    x = np.array([[1.5 * np.sin(th), 0.0, 1.5 * np.cos(th)], [0, 0, 0], [0, 0, 1.5],
                  [1.5 * np.sin(th) * np.cos(phi), 1.5 * np.sin(th) * np.sin(phi), 1.5 - 1.5 * np.cos(th)]])
    _, _, terms = osys.ligand_ff(x)
    expect = sum(0.5 * V[0, n - 1] * (1 + np.cos(n * phi - gam[0, n - 1])) for n in (1, 2, 3))
    assert terms[2] == pytest.approx(expect, rel=1e-10, abs=1e-12)
    assert terms[1] == pytest.approx(0.0, abs=1e-18)


def test_nonbonded_exclusions_and_one_four_scaling():
    n = 5
    lig, osys = _chain(n, eps=np.full(n, 0.1), charge=np.array([0.3, 0.0, 0.0, -0.2, 0.5]))
    pairs, slj, sel = osys.pairs()
    got = {(int(a), int(b)): (l, e) for (a, b), l, e in zip(pairs, slj, sel)}
    assert set(got) == {(0, 3), (1, 4), (0, 4)}  # 1-2 and 1-3 excluded
    assert got[(0, 3)] == (0.5, pytest.approx(1 / 1.2)) and got[(1, 4)][0] == 0.5
    assert got[(0, 4)] == (1.0, 1.0)
    # atoms 0 and 4 close together, the rest far apart along x
    x = np.zeros((n, 3))
    x[:, 0] = [0.0, 100.0, 200.0, 300.0, 3.4]
    _, _, terms = osys.ligand_ff(x)
    R = 1.7 + 1.7  # Lorentz-Berthelot: R_ij = R*_i + R*_j

    def lj(r):
        return 0.1 * ((R / r) ** 12 - 2 * (R / r) ** 6)

    def coul(qi, qj, r):
        return 332.0637 * qi * qj / r

    assert lj(3.4) == pytest.approx(-0.1)  # depth eps_ij at r = R_ij
    expect = (lj(3.4) + coul(0.3, 0.5, 3.4)                      # 1-5: unscaled
              + 0.5 * lj(96.6) + coul(0.0, 0.5, 96.6) / 1.2     # 1-4 (1, 4)
              + 0.5 * lj(300.0) + coul(0.3, -0.2, 300.0) / 1.2)  # 1-4 (0, 3)
    assert terms[3] == pytest.approx(expect, rel=1e-12)


def test_restraint_hand_values():
    lig, osys = _chain(2)
    x = np.array([[3.0, 0, 0], [3.0, 0, 0]])  # COM at 3 A: inside the flat bottom
    assert osys.restraint(x)[0] == 0.0
    x = np.array([[6.5, 0, 0], [6.5, 0, 0]])
    e, F = osys.restraint(x)
    k = 10000.0 / 4.184 / 100.0
    assert e == pytest.approx(0.5 * k * 0.25, rel=1e-12)
    assert F[0, 0] == pytest.approx(-k * 0.5 * 0.5, rel=1e-12)  # half the mass on each atom
