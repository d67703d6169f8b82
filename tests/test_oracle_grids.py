"""Oracle pins for the receptor grids and their interpolation (Methodology, "Thermodynamic
Cycle": electrostatic and van der Waals grids, power-4 transform, soft grids)."""
import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator

import oracle
from paper_1507_03703_gb300 import synthetic as S


def _grid(n=9, h=0.5, center=(0.0, 0.0, 0.0)):
    return S.cube_grid(np.array(center), h, n)


def _rgi(L, g):
    ax = [g.origin[d] + g.spacing * np.arange(g.n[d]) for d in range(3)]
    return RegularGridInterpolator(tuple(ax), np.transpose(L, (2, 1, 0)), method="linear")


def test_interp_exact_at_nodes():
    g = _grid(7, 0.4)
    rng = np.random.default_rng(0)
    L = rng.normal(size=(7, 7, 7))
    for _ in range(50):
        i, j, k = rng.integers(0, 7, size=3)
        x = g.origin + g.spacing * np.array([i, j, k])
        v, _ = oracle.interp(L, g, x)
        assert v == pytest.approx(L[k, j, i], abs=1e-13)


def test_interp_reproduces_affine_and_trilinear_fields():
    g = _grid(8, 0.5, center=(1.0, -2.0, 0.5))
    rng = np.random.default_rng(1)
    nodes = np.stack(np.meshgrid(*[g.origin[d] + g.spacing * np.arange(g.n[d]) for d in range(3)],
                                 indexing="ij"), -1)  # [x,y,z,3]
    a, b = rng.normal(size=3), rng.normal()
    aff = (nodes @ a + b).transpose(2, 1, 0)
    c = rng.normal(size=(3, 2))
    tri = ((c[0, 0] + c[0, 1] * nodes[..., 0]) * (c[1, 0] + c[1, 1] * nodes[..., 1])
           * (c[2, 0] + c[2, 1] * nodes[..., 2])).transpose(2, 1, 0)
    lo, hi = g.origin, g.origin + g.spacing * (np.array(g.n) - 1)
    for _ in range(100):
        x = rng.uniform(lo, hi)
        v, grad = oracle.interp(aff, g, x)
        assert v == pytest.approx(x @ a + b, abs=1e-11)
        assert np.allclose(grad, a, atol=1e-10)
        v, grad = oracle.interp(tri, g, x)
        f = [c[d, 0] + c[d, 1] * x[d] for d in range(3)]
        assert v == pytest.approx(f[0] * f[1] * f[2], abs=1e-10)
        exact_grad = [c[0, 1] * f[1] * f[2], f[0] * c[1, 1] * f[2], f[0] * f[1] * c[2, 1]]
        assert np.allclose(grad, exact_grad, atol=1e-9)


def test_interp_matches_scipy_regular_grid_interpolator():
    g = _grid(11, 0.25)
    rng = np.random.default_rng(2)
    L = rng.normal(size=(11, 11, 11)) ** 3
    f = _rgi(L, g)
    lo, hi = g.origin, g.origin + g.spacing * 10
    pts = rng.uniform(lo, hi, size=(200, 3))
    ref = f(pts)
    for p, r in zip(pts, ref):
        assert oracle.interp(L, g, p)[0] == pytest.approx(r, abs=1e-12)


def test_interp_clamps_outside_with_zero_normal_gradient():
    g = _grid(5, 1.0)
    rng = np.random.default_rng(3)
    L = rng.normal(size=(5, 5, 5))
    inside = np.array([0.3, -0.7, 1.1])
    out = inside.copy()
    out[0] = g.origin[0] - 3.0
    v_out, g_out = oracle.interp(L, g, out)
    edge = inside.copy()
    edge[0] = g.origin[0]
    v_edge, g_edge = oracle.interp(L, g, edge)
    assert v_out == pytest.approx(v_edge, abs=1e-14)
    assert g_out[0] == 0.0 and g_out[1] == pytest.approx(g_edge[1]) and g_out[2] == pytest.approx(g_edge[2])
    out[2] = g.origin[2] + 9.0
    v2, g2 = oracle.interp(L, g, out)
    assert g2[0] == 0.0 and g2[2] == 0.0


def _one_atom_system(g, ljr, lja, elec, lig, T=300.0, alpha=1.0):
    return oracle.OracleSystem(g, ljr, lja, elec, lig, [T], [alpha], [2.0], site=g.center)


@pytest.mark.parametrize("dist_factor", [1.0, 2.0 ** (-1.0 / 6.0), 1.3])
def test_grid_node_energy_is_the_lj_pair_potential(dist_factor):
    """One receptor atom and a one-atom ligand at a node: the grid energy equals the 12-6 pair
    potential with geometric combining, eps_ij [(R_ij/r)^12 - 2 (R_ij/r)^6] with
    eps_ij = sqrt(eps_i eps_j) and R_ij = 2 sqrt(R*_i R*_j): depth -eps_ij at r = R_ij and zero at
    r = R_ij 2^(-1/6)."""
    g = _grid(9, 0.5)
    lig = S.one_atom_ligand(rstar=1.7, eps=0.15, charge=0.0)
    rs_j, e_j = 1.9, 0.08
    R = 2.0 * np.sqrt(1.7 * rs_j) * dist_factor
    node = g.origin + g.spacing * np.array([4, 4, 4])
    rec = S.Receptor(xyz=(node + np.array([R, 0.0, 0.0]))[None, :], rstar=np.array([rs_j]),
                     eps=np.array([e_j]), charge=np.array([0.0]))
    ljr, lja, elec = oracle.grid_direct_sum(rec, g)
    sys_ = _one_atom_system(g, ljr, lja, elec, lig)
    psi, _, _ = sys_.grid_terms(node[None, :])
    eij = np.sqrt(0.15 * e_j)
    Rij = 2.0 * np.sqrt(1.7 * rs_j)
    expect = eij * ((Rij / R) ** 12 - 2.0 * (Rij / R) ** 6)
    assert psi[1] == pytest.approx(expect, rel=1e-11, abs=1e-14)
    if dist_factor == 1.0:
        assert psi[1] == pytest.approx(-eij, rel=1e-11)


def test_grid_node_coulomb_with_distance_dependent_dielectric():
    g = _grid(9, 0.5)
    lig = S.one_atom_ligand(rstar=1.7, eps=0.0, charge=-0.35)
    node = g.origin + g.spacing * np.array([3, 5, 4])
    r = 3.7
    rec = S.Receptor(xyz=(node + np.array([0.0, r, 0.0]))[None, :], rstar=np.array([1.8]),
                     eps=np.array([0.0]), charge=np.array([0.6]))
    ljr, lja, elec = oracle.grid_direct_sum(rec, g)
    sys_ = _one_atom_system(g, ljr, lja, elec, lig)
    psi, _, _ = sys_.grid_terms(node[None, :])
    assert psi[1] == pytest.approx(332.0637 * (-0.35) * 0.6 / (4.0 * r * r), rel=1e-12)


def test_grid_direct_sum_is_additive_over_receptor_atoms():
    g = _grid(5, 0.7)
    rec = S.make_receptor(30, np.zeros(3), seed=4, pocket_radius=2.0)
    full = oracle.grid_direct_sum(rec, g)
    acc = [np.zeros_like(full[0]) for _ in range(3)]
    for j in range(rec.n_atoms):
        one = S.Receptor(xyz=rec.xyz[j:j + 1], rstar=rec.rstar[j:j + 1], eps=rec.eps[j:j + 1],
                         charge=rec.charge[j:j + 1])
        part = oracle.grid_direct_sum(one, g)
        for a, p in zip(acc, part):
            a += p
    for a, f in zip(acc, full):
        assert np.allclose(a, f, rtol=1e-12, atol=1e-300)


def test_power_four_transform_reproduces_fourth_power_of_trilinear_field():
    """A repulsive grid whose 4th root is affine is reproduced exactly between nodes."""
    g = _grid(8, 0.5)
    rng = np.random.default_rng(5)
    nodes = np.stack(np.meshgrid(*[g.origin[d] + g.spacing * np.arange(g.n[d]) for d in range(3)],
                                 indexing="ij"), -1)
    a = rng.uniform(0.05, 0.2, size=3)
    root = (nodes @ a + 2.0).transpose(2, 1, 0)  # positive everywhere on the lattice
    ljr = root ** 4
    zeros = np.zeros_like(ljr)
    lig = S.one_atom_ligand(rstar=1.6, eps=0.1, charge=0.0)
    sys_ = _one_atom_system(g, ljr, zeros, zeros, lig)
    sA = np.sqrt(0.1 * (2 * 1.6) ** 12)
    lo, hi = g.origin, g.origin + g.spacing * 7
    for _ in range(50):
        x = rng.uniform(lo, hi)
        psi, _, grad_g = sys_.grid_terms(x[None, :])
        lin = x @ a + 2.0
        assert psi[1] == pytest.approx(sA * lin ** 4, rel=1e-11)
        assert np.allclose(grad_g[0], 4.0 * sA * lin ** 3 * a, rtol=1e-10)


def test_soft_caps_bound_energies_per_atom():
    """Soft grids: the repulsive cap v_r bounds each atom's soft repulsion, and the electrostatic
    cap makes |q_i| v_e <= sqrt(A_i) v_r for every ligand atom (equality for the tightest)."""
    lig = S.make_ligand(25, seed=7)
    ve = oracle.soft_elec_cap(lig)
    sA = np.sqrt(lig.eps * (2 * lig.rstar) ** 12)
    lhs = np.abs(lig.charge) * ve
    rhs = sA * oracle.VMAX_R
    assert np.all(lhs <= rhs * (1 + 1e-12))
    assert np.isclose(np.max(lhs / rhs), 1.0, rtol=1e-12)
    rng = np.random.default_rng(8)
    raw_r = 10.0 ** rng.uniform(-6, 12, size=2000)
    raw_e = rng.normal(scale=3000.0, size=2000)
    lr, slr, sle = oracle.prepare_lattices(raw_r, raw_e, oracle.VMAX_R, ve)
    assert np.all(slr ** 4 <= oracle.VMAX_R * (1 + 1e-12))
    assert np.all(np.abs(sle) <= ve * (1 + 1e-12))
    small = raw_r < 1e-4 * oracle.VMAX_R
    assert np.allclose(slr[small] ** 4, raw_r[small], rtol=1e-7)
    assert np.allclose(lr ** 4, np.minimum(raw_r, 1e10), rtol=1e-12)
