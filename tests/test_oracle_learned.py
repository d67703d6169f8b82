"""Oracle pins for the learned pose proposal (an extension of the paper's external-coordinate
moves, "Sampling"): the move is an involution with unit Jacobian, torsion increments are exact,
the network and mixture gradients match finite differences, the mixture is a normalised density
sampled correctly, and the involutive Metropolis-Hastings chain reproduces closed-form
equilibrium distributions even with an arbitrary (random) network."""
import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_1507_03703_gb300 import synthetic as S


def _vacuum(lig, T=300.0, k_rest=oracle.K_RESTRAINT, d0=oracle.D0):
    g = S.cube_grid(np.zeros(3), 1.0, 3)
    z = np.zeros((3, 3, 3))
    return oracle.OracleSystem(g, z, z, z, lig, [T], [np.nan], [2.0], site=np.zeros(3), k_rest=k_rest, d0=d0)


def test_move_is_an_involution_with_unit_jacobian():
    lig = S.make_ligand(7, seed=3)
    osys = _vacuum(lig)
    T = osys.learned_ntorsions()
    assert T >= 1
    rng = np.random.default_rng(0)
    x = lig.x0
    for _ in range(5):
        d = rng.normal(scale=0.7, size=6 + T)
        y = osys.apply(x, d)
        assert np.max(np.abs(osys.apply(y, -d) - x)) < 1e-12
    d = rng.normal(scale=0.5, size=6 + T)
    n = 3 * lig.n_atoms
    J = np.zeros((n, n))
    h = 1e-6
    for i in range(n):
        xp, xm = x.ravel().copy(), x.ravel().copy()
        xp[i] += h
        xm[i] -= h
        J[:, i] = (osys.apply(xp.reshape(-1, 3), d).ravel() - osys.apply(xm.reshape(-1, 3), d).ravel()) / (2 * h)
    assert abs(np.linalg.det(J) - 1.0) < 1e-6


def test_torsion_increments_are_exact_and_internal_geometry_kept():
    lig = S.make_ligand(12, seed=4)
    osys = _vacuum(lig)
    T = osys.learned_ntorsions()
    rng = np.random.default_rng(1)
    d = np.zeros(6 + T)
    d[6:] = rng.uniform(-2.0, 2.0, size=T)
    x = lig.x0
    y = osys.apply(x, d)
    back = osys.pose_delta(x, y)[6:]
    wrap = (back - d[6:] + np.pi) % (2 * np.pi) - np.pi
    assert np.max(np.abs(wrap)) < 1e-10
    for a, b in lig.bonds:  # bond lengths unchanged
        assert np.linalg.norm(y[a] - y[b]) == pytest.approx(np.linalg.norm(x[a] - x[b]), abs=1e-12)
    for i, j, k in lig.angles:
        def ang(z):
            u, w = z[i] - z[j], z[k] - z[j]
            return np.arccos(np.dot(u, w) / np.linalg.norm(u) / np.linalg.norm(w))
        assert ang(y) == pytest.approx(ang(x), abs=1e-10)
    # a pure rigid move: translation of the centre of mass by t, rotation recovered
    d = np.zeros(6 + T)
    d[:3] = [0.3, -1.1, 0.5]
    d[3:6] = [0.2, 0.4, -0.3]
    y = osys.apply(x, d)
    est = osys.pose_delta(x, y)
    assert np.allclose(est[:6], d[:6], atol=1e-10)


def _params(seed):
    return S.mlp_init(seed, out_scale=0.5)


def test_mlp_backward_matches_finite_differences():
    p = _params(2)
    rng = np.random.default_rng(3)
    X = rng.normal(size=(3, oracle.NFEAT))
    dout = rng.normal(size=(3, oracle.NOUT))
    out, h1, h2, h3 = oracle.mlp_forward(p, X)
    g = oracle.mlp_backward(p, X, h1, h2, h3, dout)
    obj = lambda q: float(np.sum(oracle.mlp_forward(q, X)[0] * dout))
    for key in oracle._MLP_KEYS:
        flat = p[key].ravel()
        for idx in rng.choice(flat.size, size=4, replace=False):
            q = {k: v.copy() for k, v in p.items()}
            eps = 1e-6
            q[key].ravel()[idx] += eps
            fp = obj(q)
            q[key].ravel()[idx] -= 2 * eps
            fm = obj(q)
            fd = (fp - fm) / (2 * eps)
            assert g[key].ravel()[idx] == pytest.approx(fd, rel=1e-5, abs=1e-7), (key, idx)


def test_mixture_gradient_and_normalisation():
    rng = np.random.default_rng(4)
    o = rng.normal(size=oracle.NOUT)
    D = 7
    dl = rng.normal(size=D)
    lq, g = oracle.mixture_logq(o, D, dl, grad=True)
    for idx in list(range(8)) + list(rng.choice(np.arange(8, oracle.NOUT), size=30, replace=False)):
        op, om = o.copy(), o.copy()
        op[idx] += 1e-6
        om[idx] -= 1e-6
        fd = (oracle.mixture_logq(op, D, dl) - oracle.mixture_logq(om, D, dl)) / 2e-6
        assert g[idx] == pytest.approx(fd, rel=1e-5, abs=1e-8)
    # a 1-D mixture integrates to one
    o1 = rng.normal(scale=0.5, size=oracle.NOUT)
    Z = integrate.quad(lambda t: np.exp(oracle.mixture_logq(o1, 1, [t])), -40, 40, limit=400)[0]
    assert Z == pytest.approx(1.0, abs=1e-8)


def test_mixture_samples_follow_the_density():
    rng = np.random.default_rng(5)
    o = rng.normal(scale=0.8, size=oracle.NOUT)
    D = 2
    xs = np.array([oracle.mixture_sample(o, D, 11, r, 0) for r in range(20000)])
    w = np.exp(o[:8] - o[:8].max())
    w /= w.sum()
    mu = o[8:8 + 8 * 22].reshape(8, 22)[:, :D]
    sig = np.exp(-2 + 4 * np.tanh(o[8 + 8 * 22:].reshape(8, 22)[:, :D] / 4))
    mean = (w[:, None] * mu).sum(0)
    var = (w[:, None] * (sig ** 2 + mu ** 2)).sum(0) - mean ** 2
    se = np.sqrt(var / len(xs))
    assert np.all(np.abs(xs.mean(0) - mean) < 5 * se)


def test_learned_chain_samples_a_harmonic_well():
    """One atom, pure harmonic restraint (d0 = 0), no grid: with a random network the chain of
    learned proposals still gives <|r - c|^2> = 3 kT / k (the proposal depends on the position
    through the features, so it is asymmetric and the q ratio matters)."""
    k = 5.0
    osys = _vacuum(S.one_atom_ligand(charge=0.0), k_rest=k, d0=0.0)
    p = _params(6)
    R = 256
    rng = np.random.default_rng(7)
    x = rng.normal(scale=0.3, size=(R, 1, 3))
    comps = np.array([osys.energy_force(xi)[0] for xi in x])
    vals = []
    for cyc in range(80):
        x, comps, acc, _ = osys.learned_mh(p, x, comps, np.zeros(R, dtype=np.int32), 4, seed=8, cycle=cyc)
        if cyc >= 10:
            vals.append((x[:, 0, :] ** 2).sum(-1))
    per = np.array(vals).mean(0)
    exact = 3 * oracle.KB * 300.0 / k
    assert abs(per.mean() - exact) < 4 * per.std(ddof=1) / np.sqrt(R), (per.mean(), exact)


def test_learned_chain_samples_the_dihedral_marginal():
    """A 4-atom chain in vacuum: the learned move changes only the rigid-body pose and the one
    torsion, so the sampled dihedral follows p(phi) ~ exp(-beta (V_tors(phi) + E_14(phi)))."""
    lig = S.Ligand(
        mass=np.full(4, 12.0), charge=np.array([0.3, 0.0, 0.0, -0.3]), rstar=np.full(4, 1.7),
        eps=np.full(4, 0.1), bonds=np.array([[0, 1], [1, 2], [2, 3]], dtype=np.int32), bond_k=np.full(3, 400.0),
        bond_r0=np.full(3, 1.5), angles=np.array([[0, 1, 2], [1, 2, 3]], dtype=np.int32), angle_k=np.full(2, 60.0),
        angle_theta0=np.full(2, np.radians(110.0)), torsions=np.array([[0, 1, 2, 3]], dtype=np.int32),
        torsion_V=np.array([[0.8, 0.4, 1.5]]), torsion_gamma=np.array([[0.0, np.pi, 0.0]]), x0=np.zeros((4, 3)))
    th = np.radians(110.0)
    x0 = np.array([[1.5 * np.sin(th), 0.0, 1.5 * np.cos(th)], [0, 0, 0], [0, 0, 1.5],
                   [1.5 * np.sin(th), 0.0, 1.5 - 1.5 * np.cos(th)]])
    osys = _vacuum(lig, d0=50.0)
    assert osys.learned_ntorsions() == 1
    beta = oracle.beta(300.0)

    def phi_of(x):
        b1, b2, b3 = x[1] - x[0], x[2] - x[1], x[3] - x[2]
        n1, n2 = np.cross(b1, b2), np.cross(b2, b3)
        return np.arctan2(np.linalg.norm(b2) * np.dot(b1, n2), np.dot(n1, n2))

    def energy_at(phi):
        y = osys.apply(x0, [0, 0, 0, 0, 0, 0, phi - phi_of(x0)])
        return osys.energy_force(y)[0][0]

    p = _params(9)
    p["b4"][8 + 8 * 22:] = 2.0  # log sigma ~ -0.15: moves of ~0.9 rad, so the chains mix quickly
    R = 512
    rng = np.random.default_rng(12)
    x = np.array([osys.apply(x0, [0, 0, 0, 0, 0, 0, t]) for t in rng.uniform(-np.pi, np.pi, size=R)])
    comps = np.array([osys.energy_force(xi)[0] for xi in x])
    phis = []
    for cyc in range(60):
        x, comps, acc, _ = osys.learned_mh(p, x, comps, np.zeros(R, dtype=np.int32), 3, seed=10, cycle=cyc)
        if cyc >= 10:
            phis.extend(phi_of(xi) for xi in x)
    edges = np.linspace(-np.pi, np.pi, 13)
    hist = np.histogram(phis, bins=edges)[0]
    w = np.array([integrate.quad(lambda t: np.exp(-beta * energy_at(t)), a, b)[0] for a, b in zip(edges[:-1],
                                                                                                   edges[1:])])
    expect = w / w.sum() * len(phis)
    # samples within a chain are correlated: allow a generous multiple of the Poisson error
    assert np.all(np.abs(hist - expect) < 6 * np.sqrt(expect * 5) + 20), (hist, expect.round())


def test_features_of_a_closed_form_geometry():
    """The feature vector (reading L1 of the learned proposal's definitions) of a four-atom chain
    whose every feature is known in closed form: equal masses (the centre of mass is the mean of
    the positions), a dihedral of exactly 60 degrees about the one rotatable bond 1-2 (cos 1/2,
    sin sqrt(3)/2 with the usual sign convention), a state with alpha = 1/2 (alpha_sg = 1 and
    alpha_g = 0 exactly) at 450 K, and components whose asinh(c / 10) are 1, 0, -1/2, 2."""
    lig = S.make_ligand(4, seed=7)
    lig.bonds = np.array([[0, 1], [1, 2], [2, 3]], dtype=np.int32)
    lig.angles = np.array([[0, 1, 2], [1, 2, 3]], dtype=np.int32)
    lig.angle_k, lig.angle_theta0 = np.full(2, 60.0), np.full(2, 1.9)
    lig.torsions = np.array([[0, 1, 2, 3]], dtype=np.int32)
    lig.torsion_V, lig.torsion_gamma = np.zeros((1, 3)), np.zeros((1, 3))
    lig.bond_k, lig.bond_r0 = np.full(3, 300.0), np.full(3, 1.5)
    lig.mass = np.full(4, 12.0)
    phi = np.pi / 3
    x = np.array([[0.0, 1.5, 0.0], [0.0, 0.0, 0.0], [1.5, 0.0, 0.0],
                  [1.5, 1.5 * np.cos(phi), 1.5 * np.sin(phi)]])
    site = np.array([0.25, -0.5, 1.0])
    g = S.cube_grid(np.zeros(3), 1.0, 3)
    z = np.zeros((3, 3, 3))
    osys = oracle.OracleSystem(g, z, z, z, lig, [450.0], [0.5], [2.0], site=site, d0=4.0)
    assert osys.learned_ntorsions() == 1
    comps = np.array([10 * np.sinh(1.0), 0.0, -10 * np.sinh(0.5), 10 * np.sinh(2.0)])
    f = osys.features(x, comps, 0)
    com = np.array([0.75, (1.5 + 0.75) / 4, 1.5 * np.sqrt(3) / 8])
    want = np.zeros(64)
    want[0:3] = (com - site) / 4.0
    want[3:6] = (x[0] - com) / np.linalg.norm(x[0] - com)
    want[6:9] = (x[3] - com) / np.linalg.norm(x[3] - com)
    want[9:11] = [0.5, np.sqrt(3) / 2]
    want[41:44] = [1.0, 0.0, 2.0 / 3.0]
    want[44:48] = [1.0, 0.0, -0.5, 2.0]
    assert np.max(np.abs(f - want)) < 1e-12, np.nonzero(np.abs(f - want) > 1e-12)
    # the opposite handedness flips only the sine
    x2 = x.copy()
    x2[3, 2] = -x2[3, 2]
    f2 = osys.features(x2, comps, 0)
    assert abs(f2[9] - 0.5) < 1e-12 and abs(f2[10] + np.sqrt(3) / 2) < 1e-12


def test_mlp_forward_of_a_hand_valued_network():
    """A network with a handful of dyadic weights, evaluated by hand: every value is exact in
    FP64, every bias enters, and ReLU cuts exactly the negative pre-activations (h1[1], h1[2],
    h2[1] below), so a dropped bias, a misplaced ReLU or a transposed weight changes the result."""
    oracle.set_bf16_activations(False)
    p = {"W1": np.zeros((256, 64)), "b1": np.zeros(256), "W2": np.zeros((256, 256)), "b2": np.zeros(256),
         "W3": np.zeros((256, 256)), "b3": np.zeros(256), "W4": np.zeros((360, 256)), "b4": np.zeros(360)}
    p["W1"][0, 0], p["b1"][0] = 2.0, -1.0      # h1[0] = relu(2 - 1) = 1
    p["W1"][1, 0], p["b1"][1] = -3.0, 0.5      # h1[1] = relu(-3 + 0.5) = 0
    p["W1"][2, 1] = 1.0                        # h1[2] = relu(x1 = -2) = 0
    p["W1"][3, 1], p["b1"][3] = -0.25, 0.0     # h1[3] = relu(0.5) = 0.5
    p["W2"][0, 0], p["W2"][0, 1], p["W2"][0, 3], p["b2"][0] = 3.0, 7.0, 0.5, 0.25   # h2[0] = 3 + 0.25 + 0.25 = 3.5
    p["W2"][1, 0], p["b2"][1] = -1.0, 0.5      # h2[1] = relu(-0.5) = 0
    p["W3"][0, 0], p["b3"][0] = 0.5, -1.0      # h3[0] = relu(1.75 - 1) = 0.75
    p["W3"][1, 0], p["W3"][1, 1], p["b3"][1] = 1.0, 9.0, 0.125   # h3[1] = 3.625
    p["W4"][0, 0], p["W4"][0, 1], p["b4"][0] = 2.0, -1.0, 0.5    # out[0] = 1.5 - 3.625 + 0.5 = -1.625
    p["W4"][5, 1] = 1.0                        # out[5] = 3.625
    p["b4"][7] = -4.0                          # out[7] = -4
    X = np.zeros((2, 64))
    X[0, 0], X[0, 1] = 1.0, -2.0
    out, h1, h2, h3 = oracle.mlp_forward(p, X)
    w1 = np.zeros(256)
    w1[[0, 3]] = [1.0, 0.5]
    w2 = np.zeros(256)
    w2[0] = 3.5
    w3 = np.zeros(256)
    w3[[0, 1]] = [0.75, 3.625]
    wo = np.zeros(360)
    wo[[0, 5, 7]] = [-1.625, 3.625, -4.0]
    assert np.array_equal(h1[0], w1) and np.array_equal(h2[0], w2) and np.array_equal(h3[0], w3)
    assert np.array_equal(out[0], wo)
    # the zero input: only the biases that survive ReLU reach the output
    z1 = np.zeros(256)
    z1[1] = 0.5
    assert np.array_equal(h1[1], z1)
    assert h2[1, 0] == 0.25 + 7.0 * 0.5 and h2[1, 1] == 0.5
