"""Seeded synthetic inputs shaped like the paper's workloads.

The paper's own inputs (the Astex diverse set, AMBER/GAFF2 parameter files, APBS grids) are not
available, so every system here is generated from a seed with the shapes and parameter ranges of
the paper's calculations (Methodology: ligands of tens of heavy atoms, protein receptors of
thousands of atoms at protein density, grids at 0.25-0.5 A spacing, tens to a hundred
thermodynamic states per leg).

This module draws random numbers and arranges atoms in space; it holds none of the method's
arithmetic (no grid values, no energies, no forces, no state weights).  Both the CUDA path and
the FP64 oracle consume what it returns.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

HEAVY_MASSES = np.array([12.011, 14.007, 15.999])  # C, N, O (amu)


@dataclass
class Ligand:
    """A flexible, acyclic (tree) ligand with a GAFF-like parameter set.

    Units: A, kcal/mol, amu, e, radians.  ``rstar`` is the AMBER per-atom radius R* (half the
    Lennard-Jones minimum distance of a like pair); ``eps`` the well depth.
    """

    mass: np.ndarray
    charge: np.ndarray
    rstar: np.ndarray
    eps: np.ndarray
    bonds: np.ndarray        # int32 [nb, 2]
    bond_k: np.ndarray       # kcal/mol/A^2, energy k (r - r0)^2
    bond_r0: np.ndarray      # A
    angles: np.ndarray       # int32 [na, 3]  (i, j-centre, k)
    angle_k: np.ndarray      # kcal/mol/rad^2, energy k (theta - theta0)^2
    angle_theta0: np.ndarray  # rad
    torsions: np.ndarray     # int32 [nt, 4]
    torsion_V: np.ndarray    # kcal/mol [nt, 3] for n = 1, 2, 3
    torsion_gamma: np.ndarray  # rad [nt, 3], each 0 or pi
    x0: np.ndarray           # start geometry [n, 3], centre of mass at the origin

    @property
    def n_atoms(self) -> int:
        return int(self.mass.shape[0])


@dataclass
class Receptor:
    """A rigid receptor: atoms at protein heavy-atom density around a surface pocket."""

    xyz: np.ndarray
    rstar: np.ndarray
    eps: np.ndarray
    charge: np.ndarray

    @property
    def n_atoms(self) -> int:
        return int(self.xyz.shape[0])


@dataclass
class GridSpec:
    """A regular lattice: node (i, j, k) sits at origin + h * (i, j, k); x varies fastest."""

    origin: np.ndarray
    spacing: float
    n: tuple

    @property
    def n_nodes(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])

    @property
    def center(self) -> np.ndarray:
        return self.origin + 0.5 * self.spacing * (np.asarray(self.n, dtype=np.float64) - 1.0)


@dataclass
class Ladder:
    """One replica-exchange leg: temperatures (K) and alchemical progress (NaN = no grid)."""

    T: np.ndarray
    alpha: np.ndarray
    dt_fs: np.ndarray

    @property
    def K(self) -> int:
        return int(self.T.shape[0])


@dataclass
class System:
    ligand: Ligand
    receptor: Receptor
    grid: GridSpec
    site: np.ndarray
    legs: list = field(default_factory=list)


def _unit(v):
    return v / np.linalg.norm(v)


def _random_unit(rng):
    while True:
        v = rng.normal(size=3)
        n = np.linalg.norm(v)
        if n > 1e-6:
            return v / n


def make_ligand(n_atoms: int, seed: int, max_degree: int = 3, min_sep: float = None) -> Ligand:
    """Random tree topology grown atom by atom, with a clash-free start geometry.

    Parameter ranges: bonds 1.3-1.6 A with k 300-500 kcal/mol/A^2; angles 105-120 deg with
    k 50-80 kcal/mol/rad^2; three cosine torsion terms V_n in [0, 2] kcal/mol with phase 0 or pi;
    R* in [1.5, 2.0] A; eps in [0.01, 0.2] kcal/mol; charges N(0, 0.3) e shifted to net zero;
    masses of C, N or O.

    min_sep (A): grow every new atom at least this far from all atoms other than its parent and
    the parent's neighbours, trying the open parents in random order (large trees otherwise crowd
    atoms into clashes).  None keeps the original growth (and its random draws).
    """
    if n_atoms < 1:
        raise ValueError("n_atoms must be >= 1")
    rng = np.random.default_rng(np.random.SeedSequence([0x4C1, seed]))
    parent = [-1]
    degree = [0]
    pos = [np.zeros(3)]
    bond_r0 = []
    nbrs = [[]]

    def grow(a, p, r0):
        best, best_score = None, -np.inf
        for _ in range(400):
            d = _random_unit(rng)
            # prefer ~109.5 deg to the existing bonds at the parent
            angs = [np.degrees(np.arccos(np.clip(np.dot(d, _unit(pos[q] - pos[p])), -1, 1)))
                    for q in nbrs[p]]
            ang_pen = max([abs(t - 109.5) for t in angs], default=0.0)
            cand = pos[p] + r0 * d
            others = [pos[q] for q in range(a) if q != p]
            dmin = min([np.linalg.norm(cand - o) for o in others], default=10.0)
            score = min(dmin, 3.0) * 10.0 - ang_pen
            if score > best_score:
                best, best_score = cand, score
            if dmin >= 2.9 and ang_pen < 8.0:
                break
        return best

    def grow_apart(a, p, r0, sep, n_try=400):
        # all candidate directions at once; the first that keeps sep from every atom other than
        # the parent and its neighbours with a near-tetrahedral angle, else the best scored
        D = rng.normal(size=(n_try, 3))
        D /= np.linalg.norm(D, axis=1)[:, None]
        P = np.array(pos)
        cand = P[p] + r0 * D
        if nbrs[p]:
            U = P[nbrs[p]] - P[p]
            U /= np.linalg.norm(U, axis=1)[:, None]
            ang_pen = np.abs(np.degrees(np.arccos(np.clip(D @ U.T, -1.0, 1.0))) - 109.5).max(axis=1)
        else:
            ang_pen = np.zeros(n_try)
        keep = [q for q in range(a) if q != p and q not in nbrs[p]]
        if keep:
            dmin = np.linalg.norm(cand[:, None, :] - P[keep][None], axis=2).min(axis=1)
        else:
            dmin = np.full(n_try, 10.0)
        ok = (dmin >= sep) & (ang_pen < 12.0)
        if ok.any():
            return cand[int(np.argmax(ok))], True
        score = np.minimum(dmin, sep + 0.5) * 10.0 - ang_pen
        return cand[int(np.argmax(score))], False

    for a in range(1, n_atoms):
        cands = [p for p in range(a) if degree[p] < max_degree]
        if min_sep is None:
            p = int(rng.choice(cands))
            r0 = float(rng.uniform(1.3, 1.6))
            best = grow(a, p, r0)
        else:
            fallback = None
            for p in rng.permutation(cands):
                p = int(p)
                r0 = float(rng.uniform(1.3, 1.6))
                best, ok = grow_apart(a, p, r0, float(min_sep))
                if ok:
                    break
                if fallback is None:
                    fallback = (p, r0, best)
            if not ok:
                p, r0, best = fallback
        parent.append(p)
        degree.append(1)
        degree[p] += 1
        nbrs.append([p])
        nbrs[p].append(a)
        pos.append(best)
        bond_r0.append(r0)
    x0 = np.array(pos)
    bonds = np.array([[parent[a], a] for a in range(1, n_atoms)], dtype=np.int32).reshape(-1, 2)
    nb = bonds.shape[0]
    bond_k = rng.uniform(300.0, 500.0, size=nb)
    bond_r0 = np.array(bond_r0, dtype=np.float64)
    angles = []
    for j in range(n_atoms):
        nj = sorted(nbrs[j])
        for u in range(len(nj)):
            for w in range(u + 1, len(nj)):
                angles.append([nj[u], j, nj[w]])
    angles = np.array(angles, dtype=np.int32).reshape(-1, 3)
    na = angles.shape[0]
    angle_k = rng.uniform(50.0, 80.0, size=na)
    angle_theta0 = np.radians(rng.uniform(105.0, 120.0, size=na))
    torsions = []
    for (j, k) in bonds:
        for i in sorted(nbrs[j]):
            if i == k:
                continue
            for l in sorted(nbrs[k]):
                if l == j:
                    continue
                torsions.append([i, j, k, l])
    torsions = np.array(torsions, dtype=np.int32).reshape(-1, 4)
    nt = torsions.shape[0]
    torsion_V = rng.uniform(0.0, 2.0, size=(nt, 3))
    torsion_gamma = np.pi * rng.integers(0, 2, size=(nt, 3)).astype(np.float64)
    mass = HEAVY_MASSES[rng.integers(0, 3, size=n_atoms)]
    rstar = rng.uniform(1.5, 2.0, size=n_atoms)
    eps = rng.uniform(0.01, 0.2, size=n_atoms)
    charge = rng.normal(0.0, 0.3, size=n_atoms)
    if n_atoms > 1:
        charge = charge - charge.mean()
    com = (mass[:, None] * x0).sum(0) / mass.sum()
    x0 = x0 - com
    return Ligand(mass=mass, charge=charge, rstar=rstar, eps=eps, bonds=bonds, bond_k=bond_k,
                  bond_r0=bond_r0, angles=angles, angle_k=angle_k, angle_theta0=angle_theta0,
                  torsions=torsions, torsion_V=torsion_V, torsion_gamma=torsion_gamma, x0=x0)


def one_atom_ligand(rstar=1.8, eps=0.1, charge=0.4, mass=12.011) -> Ligand:
    """A single-atom ligand (no intramolecular terms)."""
    z2 = np.zeros((0, 2), dtype=np.int32)
    return Ligand(mass=np.array([mass]), charge=np.array([charge]), rstar=np.array([rstar]),
                  eps=np.array([eps]), bonds=z2, bond_k=np.zeros(0), bond_r0=np.zeros(0),
                  angles=np.zeros((0, 3), dtype=np.int32), angle_k=np.zeros(0),
                  angle_theta0=np.zeros(0), torsions=np.zeros((0, 4), dtype=np.int32),
                  torsion_V=np.zeros((0, 3)), torsion_gamma=np.zeros((0, 3)),
                  x0=np.zeros((1, 3)))


def make_receptor(n_atoms: int, site, seed: int, pocket_radius: float = 7.0,
                  density: float = 0.06, surface_z: float = 2.0) -> Receptor:
    """Receptor atoms at protein density in a half-ball below a surface, with a pocket.

    Atoms sit on a jittered cubic lattice of density ``density`` atoms/A^3 (nearest separation
    about 1.9 A), inside the ball around ``site`` whose radius makes exactly ``n_atoms`` fit,
    below the plane z = site_z + surface_z, and outside a pocket sphere of ``pocket_radius``
    centred on ``site``.  The pocket therefore opens to the solvent above the surface.
    LJ parameters and charges are drawn like the ligand's (charges shifted to net zero).
    """
    rng = np.random.default_rng(np.random.SeedSequence([0x2EC, seed]))
    site = np.asarray(site, dtype=np.float64)
    a = density ** (-1.0 / 3.0)
    # half-ball volume minus the pocket's lower half, with margin; trim to n_atoms afterwards
    R = ((n_atoms / density) / (2.0 / 3.0 * np.pi) + pocket_radius ** 3) ** (1.0 / 3.0) + 2.0 * a
    m = int(np.ceil(R / a)) + 1
    ax = np.arange(-m, m + 1) * a
    g = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    g = g + rng.uniform(-0.3, 0.3, size=g.shape)
    r = np.linalg.norm(g, axis=1)
    keep = (g[:, 2] < surface_z) & (r > pocket_radius)
    g, r = g[keep], r[keep]
    order = np.argsort(r, kind="stable")
    xyz = g[order[:n_atoms]] + site
    if xyz.shape[0] < n_atoms:
        raise RuntimeError("receptor lattice too small")
    rstar = rng.uniform(1.5, 2.0, size=n_atoms)
    eps = rng.uniform(0.01, 0.2, size=n_atoms)
    charge = rng.normal(0.0, 0.3, size=n_atoms)
    charge -= charge.mean()
    return Receptor(xyz=xyz, rstar=rstar, eps=eps, charge=charge)


def cube_grid(center, spacing: float, n: int) -> GridSpec:
    center = np.asarray(center, dtype=np.float64)
    origin = center - 0.5 * spacing * (n - 1)
    return GridSpec(origin=origin, spacing=float(spacing), n=(int(n), int(n), int(n)))


def geometric_temperatures(K: int, T_low: float, T_high: float) -> np.ndarray:
    if K == 1:
        return np.array([T_low])
    return T_low * (T_high / T_low) ** (np.arange(K) / (K - 1))


def bc_ladder(K: int, T_target=300.0, T_high=600.0, dt_fs=2.0) -> Ladder:
    """Warming leg B -> C: no receptor grids, temperature geometric from T_target to T_high."""
    return Ladder(T=geometric_temperatures(K, T_target, T_high), alpha=np.full(K, np.nan),
                  dt_fs=np.full(K, float(dt_fs)))


def cd_ladder(K: int, T_target=300.0, T_high=600.0, dt_fs=2.0) -> Ladder:
    """Coupling leg C -> D: alpha uniform on [0, 1]; temperature follows the protocol's T(alpha)."""
    alpha = np.linspace(0.0, 1.0, K) if K > 1 else np.array([1.0])
    T = (T_target - T_high) * alpha + T_high
    return Ladder(T=T, alpha=alpha, dt_fs=np.full(K, float(dt_fs)))


def rotation_matrix(q):
    q = q / np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def place_ligand(lig: Ligand, receptor: Receptor, site, n_copies: int, seed: int,
                 d0: float = 6.0, n_tries: int = 64) -> np.ndarray:
    """Rigid copies of the start geometry with the centre of mass within ``d0`` of the site.

    For each copy, ``n_tries`` random orientations and offsets are drawn and the one farthest
    (by minimum atom-atom distance) from the receptor atoms is kept.  Pure geometry: no energy is
    evaluated.  Returns float32 [n_copies, n_atoms, 3].
    """
    rng = np.random.default_rng(np.random.SeedSequence([0x91A, seed]))
    site = np.asarray(site, dtype=np.float64)
    near = receptor.xyz[np.linalg.norm(receptor.xyz - site, axis=1) < d0 + 20.0]
    out = np.empty((n_copies, lig.n_atoms, 3), dtype=np.float32)
    for c in range(n_copies):
        best, best_d = None, -1.0
        for _ in range(n_tries):
            Rm = rotation_matrix(rng.normal(size=4))
            off = _random_unit(rng) * d0 * rng.uniform(0, 1) ** (1.0 / 3.0)
            if off[2] < 0:
                off[2] = -off[2]
            x = lig.x0 @ Rm.T + site + off
            d = np.sqrt(((x[:, None, :] - near[None, :, :]) ** 2).sum(-1)).min() if near.size else 99.0
            if d > best_d:
                best, best_d = x, d
        out[c] = best
    return out


def make_system(n_lig_atoms: int, n_rec_atoms: int, grid_n: int, spacing: float, seed: int,
                K_bc: int, K_cd: int, dt_fs: float = 2.0) -> System:
    site = np.zeros(3)
    lig = make_ligand(n_lig_atoms, seed)
    rec = make_receptor(n_rec_atoms, site, seed)
    grid = cube_grid(site, spacing, grid_n)
    return System(ligand=lig, receptor=rec, grid=grid, site=site,
                  legs=[bc_ladder(K_bc, dt_fs=dt_fs), cd_ladder(K_cd, dt_fs=dt_fs)])


def ligand_atoms_for_seed(seed: int, lo: int = 30, hi: int = 60) -> int:
    return int(np.random.default_rng(np.random.SeedSequence([0xA70, seed])).integers(lo, hi + 1))


def config_small(seed: int = 1) -> System:
    """20-atom ligand, 1500-atom receptor, 33^3 grids at 0.5 A, 8 BC + 8 CD states, 2 fs."""
    return make_system(20, 1500, 33, 0.5, seed, K_bc=8, K_cd=8, dt_fs=2.0)


def config_paper_scale(seed: int = 2) -> System:
    """Paper-scale plain method: 30-60-atom ligand, 4000-atom receptor, 129^3 grids at 0.25 A,
    32 BC + 96 CD states, 2 fs."""
    return make_system(ligand_atoms_for_seed(seed), 4000, 129, 0.25, seed, K_bc=32, K_cd=96,
                       dt_fs=2.0)


def config_batch(seed: int = 3, n_ligands: int = 256, lo: int = 10, hi: int = 70):
    """Many ligands against one paper-scale grid set: n_ligands clash-free ligands of U[lo, hi]
    atoms, a 4000-atom receptor with an 11 A pocket (room for the largest), 129^3 grids at 0.25 A,
    16 BC + 48 CD states, 2 fs.  Returns (system without its own ligand, ligands)."""
    rng = np.random.default_rng(np.random.SeedSequence([0xBA7, seed]))
    sizes = rng.integers(lo, hi + 1, size=n_ligands)
    ligs = [make_ligand(int(n), seed=int(1000 * seed + i), min_sep=2.6) for i, n in enumerate(sizes)]
    site = np.zeros(3)
    rec = make_receptor(4000, site, seed, pocket_radius=11.0)
    sys_ = System(ligand=None, receptor=rec, grid=cube_grid(site, 0.25, 129), site=site,
                  legs=[bc_ladder(16, dt_fs=2.0), cd_ladder(48, dt_fs=2.0)])
    return sys_, ligs


def harmonic_oscillator_samples(K: int, N_per: int, seed: int, D: int = 1):
    """Exact samples of K harmonic wells u_k(x) = 0.5 beta_k k_k |x - mu_k|^2 in D dimensions.

    Returns (beta*k per state [K], mu [K, D], samples [K*N_per, D], N_k [K]).  Used to check a
    multistate estimator against closed-form free energies.
    """
    rng = np.random.default_rng(np.random.SeedSequence([0x4A2, seed]))
    bk = rng.uniform(0.5, 4.0, size=K)
    mu = rng.uniform(-1.0, 1.0, size=(K, D))
    xs = [mu[k] + rng.normal(size=(N_per, D)) / np.sqrt(bk[k]) for k in range(K)]
    return bk, mu, np.concatenate(xs, 0), np.full(K, N_per, dtype=np.int64)


def mlp_init(seed: int, n_feat: int = 64, n_hid: int = 256, n_out: int = 360, out_scale: float = 0.01):
    """Random initial weights of the proposal network (He-normal hidden layers, a small output
    layer, zero biases); row-major [out][in], float64."""
    rng = np.random.default_rng(np.random.SeedSequence([0x3E7, seed]))
    sizes = [(n_hid, n_feat), (n_hid, n_hid), (n_hid, n_hid), (n_out, n_hid)]
    p = {}
    for i, (o, n) in enumerate(sizes, 1):
        scale = np.sqrt(2.0 / n) if i < 4 else out_scale / np.sqrt(n)
        p["W%d" % i] = rng.normal(scale=scale, size=(o, n))
        p["b%d" % i] = np.zeros(o)
    return p
