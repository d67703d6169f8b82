"""Shared test fixtures: the same seeded inputs handed to the oracle and to the CUDA library."""
import numpy as np
from scipy.interpolate import RegularGridInterpolator

import oracle
from paper_1507_03703_gb300 import synthetic as S


def raw_grids32(system, n_threads=0):
    """Raw direct-sum grids from the oracle (FP64), rounded to the FP32 the library takes.  Both
    sides then interpolate the same node values."""
    ljr, lja, elec = oracle.grid_direct_sum(system.receptor, system.grid, n_threads=n_threads)
    return ljr.astype(np.float32), lja.astype(np.float32), elec.astype(np.float32)


def state_table(system):
    T = np.concatenate([leg.T for leg in system.legs])
    alpha = np.concatenate([leg.alpha for leg in system.legs])
    dt = np.concatenate([leg.dt_fs for leg in system.legs])
    return T, alpha, dt


def oracle_system(system, grids32, T, alpha, dt, ligand=None):
    g = [a.astype(np.float64) for a in grids32]
    return oracle.OracleSystem(system.grid, g[0], g[1], g[2], ligand or system.ligand, T, alpha, dt,
                               site=system.site)


def gpu_context(system, grids32, T, alpha, dt, ligand=None, device=0):
    from paper_1507_03703_gb300.algdock import Context
    lig = ligand or system.ligand
    ctx = Context(device)
    ctx.grids_load(system.grid, grids32[0], grids32[1], grids32[2], ligand=lig)
    ctx.ligand_load(lig, system.site)
    ctx.states_set(T, alpha, dt)
    return ctx


def configurations(system, n, seed, jitter=0.3, ligand=None):
    """n placements of the ligand in the binding site plus a small random distortion (float32)."""
    lig = ligand or system.ligand
    x = S.place_ligand(lig, system.receptor, system.site, n, seed=seed, n_tries=8)
    rng = np.random.default_rng(seed + 1000)
    return (x + rng.normal(scale=jitter, size=x.shape)).astype(np.float32)


def quadrature_bpmf(grid, ljr, lja, elec, lig, T=300.0, d0=6.0, k=oracle.K_RESTRAINT):
    """One-atom BPMF (kT) by quadrature: the numerator on a sub-lattice of the receptor grid with
    scipy's trilinear interpolator, the denominator in closed form."""
    b = oracle.beta(T)
    ax = tuple(grid.origin[d] + grid.spacing * np.arange(grid.n[d]) for d in range(3))
    rgi = lambda L: RegularGridInterpolator(ax, np.transpose(L, (2, 1, 0)), method="linear")
    root = np.minimum(ljr, 1e10) ** 0.25
    sA = np.sqrt(lig.eps[0] * (2 * lig.rstar[0]) ** 12)
    sB = np.sqrt(2 * lig.eps[0] * (2 * lig.rstar[0]) ** 6)
    q = lig.charge[0]
    hq = grid.spacing / 8
    R = d0 + 1.0
    s = np.arange(-R + hq / 2, R, hq)
    X, Y, Z = np.meshgrid(s, s, s, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    d = np.linalg.norm(P, axis=1)
    keep = d < R
    P, d = P[keep] + grid.center, d[keep]
    UI = np.where(d > d0, 0.5 * k * (d - d0) ** 2, 0.0)
    psi = sA * rgi(root)(P) ** 4 + sB * rgi(lja)(P) + q * rgi(elec)(P)
    num = np.sum(np.exp(-b * (psi + UI))) * hq ** 3
    a = b * k / 2
    den = 4 / 3 * np.pi * d0 ** 3 + 4 * np.pi * (d0 ** 2 * np.sqrt(np.pi) / (2 * np.sqrt(a)) + d0 / a
                                                + np.sqrt(np.pi) / (4 * a ** 1.5))
    return -np.log(num / den)


def uniform_in_sphere(rng, n, radius, center):
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    return (v * radius * rng.uniform(0, 1, size=(n, 1)) ** (1 / 3))[:, None, :] + center
