"""GPU parity of the end-point corrections against the FP64 oracle ("Thermodynamic Cycle": the
target force field computes the receptor-ligand interaction directly; "Estimation": f_AB and f_DE
by Zwanzig free energy perturbation of milestone samples).

Tolerances follow from the kernels' arithmetic:
- target interaction: each pair term is FP32 (relative error a few 1e-6 for r^-12: six times the
  error of r^2 and of the reciprocal) and a tile of 256 terms is summed in FP32 before the FP64
  sum (recursive-summation bound 255 u = 1.5e-5 of the tile's absolute sum).  So per
  configuration |gpu - oracle| <= 2e-5 M, M = the sum over atom pairs of |term|, computed here in
  numpy; the median error must also stay below 2e-6 M (no systematic drift).
- FEP: FP64 throughout, summed in another order: 1e-12 relative on f, n_eff and sigma; the
  smallest difference is exact.
- f_DE from sampled configurations: f moves by at most the largest change of any du, so the bound
  is beta times the largest per-configuration bound above."""
import math

import numpy as np
import pytest

import oracle
from paper_1507_03703_gb300 import synthetic as S

from systems import configurations, gpu_context, raw_grids32

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def magnitude(receptor, ligand, x):
    """Sum over ligand-receptor atom pairs of the absolute value of each interaction term."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, ligand.n_atoms, 3)
    sA_r = np.sqrt(receptor.eps * (2 * receptor.rstar) ** 12)
    sB_r = np.sqrt(2 * receptor.eps * (2 * receptor.rstar) ** 6)
    sA_l = np.sqrt(ligand.eps * (2 * ligand.rstar) ** 12)
    sB_l = np.sqrt(2 * ligand.eps * (2 * ligand.rstar) ** 6)
    out = np.zeros(x.shape[0])
    for s in range(x.shape[0]):
        r2 = ((x[s][:, None, :] - receptor.xyz[None]) ** 2).sum(-1)
        rr2, ra2 = np.maximum(r2, 1e-4), np.maximum(r2, 4.0)
        t = (np.abs(sA_l[:, None] * sA_r[None]) / rr2 ** 6 + np.abs(sB_l[:, None] * sB_r[None]) / ra2 ** 3
             + 332.0637 * np.abs(ligand.charge[:, None] * receptor.charge[None]) / (4 * ra2))
        out[s] = t.sum()
    return out


def _ctx(sys_, ligand=None, receptor=None):
    from paper_1507_03703_gb300.algdock import Context
    ctx = Context(0)
    ctx.ligand_load(ligand or sys_.ligand, sys_.site)
    ctx.receptor_load(receptor or sys_.receptor)
    return ctx


def _check_psi(receptor, ligand, x, got):
    want = oracle.target_interaction(receptor, ligand, x.astype(np.float64))
    M = magnitude(receptor, ligand, x)
    err = np.abs(got - want)
    assert np.all(err <= 2e-5 * M + 1e-9), (err / M).max()
    assert np.median(err / np.maximum(M, 1e-300)) < 2e-6
    return want


@pytest.fixture(scope="module")
def small():
    return S.config_small(1)


def test_target_interaction_matches_the_oracle(small):
    """20-atom ligand (25 configurations per block), 1500 receptor atoms (a ragged last tile),
    157 configurations (a ragged last block)."""
    sys_ = small
    ctx = _ctx(sys_)
    x = configurations(sys_, 157, seed=3, jitter=0.2)
    got = ctx.target_interaction(torch.from_numpy(x).cuda()).cpu().numpy()
    _check_psi(sys_.receptor, sys_.ligand, x, got)


@pytest.mark.parametrize("n_atoms,n_rec,N", [(1, 300, 1030), (96, 257, 11), (45, 1, 23), (33, 513, 1)])
def test_ligand_and_receptor_sizes(n_atoms, n_rec, N):
    """1 atom (512 configurations per block), 96 atoms (5 per block, 480 of 512 points), one
    receptor atom, a single configuration."""
    lig = S.make_ligand(n_atoms, seed=n_atoms)
    rec = S.make_receptor(max(n_rec, 200), np.zeros(3), seed=5)
    rec = S.Receptor(xyz=rec.xyz[:n_rec], rstar=rec.rstar[:n_rec], eps=rec.eps[:n_rec], charge=rec.charge[:n_rec])
    sys_ = S.System(ligand=lig, receptor=rec, grid=S.cube_grid(np.zeros(3), 0.5, 9), site=np.zeros(3), legs=[])
    ctx = _ctx(sys_)
    rng = np.random.default_rng(n_rec)
    x = (lig.x0[None] + rng.normal(scale=2.0, size=(N, 1, 3))).astype(np.float32)
    got = ctx.target_interaction(torch.from_numpy(x).cuda()).cpu().numpy()
    _check_psi(rec, lig, x, got)


def test_empty_inputs(small):
    sys_ = small
    ctx = _ctx(sys_)
    x = torch.empty((0, sys_.ligand.n_atoms, 3), dtype=torch.float32, device="cuda")
    assert ctx.target_interaction(x).numel() == 0
    empty = S.Receptor(xyz=np.zeros((0, 3)), rstar=np.zeros(0), eps=np.zeros(0), charge=np.zeros(0))
    ctx.receptor_load(empty)
    xs = torch.from_numpy(configurations(sys_, 9, seed=4)).cuda()
    assert torch.equal(ctx.target_interaction(xs), torch.zeros(9, dtype=torch.float64, device="cuda"))


def test_call_order_and_bad_arguments(small):
    from paper_1507_03703_gb300.algdock import AlgdockError, Context
    sys_ = small
    ctx = Context(0)
    ctx.ligand_load(sys_.ligand, sys_.site)
    x = torch.from_numpy(configurations(sys_, 3, seed=5)).cuda()
    with pytest.raises(AlgdockError):
        ctx.target_interaction(x)  # no receptor yet
    bad = S.Receptor(xyz=np.array([[0.0, np.nan, 0.0]]), rstar=np.ones(1), eps=np.ones(1), charge=np.ones(1))
    with pytest.raises(AlgdockError):
        ctx.receptor_load(bad)
    with pytest.raises(AlgdockError):
        ctx.fep(torch.empty(0, dtype=torch.float64, device="cuda"))


def test_target_interaction_at_paper_scale_sampled():
    """The bench's workload: 4000 receptor atoms, 16384 configurations in one launch; 48 sampled
    configurations against the oracle, and bitwise repeatability."""
    sys_ = S.config_paper_scale(2)
    ctx = _ctx(sys_)
    N = 16384
    base = configurations(sys_, 256, seed=6, jitter=0.2)
    x = base[np.arange(N) % 256] + np.random.default_rng(7).normal(scale=0.05, size=(N,) + base.shape[1:]).astype(
        np.float32)
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    got = ctx.target_interaction(xd)
    again = ctx.target_interaction(xd)
    assert torch.equal(got, again)
    pick = np.random.default_rng(8).choice(N, 48, replace=False)
    _check_psi(sys_.receptor, sys_.ligand, x[pick], got.cpu().numpy()[pick])


# ------------------------------------------------------------------ FEP
def _fep_close(g, o):
    assert g["du_min"] == o["du_min"]
    assert abs(g["f"] - o["f"]) <= 1e-12 * max(1.0, abs(o["f"]))
    assert abs(g["n_eff"] - o["n_eff"]) <= 1e-12 * o["n_eff"]
    if math.isnan(o["sigma"]):
        assert math.isnan(g["sigma"])
    else:
        assert abs(g["sigma"] - o["sigma"]) <= 1e-12 * max(o["sigma"], 1e-300) + 1e-15


@pytest.mark.parametrize("N", [1, 2, 255, 1000, 77_777, 1_000_003])
def test_fep_matches_the_oracle(small, N):
    ctx = _ctx(small)
    rng = np.random.default_rng(N)
    du = rng.normal(3.0, 2.0, size=N) + (rng.random(N) < 0.01) * rng.exponential(30.0, size=N)
    g = ctx.fep(torch.from_numpy(du).cuda())
    _fep_close(g, oracle.fep(du))


def test_fep_strided_columns_beta_and_weightless_samples(small):
    ctx = _ctx(small)
    rng = np.random.default_rng(9)
    N = 5003
    comps = rng.normal(-40.0, 5.0, size=(N, 4))
    psi_t = comps[:, 3] + rng.normal(0.3, 1.2, size=N)
    psi_t[::97] = np.inf  # weight 0
    beta = oracle.beta(300.0)
    cd = torch.from_numpy(comps).cuda()
    g = ctx.fep(torch.from_numpy(psi_t).cuda(), cd[:, 3], beta=beta)
    _fep_close(g, oracle.fep(beta * (psi_t - comps[:, 3])))
    g2 = ctx.fep(torch.from_numpy(psi_t).cuda(), cd[:, 3], beta=beta)
    assert g == g2  # fixed reduction order


def test_fep_rejects_nan(small):
    from paper_1507_03703_gb300.algdock import AlgdockError
    ctx = _ctx(small)
    du = np.zeros(100)
    du[17] = np.nan
    with pytest.raises(AlgdockError):
        ctx.fep(torch.from_numpy(du).cuda())


def test_f_de_from_sampled_milestone_d(small):
    """Configurations sampled at milestone D (alpha = 1, 300 K) by the GPU HMC; f_DE from the
    library against the oracle's target energies and the same Psi_g."""
    sys_ = small
    g32 = raw_grids32(sys_)
    T, alpha, dt = np.array([300.0]), np.array([1.0]), np.array([2.0])
    ctx = gpu_context(sys_, g32, T, alpha, dt)
    ctx.receptor_load(sys_.receptor)
    R = 512
    x = torch.from_numpy(configurations(sys_, R, seed=10, jitter=0.1)).cuda()
    st = torch.zeros(R, dtype=torch.int32, device="cuda")
    comps = torch.empty((R, 4), dtype=torch.float64, device="cuda")
    dH = torch.empty(R, dtype=torch.float64, device="cuda")
    acc = torch.empty(R, dtype=torch.uint8, device="cuda")
    for cyc in range(10):
        ctx.hmc_cycle(st, x, comps, dH, acc, n_steps=20, seed=11, cycle=cyc)
    psi_t = ctx.target_interaction(x)
    beta = oracle.beta(300.0)
    g = ctx.fep(psi_t, comps[:, 3], beta=beta)
    xh = x.cpu().numpy()
    want_t = _check_psi(sys_.receptor, sys_.ligand, xh, psi_t.cpu().numpy())
    psi_g = comps[:, 3].cpu().numpy()
    o = oracle.fep(beta * (want_t - psi_g))
    tol = beta * (2e-5 * magnitude(sys_.receptor, sys_.ligand, xh)).max()
    assert abs(g["f"] - o["f"]) <= tol + 1e-12, (g, o, tol)
    assert np.isfinite(g["f"]) and 1.0 <= g["n_eff"] <= R
