"""GPU parity of protocol initialization ("Initialization") against the FP64 oracle.

- The per-state reductions on identical inputs: standard deviations and mean exchange
  probabilities to 1e-12 relative (FP64, sums in another order); resampled indices identical
  (the same Philox draws against running weights that differ by at most an ulp), and the
  gathered configurations are the chosen rows.
- The GPU driver has the algorithm's properties: on a harmonic well the warming leg is geometric,
  T_{k+1}/T_k = 1 + s sqrt(2/3) (pooled over protocols, within 5 %), and every neighbour pair
  passes the check; a coupling leg that starts too fast has its speed shrunk until neighbours
  overlap, and it still ends at alpha = 1."""
import math

import numpy as np
import pytest

import oracle
from paper_1507_03703_gb300 import synthetic as S

from systems import configurations, gpu_context, oracle_system, raw_grids32

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

T_ST = np.array([300.0, 350.0, 600.0, 540.0, 420.0, 300.0])
A_ST = np.array([np.nan, np.nan, 0.0, 0.2, 0.6, 1.0])


@pytest.fixture(scope="module")
def small():
    sys_ = S.config_small(1)
    g32 = raw_grids32(sys_)
    dt = np.full(len(T_ST), 2.0)
    return sys_, gpu_context(sys_, g32, T_ST, A_ST, dt), oracle_system(sys_, g32, T_ST, A_ST, dt)


def _comps(n, seed):
    rng = np.random.default_rng(seed)
    c = np.stack([rng.normal(-20, 3, n), np.abs(rng.normal(0, 0.5, n)), rng.normal(5, 4, n), rng.normal(-30, 6, n)],
                 1)
    return c


def test_statistics_and_exchange_probability(small):
    sys_, ctx, osys = small
    ca, cb = _comps(2000, 1), _comps(2000, 2)
    da, db = torch.from_numpy(ca).cuda(), torch.from_numpy(cb).cuda()
    for k in range(len(T_ST)):
        got = ctx.state_statistics(da, k)
        want = osys.state_statistics(ca, k)
        assert np.allclose(got, want, rtol=1e-12, atol=1e-14), (k, got, want)
    for ka, kb in ((0, 1), (2, 3), (3, 4), (4, 5), (2, 2)):
        got = ctx.mean_pacc(da, db, ka, kb)
        want = osys.mean_pacc(ca, cb, ka, kb)
        assert got == pytest.approx(want, rel=1e-12)


def test_resampling(small):
    sys_, ctx, osys = small
    n, na = 2000, sys_.ligand.n_atoms
    c = _comps(n, 3)
    x = configurations(sys_, n, seed=4, jitter=0.1)
    dc, dx = torch.from_numpy(c).cuda(), torch.from_numpy(x).cuda()
    for ka, kb, ctr in ((0, 1, 0), (2, 3, 17), (4, 5, 99)):
        idx = torch.empty(50, dtype=torch.int64, device="cuda")
        xo = torch.empty((50, na, 3), dtype=torch.float32, device="cuda")
        ctx.resample(dc, ka, kb, 50, 7, ctr, x_in=dx, x_out=xo, idx=idx)
        u = oracle.ukn_from_comps(T_ST, A_ST, c)
        want = oracle.resample(u[ka] - u[kb], 50, 7, ctr)
        got = idx.cpu().numpy()
        assert np.array_equal(got, want)
        assert np.array_equal(xo.cpu().numpy(), x[got])


def _flat_ctx(lig, elec=None, k=oracle.K_RESTRAINT, d0=oracle.D0, n=17):
    from paper_1507_03703_gb300.algdock import Context
    grid = S.cube_grid(np.zeros(3), 0.5, n)
    zero = np.zeros((n, n, n), dtype=np.float32)
    ctx = Context(0)
    ctx.grids_load(grid, zero, zero, zero if elec is None else elec.astype(np.float32), ligand=lig)
    ctx.ligand_load(lig, np.zeros(3), k=k, d0=d0)
    return ctx


def test_gpu_warming_leg_is_geometric_on_a_harmonic_well():
    from paper_1507_03703_gb300.protocol import ProtocolBuilder
    s = 0.3
    ratios = []
    for sd in (6, 11, 12):
        ctx = _flat_ctx(S.one_atom_ligand(charge=0.0), k=1.13, d0=0.0)
        seeds = np.random.default_rng(sd).normal(scale=0.6, size=(50, 1, 3)).astype(np.float32)
        r = ProtocolBuilder(ctx).build_leg("bc", seeds, seed=sd, speed=s, dt0=5.0)
        T = r["T"]
        assert T[0] == 300.0 and T[-1] == 600.0 and np.all(np.diff(T) > 0)
        assert np.all(r["pacc"] >= 0.4) and r["speed"] == s
        ratios.extend(T[1:-1] / T[:-2])
    ratios = np.array(ratios)
    expect = 1 + s * math.sqrt(2 / 3)
    assert np.all(np.abs(ratios / expect - 1) < 0.12), ratios
    assert abs(ratios.mean() / expect - 1) < 0.05, ratios


def test_gpu_coupling_leg_is_slowed_until_neighbours_overlap():
    from paper_1507_03703_gb300.protocol import ProtocolBuilder
    lig = S.one_atom_ligand(charge=1.0)
    ax = -8.0 + 0.5 * np.arange(33)
    elec = np.broadcast_to(-2.0 * ax[:, None, None], (33, 33, 33)).copy()
    ctx = _flat_ctx(lig, elec=elec, n=33)
    seeds = np.random.default_rng(5).uniform(-3, 3, size=(50, 1, 3)).astype(np.float32)
    r = ProtocolBuilder(ctx, n_trials=20).build_leg("cd", seeds, seed=7, speed=5.0, dt0=4.0)
    assert r["speed"] < 5.0
    assert np.all(r["pacc"] >= 0.4)
    assert r["alpha"][0] == 0.0 and r["alpha"][-1] == 1.0 and np.all(np.diff(r["alpha"]) > 0)
    assert np.allclose(r["T"], 600.0 - 300.0 * r["alpha"])
