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


def test_gpu_state_insertion_between_cycles():
    """Between cycles ("Equilibration and production"): a ladder with wide gaps (warming 300 and
    600 K; coupling alpha 0, 0.5, 1) runs 3 cycles; every neighbour pair whose exchange acceptance
    fell below 0.4 gets a state at the midpoint (the oracle's rule on the same counts), the old
    states keep their configurations bit for bit, and each new state's configurations are the
    importance-resampled draws (the oracle's indices) from its lower neighbour's configurations
    pooled over the chains.  The rebuilt run then cycles on."""
    from paper_1507_03703_gb300.sampler import Leg, ReplicaExchange
    sys_ = S.config_small(1)
    g32 = raw_grids32(sys_)
    T = np.array([300.0, 600.0, 600.0, 450.0, 300.0])
    A = np.array([np.nan, np.nan, 0.0, 0.5, 1.0])
    D = np.full(5, 2.0)
    ctx = gpu_context(sys_, g32, T, A, D)
    C = 32
    legs = [Leg(2, 0), Leg(3, 2)]
    run = ReplicaExchange(ctx, legs, C, configurations(sys_, C * 5, seed=9, jitter=0.1), seed=5)
    for cyc in range(3):
        run.cycle(cyc, 20)
    na = sys_.ligand.n_atoms
    att = [run.attempts[li][0].cpu().numpy()[:l.K - 1] for li, l in enumerate(legs)]
    acc = [run.accepts[li][0].cpu().numpy()[:l.K - 1] for li, l in enumerate(legs)]
    by_state = []
    for li, leg in enumerate(legs):
        sl = run.leg_slice(li)
        cfg = run.config_of[li].view(C, leg.K).long().cpu().numpy()
        rows = (np.arange(C)[:, None] * leg.K + cfg).reshape(-1)
        by_state.append((run.x[sl].cpu().numpy()[rows].reshape(C, leg.K, na, 3),
                         run.comps[sl].cpu().numpy()[rows].reshape(C, leg.K, 4)))
    nT, nA, nD, ins = run.insert_states(T, A, D, seed=13, counter=0)
    off_old, off_new = 0, 0
    for li, leg in enumerate(legs):
        sl = slice(off_old, off_old + leg.K)
        oT, oA, oD, o_ins = oracle.split_ladder(T[sl], A[sl], D[sl], att[li], acc[li])
        assert ins[li] == o_ins
        K2 = oT.size
        assert np.allclose(nT[off_new:off_new + K2], oT, rtol=1e-15) and np.array_equal(nD[off_new:off_new + K2], oD)
        xk, ck = by_state[li]
        new_leg = run.legs[li]
        assert new_leg.K == K2 and new_leg.state_offset == off_new
        x2 = run.x[run.leg_slice(li)].cpu().numpy().reshape(C, K2, na, 3)
        c2 = run.comps[run.leg_slice(li)].cpu().numpy().reshape(C, K2, 4)
        old_pos = [k for k in range(K2) if k not in o_ins]
        assert np.array_equal(x2[:, old_pos], xk) and np.array_equal(c2[:, old_pos], ck)
        for j, n in enumerate(o_ins):
            lower = old_pos.index(n - 1)
            pool_c = ck[:, lower]
            u = oracle.ukn_from_comps(nT, nA, pool_c)
            idx = oracle.resample(u[off_new + n - 1] - u[off_new + n], C, 13, 1000 * li + j)
            assert np.array_equal(x2[:, n], xk[idx, lower]) and np.array_equal(c2[:, n], pool_c[idx])
        off_old += leg.K
        off_new += K2
    assert sum(len(i) for i in ins) >= 2  # the wide gaps exchange rarely
    assert run.R == C * sum(l.K for l in run.legs) and run.history == []
    for cyc in range(3, 5):
        run.cycle(cyc, 20)
    torch.cuda.synchronize()
    assert all(np.all(np.isfinite(run.acceptance(li)[~np.isnan(run.acceptance(li))])) for li in range(2))
