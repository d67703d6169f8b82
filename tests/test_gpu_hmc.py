"""GPU parity of the fused HMC trial ("Sampling": velocity Verlet + Metropolis) against the FP64
oracle on the same seeded inputs and Philox streams.

- Zero steps: positions unchanged, dH = 0, every trial accepted.
- Accept decisions are bit-exact given the kernel's own energy change: each equals
  u < exp(-dH/kT) evaluated on the host in FP64 with the oracle's Philox uniform.
- Trajectories: FP32 dynamics against FP64 dynamics from the same start and momenta; after 10
  steps of 2 fs the positions agree to 1e-3 A and dH to 2e-3 kcal/mol + 1e-4 relative (the
  FP32 force error of ~1e-6 relative grows through the chaotic dynamics, measured margin >10x).
- Decisions agree with the oracle's wherever the oracle's log-acceptance margin exceeds the dH
  tolerance.
- Determinism and independence: identical calls give identical bits; splitting the replicas over
  two launches (rep_offset) changes nothing.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1507_03703_gb300 import synthetic as S

from systems import configurations, gpu_context, oracle_system, raw_grids32, state_table

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def small():
    sys_ = S.config_small(1)
    g32 = raw_grids32(sys_)
    T, alpha, dt = state_table(sys_)
    ctx = gpu_context(sys_, g32, T, alpha, dt)
    osys = oracle_system(sys_, g32, T, alpha, dt)
    return sys_, g32, T, alpha, dt, ctx, osys


def _run_gpu(ctx, x, states, n_steps, seed, cycle, rep_offset=0):
    R = x.shape[0]
    xd = torch.from_numpy(x.copy()).cuda()
    sd = torch.from_numpy(states.astype(np.int32)).cuda()
    comps = torch.empty((R, 4), dtype=torch.float64, device="cuda")
    dH = torch.empty(R, dtype=torch.float64, device="cuda")
    acc = torch.empty(R, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    ctx.hmc_cycle(sd, xd, comps, dH, acc, n_steps=n_steps, seed=seed, cycle=cycle, rep_offset=rep_offset,
                  counters=cnt)
    torch.cuda.synchronize()
    return xd.cpu().numpy(), comps.cpu().numpy(), dH.cpu().numpy(), acc.cpu().numpy(), cnt.cpu().numpy()


def _uniform(seed, rep, cycle):
    o = oracle.philox4x32_10([0, rep & 0xFFFFFFFF, cycle & 0xFFFFFFFF, 2], [seed & 0xFFFFFFFF, seed >> 32])
    return oracle.u53(int(o[0]), int(o[1]))


def test_zero_steps_is_identity(small):
    sys_, g32, T, alpha, dt, ctx, osys = small
    x = configurations(sys_, 40, seed=11)
    states = np.arange(40) % len(T)
    xn, comps, dH, acc, cnt = _run_gpu(ctx, x, states, 0, seed=5, cycle=0)
    assert np.array_equal(xn, x)
    assert np.all(dH == 0.0) and np.all(acc == 1) and cnt[0] == 40


def test_trajectories_and_accept_decisions_match_oracle(small):
    sys_, g32, T, alpha, dt, ctx, osys = small
    R = 160  # 10 replicas per state, 40 warps: several blocks and a ragged last block
    x = configurations(sys_, R, seed=12, jitter=0.1)
    states = np.arange(R) % len(T)
    seed, cycle = 0x1234ABCD5678, 7
    xg, cg, dHg, ag, cnt = _run_gpu(ctx, x, states, 10, seed, cycle)
    xo, co, dHo, ao, _ = osys.hmc(x.astype(np.float64), states, 10, seed, cycle)
    kT = oracle.KB * T[states]
    for r in range(R):
        u = _uniform(seed, r, cycle)
        assert bool(ag[r]) == (u < math.exp(-dHg[r] / kT[r])), r  # bit-exact given the kernel's dH
    tol_dH = 2e-3 + 1e-4 * np.abs(dHo)
    assert np.all(np.abs(dHg - dHo) <= tol_dH), np.max(np.abs(dHg - dHo) - tol_dH)
    margin = np.array([abs(math.log(max(_uniform(seed, r, cycle), 1e-300)) + dHo[r] / kT[r]) for r in range(R)])
    clear = margin > 2 * tol_dH / kT
    assert np.array_equal(ag[clear], ao[clear])
    both = (ag == 1) & (ao == 1)
    assert np.max(np.abs(xg[both] - xo[both])) < 1e-3
    rej = ag == 0
    assert np.array_equal(xg[rej], x[rej])
    assert cnt[0] == ag.sum()
    # the returned components are those of the returned configuration
    scale = np.maximum(np.abs(co), 1.0)
    assert np.all(np.abs(cg[both] - co[both]) <= 1e-4 * scale[both] + 1e-2)


def test_hmc_is_deterministic_and_replicas_independent(small):
    sys_, g32, T, alpha, dt, ctx, osys = small
    R = 96
    x = configurations(sys_, R, seed=13, jitter=0.1)
    states = (np.arange(R) * 7) % len(T)
    a = _run_gpu(ctx, x, states, 20, seed=99, cycle=3)
    b = _run_gpu(ctx, x, states, 20, seed=99, cycle=3)
    for u, v in zip(a[:4], b[:4]):
        assert np.array_equal(u, v)
    h1 = _run_gpu(ctx, x[:37], states[:37], 20, seed=99, cycle=3, rep_offset=0)
    h2 = _run_gpu(ctx, x[37:], states[37:], 20, seed=99, cycle=3, rep_offset=37)
    assert np.array_equal(np.concatenate([h1[0], h2[0]]), a[0])
    assert np.array_equal(np.concatenate([h1[2], h2[2]]), a[2])


def test_energy_error_scales_as_dt_squared():
    """Velocity Verlet's energy error at fixed trajectory length falls as dt^2: halving dt cuts
    the median |dH| about fourfold (a property of the integrator, independent of the oracle)."""
    sys_ = S.config_small(1)
    g32 = raw_grids32(sys_)
    T = np.full(3, 300.0)
    alpha = np.array([np.nan, np.nan, np.nan])
    dts = np.array([1.0, 0.5, 0.25])
    ctx = gpu_context(sys_, g32, T, alpha, dts)
    R = 512
    x = configurations(sys_, R, seed=14, jitter=0.02)
    med = []
    for k, dt in enumerate(dts):
        n = int(round(20.0 / dt))
        _, _, dH, _, _ = _run_gpu(ctx, x, np.full(R, k), n, seed=1, cycle=0)
        med.append(np.median(np.abs(dH)))
    r1, r2 = med[0] / med[1], med[1] / med[2]
    assert 2.5 < r1 < 6.0 and 2.5 < r2 < 6.0, med
