"""The all-FP64 GPU path (the precision study's FP64 arm) against the FP64 oracle, and the three
arms of the study side by side at paper scale (FP32 GPU path, FP64 GPU path, FP64 oracle).

Both FP64 sides evaluate the same energy function on the same FP64 lattices and parameters, in
another order of summation and with another maths library: components agree to 1e-10 relative
(+1e-9 kcal/mol) and forces to 1e-10 relative per configuration, at every state, with atoms
outside the lattice and at 1, 20, 33 and 96 atoms."""
import time

import numpy as np
import pytest

import oracle
from paper_1507_03703_gb300 import synthetic as S

from systems import configurations, state_table

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _arms(sys_, lig, T, alpha, dt, raw64, fp32=False):
    from paper_1507_03703_gb300.algdock import Context
    cap = oracle.soft_elec_cap(lig)
    ctx = Context(0)
    ctx.grids_load_f64(sys_.grid, *raw64, vmax_e=cap)
    if fp32:
        ctx.grids_load(sys_.grid, *[a.astype(np.float32) for a in raw64], vmax_e=cap)
    ctx.ligand_load(lig, sys_.site)
    ctx.states_set(T, alpha, dt)
    osys = oracle.OracleSystem(sys_.grid, *raw64, lig, T, alpha, dt, site=sys_.site, vmax_e=cap)
    return ctx, osys


def _check(ctx, osys, x, states):
    xd = torch.from_numpy(x).cuda()
    F = torch.empty(x.shape, dtype=torch.float64, device="cuda")
    c = ctx.energy_force_f64(xd, torch.from_numpy(states.astype(np.int32)).cuda(), force=F)
    c0 = ctx.energy_force_f64(xd)  # no states: components only
    c, c0, F = c.cpu().numpy(), c0.cpu().numpy(), F.cpu().numpy()
    w_sg, w_g, _ = osys.state_weights()
    # with and without forces the compiler may fuse multiply-adds differently: equal to rounding
    assert np.allclose(c, c0, rtol=1e-13, atol=1e-12)
    for n in range(x.shape[0]):
        k = states[n]
        co, Fo = osys.energy_force(x[n].astype(np.float64), w_sg[k], w_g[k])
        assert np.all(np.abs(c[n] - co) <= 1e-10 * np.abs(co) + 1e-9), (n, c[n], co)
        nF = np.linalg.norm(Fo)
        assert np.linalg.norm(F[n] - Fo) <= 1e-10 * max(nF, 1.0), (n, np.linalg.norm(F[n] - Fo) / nF)


@pytest.fixture(scope="module")
def small():
    sys_ = S.config_small(1)
    return sys_, oracle.grid_direct_sum(sys_.receptor, sys_.grid), state_table(sys_)


def test_fp64_path_matches_the_oracle(small):
    sys_, raw64, (T, alpha, dt) = small
    ctx, osys = _arms(sys_, sys_.ligand, T, alpha, dt, raw64)
    x = configurations(sys_, 48, seed=3, jitter=0.2)
    x[:3] += np.array([9.0, 0.0, 0.0], dtype=np.float32)  # partly outside the 16 A lattice
    _check(ctx, osys, x, np.arange(48) % len(T))


@pytest.mark.parametrize("n_atoms", [1, 33, 96])
def test_fp64_path_ligand_sizes(small, n_atoms):
    sys_, raw64, (T, alpha, dt) = small
    lig = S.one_atom_ligand() if n_atoms == 1 else S.make_ligand(n_atoms, seed=n_atoms, min_sep=2.6)
    ctx, osys = _arms(sys_, lig, T, alpha, dt, raw64)
    x = configurations(sys_, 16, seed=4, jitter=0.1, ligand=lig)
    _check(ctx, osys, x, np.arange(16) % len(T))


def test_precision_study_three_arms_paper_scale(capsys):
    """FP32 GPU path, FP64 GPU path and the FP64 oracle on the same paper-scale configurations
    (raw grids in FP64, rounded to FP32 for the FP32 path): per-quantity errors of the FP32 path
    against each FP64 arm, the FP64 arms' agreement, and the throughput of the two GPU paths."""
    sys_ = S.config_paper_scale(2)
    raw64 = oracle.grid_direct_sum(sys_.receptor, sys_.grid)
    T, alpha, dt = state_table(sys_)
    ctx, osys = _arms(sys_, sys_.ligand, T, alpha, dt, raw64, fp32=True)
    K = len(T)
    R = 64
    x = configurations(sys_, R, seed=16, jitter=0.1)
    states = ((np.arange(R) * 2) % K).astype(np.int32)
    xd, sd = torch.from_numpy(x).cuda(), torch.from_numpy(states).cuda()
    F32 = torch.empty_like(xd)
    c32 = torch.empty((R, 4), dtype=torch.float64, device="cuda")
    ctx.energy_force(sd, xd, F32, c32)
    F64 = torch.empty(x.shape, dtype=torch.float64, device="cuda")
    c64 = ctx.energy_force_f64(xd, sd, force=F64)
    F32, c32, F64, c64 = (t.cpu().numpy().astype(np.float64) for t in (F32, c32, F64, c64))
    w_sg, w_g, _ = osys.state_weights()
    f32_64, f64_o, cerr, cerr_o = [], [], [], []
    for n in range(R):
        co, Fo = osys.energy_force(x[n].astype(np.float64), w_sg[states[n]], w_g[states[n]])
        f32_64.append(np.linalg.norm(F32[n] - F64[n]) / np.linalg.norm(F64[n]))
        f64_o.append(np.linalg.norm(F64[n] - Fo) / np.linalg.norm(Fo))
        cerr.append(np.abs(c32[n] - c64[n]))
        cerr_o.append(np.abs(c64[n] - co))
    f32_64, f64_o, cerr, cerr_o = map(np.array, (f32_64, f64_o, cerr, cerr_o))
    # throughput of the two GPU paths on 8192 configurations
    Nt = 8192
    xt = torch.from_numpy(configurations(sys_, 256, seed=17, jitter=0.1)[np.arange(Nt) % 256]).cuda()
    st = torch.from_numpy((np.arange(Nt) % K).astype(np.int32)).cuda()
    Ft32 = torch.empty_like(xt)
    Ft64 = torch.empty(xt.shape, dtype=torch.float64, device="cuda")
    ct = torch.empty((Nt, 4), dtype=torch.float64, device="cuda")
    times = {}
    for name, fn in (("fp32", lambda: ctx.energy_force(st, xt, Ft32, ct)),
                     ("fp64", lambda: ctx.energy_force_f64(xt, st, force=Ft64, comps=ct))):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        times[name] = (time.perf_counter() - t0) / 3
    with capsys.disabled():
        print("\nprecision, three arms (paper scale, %d configurations):" % R)
        print("  force rel.: FP32 GPU vs FP64 GPU median %.2e max %.2e; FP64 GPU vs oracle max %.2e"
              % (np.median(f32_64), f32_64.max(), f64_o.max()))
        for i, name in enumerate(("U_L", "U_I", "Psi_sg", "Psi_g")):
            print("  %s (kcal/mol): FP32 GPU vs FP64 GPU median %.2e max %.2e; FP64 GPU vs oracle max %.2e"
                  % (name, np.median(cerr[:, i]), cerr[:, i].max(), cerr_o[:, i].max()))
        print("  evaluation of %d configurations (energies + forces): FP32 %.3f ms, FP64 %.3f ms (%.0fx)"
              % (Nt, 1e3 * times["fp32"], 1e3 * times["fp64"], times["fp64"] / times["fp32"]))
    assert f64_o.max() < 1e-10
    assert f32_64.max() < 1e-5
