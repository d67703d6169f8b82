"""GPU parity: receptor grids, energy components and forces against the FP64 oracle
("Thermodynamic Cycle"; Eq. (binding_site); Eq. (protocol)).

Tolerances (derived from the arithmetic):
- grids_build: terms in FP32 from FP64 differences, sums in FP64, so each node carries at most a
  few FP32 roundings of its largest terms: |err| <= 2e-6 * sum_j |term_j| (for LJr and LJa the
  terms share a sign, so this is 2e-6 relative).
- forces: 1e-5 relative per configuration, ||F_gpu - F_ref|| / ||F_ref|| (FP32 per term).
- energy components: FP32 per term, FP64 sums: 1e-5 relative of the component's scale plus
  1e-4 kcal/mol.
"""
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


def _abs_receptor(rec):
    return S.Receptor(xyz=rec.xyz, rstar=rec.rstar, eps=rec.eps, charge=np.abs(rec.charge))


def test_grids_build_matches_direct_sum(small):
    from paper_1507_03703_gb300.algdock import Context
    sys_ = small[0]
    ctx = Context(0)
    shape = tuple(reversed(sys_.grid.n))
    out = [torch.empty(shape, dtype=torch.float32, device="cuda") for _ in range(3)]
    ctx.grids_build(sys_.grid, sys_.receptor, *out)
    torch.cuda.synchronize()
    g = [o.cpu().numpy().astype(np.float64) for o in out]
    o_ljr, o_lja, o_elec = oracle.grid_direct_sum(sys_.receptor, sys_.grid)
    _, _, abs_elec = oracle.grid_direct_sum(_abs_receptor(sys_.receptor), sys_.grid)
    assert np.all(np.abs(g[0] - o_ljr) <= 2e-6 * o_ljr)
    assert np.all(np.abs(g[1] - o_lja) <= 2e-6 * np.abs(o_lja))
    assert np.all(np.abs(g[2] - o_elec) <= 2e-6 * abs_elec + 1e-30)


def test_grids_build_paper_scale_sampled_nodes():
    """129^3 lattice, 4000 receptor atoms: 4000 sampled nodes including the corners."""
    from paper_1507_03703_gb300.algdock import Context
    sys_ = S.config_paper_scale(2)
    ctx = Context(0)
    nx, ny, nz = sys_.grid.n
    out = [torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda") for _ in range(3)]
    ctx.grids_build(sys_.grid, sys_.receptor, *out)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    idx = rng.integers(0, [nx, ny, nz], size=(4000, 3))
    idx[:8] = [[i * (nx - 1), j * (ny - 1), k * (nz - 1)] for i in (0, 1) for j in (0, 1) for k in (0, 1)]
    pts = sys_.grid.origin + sys_.grid.spacing * idx
    o = oracle.grid_points(sys_.receptor, pts)
    a = oracle.grid_points(_abs_receptor(sys_.receptor), pts)
    gv = [out[c][idx[:, 2], idx[:, 1], idx[:, 0]].cpu().numpy().astype(np.float64) for c in range(3)]
    assert np.all(np.abs(gv[0] - o[0]) <= 2e-6 * o[0])
    assert np.all(np.abs(gv[1] - o[1]) <= 2e-6 * np.abs(o[1]))
    assert np.all(np.abs(gv[2] - o[2]) <= 2e-6 * a[2] + 1e-30)


def _check_forces(ctx, osys, x, states, w_sg, w_g):
    N = x.shape[0]
    xd = torch.from_numpy(x).cuda()
    sd = torch.from_numpy(states.astype(np.int32)).cuda()
    F = torch.empty_like(xd)
    comps = torch.empty((N, 4), dtype=torch.float64, device="cuda")
    ctx.energy_force(sd, xd, F, comps)
    torch.cuda.synchronize()
    F, comps = F.cpu().numpy().astype(np.float64), comps.cpu().numpy()
    worst = 0.0
    for n in range(N):
        k = states[n]
        c_o, F_o = osys.energy_force(x[n].astype(np.float64), w_sg[k], w_g[k])
        rel = np.linalg.norm(F[n] - F_o) / np.linalg.norm(F_o)
        worst = max(worst, rel)
        assert rel <= 1e-5, (n, k, rel)
        scale = np.maximum(np.abs(c_o), 1.0)
        assert np.all(np.abs(comps[n] - c_o) <= 1e-5 * scale + 1e-4), (n, comps[n], c_o)
    return worst


def test_forces_and_components_every_state_small(small):
    sys_, g32, T, alpha, dt, ctx, osys = small
    K = len(T)
    x = configurations(sys_, 8 * K, seed=3)
    states = np.arange(8 * K) % K
    w_sg, w_g, _ = osys.state_weights()
    _check_forces(ctx, osys, x, states, w_sg, w_g)


def test_forces_with_atoms_outside_the_lattice(small):
    sys_, g32, T, alpha, dt, ctx, osys = small
    x = configurations(sys_, 16, seed=4)
    x[:, :3, 0] += 9.0  # push a few atoms past the +x face (16 A cube, half-width 8 A)
    x[8:, 3:6, 2] -= 12.0
    states = np.full(16, len(T) - 1)
    w_sg, w_g, _ = osys.state_weights()
    _check_forces(ctx, osys, x, states, w_sg, w_g)


def test_reduced_energies_and_ukn(small):
    sys_, g32, T, alpha, dt, ctx, osys = small
    N = 300  # several warps per block and a ragged tail
    x = configurations(sys_, N, seed=5)
    xd = torch.from_numpy(x).cuda()
    comps = torch.empty((N, 4), dtype=torch.float64, device="cuda")
    u = torch.empty((len(T), N), dtype=torch.float64, device="cuda")
    ctx.reduced_energies(N, x=xd, comps=comps, k_begin=0, k_count=len(T), u_kn=u)
    torch.cuda.synchronize()
    u_o, c_o = osys.reduced_energies(x.astype(np.float64))
    c = comps.cpu().numpy()
    assert np.all(np.abs(c - c_o) <= 1e-5 * np.maximum(np.abs(c_o), 1.0) + 1e-4)
    # u_kn from the GPU's own components is exact FP64 arithmetic: compare with the oracle's
    # formula applied to the same components, bit for bit
    u_same = oracle.ukn_from_comps(T, alpha, c)
    assert np.array_equal(u.cpu().numpy(), u_same)
    # a sub-range of states, from stored components
    u2 = torch.empty((5, N), dtype=torch.float64, device="cuda")
    ctx.reduced_energies(N, comps=comps, k_begin=7, k_count=5, u_kn=u2)
    assert np.array_equal(u2.cpu().numpy(), u_same[7:12])


_RAW64 = {}


@pytest.fixture(scope="module")
def paper_scale():
    sys_ = S.config_paper_scale(2)
    raw64 = oracle.grid_direct_sum(sys_.receptor, sys_.grid)
    _RAW64["paper"] = raw64
    g32 = tuple(a.astype(np.float32) for a in raw64)
    T, alpha, dt = state_table(sys_)
    ctx = gpu_context(sys_, g32, T, alpha, dt)
    osys = oracle_system(sys_, g32, T, alpha, dt)
    return sys_, g32, T, alpha, dt, ctx, osys


def test_forces_paper_scale_sampled(paper_scale):
    """Paper-scale system (129^3 lattices, 30-60 atom ligand): sampled configurations at sampled
    states, including both legs and the alpha range where both grid sets are active."""
    sys_, g32, T, alpha, dt, ctx, osys = paper_scale
    K = len(T)
    x = configurations(sys_, 96, seed=6)
    states = np.random.default_rng(7).integers(0, K, size=96)
    states[:4] = [0, 31, 32 + 48, K - 1]
    w_sg, w_g, _ = osys.state_weights()
    _check_forces(ctx, osys, x, states, w_sg, w_g)


def test_precision_study_paper_scale(paper_scale, capsys):
    """The precision study of the FP32 path at paper scale (FP32 lattices, FP32 force terms, FP64
    sums and decisions) against the FP64 oracle on the same FP32 node values, per quantity: force
    relative error, each energy component in kcal/mol, and the energy change of 50-step HMC
    trials.  The measured figures are printed (pytest -s) and bounded here."""
    sys_, g32, T, alpha, dt, ctx, osys = paper_scale
    K = len(T)
    R = 64
    x = configurations(sys_, R, seed=16, jitter=0.1)
    states = (np.arange(R) * 2) % K
    w_sg, w_g, _ = osys.state_weights()
    xd = torch.from_numpy(x).cuda()
    sd = torch.from_numpy(states.astype(np.int32)).cuda()
    F = torch.empty_like(xd)
    comps = torch.empty((R, 4), dtype=torch.float64, device="cuda")
    ctx.energy_force(sd, xd, F, comps)
    dH = torch.empty(R, dtype=torch.float64, device="cuda")
    xh = xd.clone()
    ch = torch.empty_like(comps)
    ctx.hmc_cycle(sd, xh, ch, dH=dH, n_steps=50, seed=17, cycle=0)
    torch.cuda.synchronize()
    F, comps, dH = F.cpu().numpy().astype(np.float64), comps.cpu().numpy(), dH.cpu().numpy()
    _, _, dH_o, _, _ = osys.hmc(x.astype(np.float64), states, 50, 17, 0)
    frel, cerr, cref = [], [], []
    for n in range(R):
        k = states[n]
        c_o, F_o = osys.energy_force(x[n].astype(np.float64), w_sg[k], w_g[k])
        frel.append(np.linalg.norm(F[n] - F_o) / np.linalg.norm(F_o))
        cerr.append(np.abs(comps[n] - c_o))
        cref.append(np.abs(c_o))
    frel, cerr, cref = np.array(frel), np.array(cerr), np.array(cref)
    herr = np.abs(dH - dH_o)
    with capsys.disabled():
        print("\nprecision (FP32 path vs FP64 oracle, %d replicas, paper scale):" % R)
        print("  force rel. error: median %.2e, max %.2e" % (np.median(frel), frel.max()))
        for i, name in enumerate(("U_L", "U_I", "Psi_sg", "Psi_g")):
            print("  %s abs. error (kcal/mol): median %.2e, max %.2e" % (name, np.median(cerr[:, i]), cerr[:, i].max()))
        print("  dH of 50-step trials (kcal/mol): median %.2e, max %.2e" % (np.median(herr), herr.max()))
    assert frel.max() < 1e-5
    assert np.all(cerr <= 1e-5 * np.maximum(cref, 1.0) + 1e-4)
    # measured: median 4.6e-4, max 1.8e-3 kcal/mol.  FP32 and FP64 trajectories part slowly over 50
    # steps, so every trial's dH is bounded, not only the typical one.
    assert np.median(herr) < 2e-3
    assert herr.max() < 2e-2


def test_precision_study_bpmf_paper_scale(paper_scale, capsys):
    """The BPMF-level error of the FP32 path at paper scale.  Samples of the two end states of the
    cycle, B (300 K, no grids) and D (alpha = 1, 300 K), are drawn by the GPU HMC; each sample's
    energy is taken from the FP32 path (the sampler's own components, FP32 lattices) and from the
    FP64 oracle on FP64 lattices (the unrounded direct sums).  The FP64 BPMF differs from the FP32
    one by Delta B = Delta f_D - Delta f_B (both legs share milestone C), each Delta f a Zwanzig
    average over that end state's samples ("Estimation"), so the estimate covers the FP32
    arithmetic and the FP32 rounding of the lattices.  Bound: the BPMF tolerance of 0.05 kT."""
    sys_, g32, T, alpha, dt, ctx, osys = paper_scale
    osys64 = oracle.OracleSystem(sys_.grid, *_RAW64["paper"], sys_.ligand, T, alpha, dt, site=sys_.site)
    K = len(T)
    w_sg, w_g, beta = osys64.state_weights()
    ends = {"B": 0, "D": K - 1}
    R = 512
    x = configurations(sys_, 2 * R, seed=21, jitter=0.1)
    states = np.array([ends["B"]] * R + [ends["D"]] * R, dtype=np.int32)
    xd = torch.from_numpy(x).cuda()
    sd = torch.from_numpy(states).cuda()
    comps = torch.empty((2 * R, 4), dtype=torch.float64, device="cuda")
    xs, cs = [], []
    for cyc in range(30):
        ctx.hmc_cycle(sd, xd, comps, n_steps=50, seed=22, cycle=cyc)
        if cyc >= 24:
            xs.append(xd.cpu().numpy().copy())
            cs.append(comps.cpu().numpy().copy())
    res = {}
    for name, k in ends.items():
        sel = states == k
        du, dU = [], []
        for xx, cc in zip(xs, cs):
            for n in np.nonzero(sel)[0]:
                c64, _ = osys64.energy_force(xx[n].astype(np.float64), w_sg[k], w_g[k])
                u64 = c64[0] + c64[1] + w_sg[k] * c64[2] + w_g[k] * c64[3]
                u32 = cc[n, 0] + cc[n, 1] + w_sg[k] * cc[n, 2] + w_g[k] * cc[n, 3]
                dU.append(u64 - u32)
                du.append(beta[k] * (u64 - u32))
        r = oracle.fep(np.array(du))
        res[name] = (r, np.array(dU))
    dB = res["D"][0]["f"] - res["B"][0]["f"]
    sB = float(np.hypot(res["D"][0]["sigma"], res["B"][0]["sigma"]))
    with capsys.disabled():
        print("\nBPMF precision (FP32 path vs FP64 oracle on FP64 lattices, %d samples per end state):" % len(res["B"][1]))
        for name in ("B", "D"):
            r, dU = res[name]
            print("  %s: U64 - U32 mean %.2e, max |.| %.2e kcal/mol; Delta f %.2e kT" % (name, dU.mean(),
                                                                                  np.abs(dU).max(), r["f"]))
        print("  Delta BPMF (FP64 - FP32): %.2e +- %.1e kT" % (dB, sB))
    assert abs(dB) < 0.05


def test_exchange_bit_exact_on_paper_scale_components(paper_scale, capsys):
    """Replica exchange (Eq. (repXacc)) on components the energy path gives for paper-scale
    configurations: U_L of hundreds of kcal/mol and grid terms of tens, over the 32 warming and 96
    coupling states.  Each decision takes the FP32 shortcut only when the FP32 log-ratio is more
    than 1e-3 + 1e-6 sum|terms| from the log-uniform; at these magnitudes that band is wide, and
    the permutations and counts must still equal the oracle's FP64 decisions bit for bit."""
    sys_, g32, T, alpha, dt, ctx, osys = paper_scale
    K = len(T)
    Kbc = int(np.sum(np.isnan(alpha)))
    for (k0, Kl), L, seed in (((0, Kbc), 8, 41), ((Kbc, K - Kbc), 8, 42)):
        x = configurations(sys_, L * Kl, seed=seed, jitter=0.1)
        c = torch.empty((L * Kl, 4), dtype=torch.float64, device="cuda")
        ctx.reduced_energies(L * Kl, x=torch.from_numpy(x).cuda(), comps=c)
        comps = c.cpu().numpy().reshape(L, Kl, 4)
        with capsys.disabled():
            print("\nexchange on paper-scale components, states %d-%d: median |U_L| %.0f, |Psi_sg| %.1f, |Psi_g| %.1f"
                  % (k0, k0 + Kl - 1, *np.median(np.abs(comps[..., [0, 2, 3]]), axis=(0, 1))))
        assert np.median(np.abs(comps[..., 0])) > 100.0
        cfg0 = np.stack([np.random.default_rng(seed + l).permutation(Kl) for l in range(L)]).astype(np.int32)
        cfg_o, att_o, acc_o = oracle.exchange(T[k0:k0 + Kl], alpha[k0:k0 + Kl], comps, cfg0, 25, 5, 0xABCDEF, 3,
                                              ladder_offset=5)
        cfg = torch.from_numpy(cfg0.copy()).cuda()
        att = torch.zeros((5, Kl), dtype=torch.int64, device="cuda")
        acc = torch.zeros((5, Kl), dtype=torch.int64, device="cuda")
        ctx.exchange(Kl, k0, c.view(L, Kl, 4), cfg, None, n_sweeps=25, max_sep=5, seed=0xABCDEF, cycle=3,
                     ladder_offset=5, attempts=att, accepts=acc)
        assert np.array_equal(cfg.cpu().numpy(), cfg_o)
        assert np.array_equal(att.cpu().numpy(), att_o)
        assert np.array_equal(acc.cpu().numpy(), acc_o)
        assert acc_o.sum() > 0
