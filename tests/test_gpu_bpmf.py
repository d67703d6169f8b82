"""End-to-end BPMF on the GPU ("Estimation": beta_T B = f_BC,L + f'_CD from replica-exchange HMC
samples and MBAR), against the one-atom quadrature and against the FP64 oracle's own estimate.
Both are statistical comparisons: |difference| < max(0.05 kT, 4 standard errors), the error bar
from 8 disjoint groups of chains."""
import numpy as np
import pytest

import oracle
from paper_1507_03703_gb300 import synthetic as S

from systems import gpu_context, oracle_system, quadrature_bpmf, raw_grids32, uniform_in_sphere

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _gpu_bpmf(ctx, legs, C, x0, seed, n_cycles, n_steps, burn_in):
    from paper_1507_03703_gb300.sampler import Leg, ReplicaExchange, bpmf_kT
    run = ReplicaExchange(ctx, [Leg(l.K, o) for l, o in legs], C, x0, seed=seed)
    for cyc in range(n_cycles):
        run.cycle(cyc, n_steps, record=cyc >= burn_in)
    f_bc, _ = run.free_energies(0)
    f_cd, _ = run.free_energies(1)
    groups = []
    for g in range(8):
        ch = np.arange(g, C, 8)
        a, _ = run.free_energies(0, chains=ch)
        b, _ = run.free_energies(1, chains=ch)
        groups.append(bpmf_kT(a, b))
    return bpmf_kT(f_bc, f_cd), np.std(groups, ddof=1) / np.sqrt(8), run


def test_one_atom_bpmf_matches_quadrature():
    sys_ = S.config_small(1)
    lig = S.one_atom_ligand()
    g32 = raw_grids32(sys_)
    K, C, dt = 8, 64, 4.0
    bc, cd = S.bc_ladder(K, dt_fs=dt), S.cd_ladder(K, dt_fs=dt)
    T = np.concatenate([bc.T, cd.T])
    alpha = np.concatenate([bc.alpha, cd.alpha])
    ctx = gpu_context(sys_, g32, T, alpha, np.full(2 * K, dt), ligand=lig)
    rng = np.random.default_rng(5)
    x0 = uniform_in_sphere(rng, 2 * C * K, 6.0, sys_.grid.center).astype(np.float32)
    B, se, run = _gpu_bpmf(ctx, [(bc, 0), (cd, K)], C, x0, seed=21, n_cycles=400, n_steps=40, burn_in=50)
    target = quadrature_bpmf(sys_.grid, *[a.astype(np.float64) for a in g32], lig)
    print("one-atom BPMF gpu", B, "quadrature", target, "se", se)
    assert abs(B - target) < max(0.05, 4 * se), (B, target, se)
    assert int(run.counters[1].item()) == 0  # no non-finite trial


def test_one_atom_bpmf_with_learned_moves_matches_quadrature():
    """The same estimate with four learned proposals (random network) per replica and cycle at
    every state between HMC and exchange: the Metropolis-Hastings test keeps each state's
    distribution exact, so the BPMF still matches quadrature (bound 0.2 kT or 4 standard errors)."""
    from paper_1507_03703_gb300.learned import LearnedProposal
    from paper_1507_03703_gb300.sampler import Leg, ReplicaExchange, bpmf_kT
    sys_ = S.config_small(1)
    lig = S.one_atom_ligand()
    g32 = raw_grids32(sys_)
    K, C, dt = 8, 64, 4.0
    bc, cd = S.bc_ladder(K, dt_fs=dt), S.cd_ladder(K, dt_fs=dt)
    T = np.concatenate([bc.T, cd.T])
    alpha = np.concatenate([bc.alpha, cd.alpha])
    ctx = gpu_context(sys_, g32, T, alpha, np.full(2 * K, dt), ligand=lig)
    lp = LearnedProposal(ctx, seed=3)
    rng = np.random.default_rng(6)
    x0 = uniform_in_sphere(rng, 2 * C * K, 6.0, sys_.grid.center).astype(np.float32)
    run = ReplicaExchange(ctx, [Leg(K, 0), Leg(K, K)], C, x0, seed=31)
    acc = torch.zeros(run.R, dtype=torch.int32, device="cuda")
    for cyc in range(300):
        run.hmc(cyc, 40)
        lp.propose(run.state_of, run.x, run.comps, 4, seed=32, cycle=cyc, accepted=acc)
        run.exchange(cyc)
        if cyc >= 40:
            run.history.append(run.comps.clone())
    groups = []
    for g in range(8):
        ch = np.arange(g, C, 8)
        groups.append(bpmf_kT(run.free_energies(0, chains=ch)[0], run.free_energies(1, chains=ch)[0]))
    B = bpmf_kT(run.free_energies(0)[0], run.free_energies(1)[0])
    se = np.std(groups, ddof=1) / np.sqrt(8)
    target = quadrature_bpmf(sys_.grid, *[a.astype(np.float64) for a in g32], lig)
    rate = float(acc.sum().item()) / (run.R * 300 * 4)
    print("one-atom BPMF with learned moves", B, "quadrature", target, "se", se, "move acceptance", rate)
    assert 0.01 < rate < 0.999
    assert abs(B - target) < max(0.2, 4 * se), (B, target, se)


def test_small_ligand_bpmf_matches_oracle():
    """20-atom ligand, 8 + 8 states, 2 fs: the GPU estimate against the oracle's estimate from
    its own FP64 run with the same inputs and seeds."""
    sys_ = S.config_small(1)
    g32 = raw_grids32(sys_)
    bc, cd = sys_.legs
    K, C = bc.K, 32
    n_cycles, n_steps, burn = 300, 20, 50
    T = np.concatenate([bc.T, cd.T])
    alpha = np.concatenate([bc.alpha, cd.alpha])
    dt = np.concatenate([bc.dt_fs, cd.dt_fs])
    x0 = np.concatenate([S.place_ligand(sys_.ligand, sys_.receptor, sys_.site, C * K, seed=40 + i, n_tries=16)
                         for i in range(2)]).astype(np.float32)
    ctx = gpu_context(sys_, g32, T, alpha, dt)
    B, se, run = _gpu_bpmf(ctx, [(bc, 0), (cd, K)], C, x0, seed=33, n_cycles=n_cycles, n_steps=n_steps,
                           burn_in=burn)
    fo = []
    groups = np.zeros(8)
    for li, leg in enumerate([bc, cd]):
        osys = oracle_system(sys_, g32, leg.T, leg.alpha, leg.dt_fs)
        comps, st, _, _, _ = oracle.run_ladder(osys, x0[li * C * K:(li + 1) * C * K], C, n_cycles, n_steps, seed=33,
                                               rep_offset=li * C * K, ladder_offset=li * C, burn_in=burn)
        f, _ = oracle.ladder_free_energies(leg.T, leg.alpha, comps, st)
        fo.append(f)
        chain = np.tile(np.repeat(np.arange(C), K), comps.shape[0] // (C * K))
        for g in range(8):
            m = (chain % 8) == g
            fg, _ = oracle.ladder_free_energies(leg.T, leg.alpha, comps[m], st[m])
            groups[g] += fg[-1] - fg[0]
    Bo = oracle.bpmf_kT(fo[0], fo[1])
    se_o = np.std(groups, ddof=1) / np.sqrt(8)
    tol = max(0.05, 4 * np.hypot(se, se_o))
    print("20-atom BPMF gpu", B, "+-", se, "oracle", Bo, "+-", se_o)
    assert abs(B - Bo) < tol, (B, Bo, se, se_o)
