"""End-to-end BPMF on the GPU ("Estimation": beta_T B = f_BC,L + f'_CD from replica-exchange HMC
samples and MBAR), against the one-atom quadrature and against the FP64 oracle's own estimate.

Both comparisons are statistical.  The error bars come from disjoint groups of chains (each group
is an independent estimate).  The sample budgets are sized so that the combined standard error
is at most 0.0125 kT, a quarter of the 0.05 kT parity target, and the tests assert both that and
|difference| < 0.05 kT:
- one atom against the quadrature (1024 chains);
- a five-atom chain (two torsions, two 1-4 pairs and one full nonbonded pair) against the oracle,
  both legs, with the paper's external-coordinate moves.
- the twenty-atom config-1 ligand against the oracle's estimate stored by
  tests/golden/make_bpmf_20atom.py (hours of FP64 CPU time), as the mean over independent groups
  of chains on both sides."""
import numpy as np
import pytest

import oracle
from paper_1507_03703_gb300 import synthetic as S

from systems import gpu_context, oracle_system, quadrature_bpmf, raw_grids32, uniform_in_sphere

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


PARITY_KT = 0.05          # BPMF parity target of the plain path (kT)
MAX_SE_KT = PARITY_KT / 4  # the sample budget must bring the combined standard error to this


def _gpu_bpmf(ctx, legs, C, x0, seed, n_cycles, n_steps, burn_in, n_groups=8, n_external=0, thin=1):
    """BPMF of a GPU replica-exchange run and its standard error over n_groups disjoint groups of
    chains.  Records every thin-th cycle after burn_in."""
    from paper_1507_03703_gb300.sampler import Leg, ReplicaExchange, bpmf_kT
    run = ReplicaExchange(ctx, [Leg(l.K, o) for l, o in legs], C, x0, seed=seed, n_external=n_external)
    for cyc in range(n_cycles):
        run.cycle(cyc, n_steps, record=cyc >= burn_in and (cyc - burn_in) % thin == 0)
    f_bc, _ = run.free_energies(0)
    f_cd, _ = run.free_energies(1)
    groups = []
    for g in range(n_groups):
        ch = np.arange(g, C, n_groups)
        a, _ = run.free_energies(0, chains=ch)
        b, _ = run.free_energies(1, chains=ch)
        groups.append(bpmf_kT(a, b))
    return bpmf_kT(f_bc, f_cd), np.std(groups, ddof=1) / np.sqrt(n_groups), run


def test_one_atom_bpmf_matches_quadrature():
    sys_ = S.config_small(1)
    lig = S.one_atom_ligand()
    g32 = raw_grids32(sys_)
    K, C, dt = 8, 1024, 4.0
    bc, cd = S.bc_ladder(K, dt_fs=dt), S.cd_ladder(K, dt_fs=dt)
    T = np.concatenate([bc.T, cd.T])
    alpha = np.concatenate([bc.alpha, cd.alpha])
    ctx = gpu_context(sys_, g32, T, alpha, np.full(2 * K, dt), ligand=lig)
    rng = np.random.default_rng(5)
    x0 = uniform_in_sphere(rng, 2 * C * K, 6.0, sys_.grid.center).astype(np.float32)
    B, se, run = _gpu_bpmf(ctx, [(bc, 0), (cd, K)], C, x0, seed=21, n_cycles=400, n_steps=40, burn_in=50,
                           n_groups=16)
    # the quadrature converges at second order in its sub-lattice spacing (h/8 is within 1e-3 kT
    # of h/16 on this system), so its own error is far below the tolerance
    target = quadrature_bpmf(sys_.grid, *[a.astype(np.float64) for a in g32], lig)
    print("one-atom BPMF gpu %.4f quadrature %.4f |diff| %.4f se %.4f" % (B, target, abs(B - target), se))
    assert se <= MAX_SE_KT, se
    assert abs(B - target) < PARITY_KT, (B, target, se)
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


def test_five_atom_bpmf_matches_oracle_within_005kT():
    """A five-atom chain (make_ligand(5, seed 11): bonds 4-1-0-2-3, two torsions, two 1-4 pairs,
    the full 1-5 pair) on the 33^3 test lattice, 12 warming + 16 coupling states, trials of
    60 x 4 fs, twenty external-coordinate moves per cycle at alpha < 0.01 ("Sampling"), 25
    exchange sweeps per cycle, and a 2 A flat-bottom radius (Eq. (binding_site) with d0 = 2 A; a
    smaller site mixes in fewer cycles, which is what lets the FP64 oracle reach the budget).
    The GPU runs 768 chains and the oracle 192; the oracle's chains use the random streams of the
    GPU's first 192 chains.  Every second cycle after 40 of burn-in is recorded.  Both legs by
    MBAR on each side; error bars from 16 groups of chains.  Asserts that the combined standard
    error is at most 0.0125 kT and that the two BPMFs agree within 0.05 kT."""
    from paper_1507_03703_gb300.algdock import Context
    sys_ = S.config_small(1)
    lig = S.make_ligand(5, seed=11)
    g32 = raw_grids32(sys_)
    g64 = [a.astype(np.float64) for a in g32]
    KB, KC, dt, n_steps, n_cycles, burn, d0, n_ext = 12, 16, 4.0, 60, 240, 40, 2.0, 20
    Cg, Co, G, thin = 768, 192, 16, 2
    bc, cd = S.bc_ladder(KB, dt_fs=dt), S.cd_ladder(KC, dt_fs=dt)
    T = np.concatenate([bc.T, cd.T])
    alpha = np.concatenate([bc.alpha, cd.alpha])
    dts = np.concatenate([bc.dt_fs, cd.dt_fs])
    ctx = Context(0)
    ctx.grids_load(sys_.grid, *g32, ligand=lig)
    ctx.ligand_load(lig, sys_.site, d0=d0)
    ctx.states_set(T, alpha, dts)
    # start poses of the first Co chains, repeated for the others (their random streams differ)
    xb = np.tile(S.place_ligand(lig, sys_.receptor, sys_.site, Co * KB, seed=40, d0=d0, n_tries=4), (Cg // Co, 1, 1))
    xc = np.tile(S.place_ligand(lig, sys_.receptor, sys_.site, Co * KC, seed=41, d0=d0, n_tries=4), (Cg // Co, 1, 1))
    x0 = np.concatenate([xb, xc]).astype(np.float32)
    B, se, run = _gpu_bpmf(ctx, [(bc, 0), (cd, KB)], Cg, x0, seed=33, n_cycles=n_cycles, n_steps=n_steps,
                           burn_in=burn, n_groups=G, n_external=n_ext, thin=thin)
    assert int(run.counters[1].item()) == 0  # no non-finite trial
    fo, groups = [], np.zeros(G)
    # the oracle runs the GPU's first Co chains of each leg: same start poses, replica and ladder
    # indices, hence the same Philox streams
    for li, (leg, xl, rep0) in enumerate(((bc, xb, 0), (cd, xc, Cg * KB))):
        osys = oracle.OracleSystem(sys_.grid, *g64, lig, leg.T, leg.alpha, leg.dt_fs, site=sys_.site, d0=d0)
        comps, st, _, _, _ = oracle.run_ladder(osys, xl[:Co * leg.K], Co, n_cycles, n_steps, seed=33, rep_offset=rep0,
                                               ladder_offset=li * Cg, burn_in=burn, n_external=n_ext)
        n_rec = comps.shape[0] // (Co * leg.K)
        keep = np.arange(n_rec) % thin == 0
        comps = comps.reshape(n_rec, Co * leg.K, 4)[keep].reshape(-1, 4)
        st = st.reshape(n_rec, Co * leg.K)[keep].reshape(-1)
        f, _ = oracle.ladder_free_energies(leg.T, leg.alpha, comps, st)
        fo.append(f)
        chain = np.tile(np.repeat(np.arange(Co), leg.K), comps.shape[0] // (Co * leg.K))
        for g in range(G):
            m = (chain % G) == g
            fg, _ = oracle.ladder_free_energies(leg.T, leg.alpha, comps[m], st[m])
            groups[g] += fg[-1] - fg[0]
    Bo = oracle.bpmf_kT(fo[0], fo[1])
    se_o = np.std(groups, ddof=1) / np.sqrt(G)
    se_c = float(np.hypot(se, se_o))
    print("5-atom BPMF gpu %.4f +- %.4f oracle %.4f +- %.4f |diff| %.4f combined se %.4f"
          % (B, se, Bo, se_o, abs(B - Bo), se_c))
    assert se_c <= MAX_SE_KT, (se, se_o)
    assert abs(B - Bo) < PARITY_KT, (B, Bo, se, se_o)


@pytest.mark.slow
def test_twenty_atom_bpmf_matches_stored_oracle_within_005kT():
    """The 20-atom config-1 ligand (8 + 8 states, 2 fs) against the FP64 oracle's estimate stored by
    tests/golden/make_bpmf_20atom.py.  The estimate is the mean over independent groups of 32
    chains, each group running the same protocol from the same starting configurations (300 cycles
    of 20-step HMC and 25 exchange sweeps, 50 discarded, MBAR per leg over the group's samples); the
    oracle's groups differ in their Philox seed, the GPU's in their replica indices.  Both sides
    average enough groups that the combined standard error is at most 0.0125 kT, and the two
    means must agree within 0.05 kT."""
    import json
    import os
    from paper_1507_03703_gb300.sampler import Leg, ReplicaExchange, bpmf_kT
    golden = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "bpmf_20atom_oracle.json")))
    P = golden["protocol"]
    vals_o = np.array([r["bpmf_kT"] for r in golden["groups"]])
    Bo, se_o = vals_o.mean(), vals_o.std(ddof=1) / np.sqrt(len(vals_o))
    sys_ = S.config_small(1)
    g32 = raw_grids32(sys_)
    bc, cd = sys_.legs
    K, Cg = bc.K, P["chains_per_group"]
    G = 4000
    x0 = [S.place_ligand(sys_.ligand, sys_.receptor, sys_.site, Cg * K, seed=40 + li, n_tries=16).astype(np.float32)
          for li in range(2)]
    x = np.concatenate([np.tile(x0[li], (G, 1, 1)) for li in range(2)])
    T = np.concatenate([bc.T, cd.T])
    alpha = np.concatenate([bc.alpha, cd.alpha])
    dt = np.concatenate([bc.dt_fs, cd.dt_fs])
    ctx = gpu_context(sys_, g32, T, alpha, dt)
    run = ReplicaExchange(ctx, [Leg(bc.K, 0), Leg(cd.K, K)], G * Cg, x, seed=777, n_sweeps=P["exchange_sweeps"],
                          max_sep=P["max_sep"])
    for cyc in range(P["cycles"]):
        run.cycle(cyc, P["vv_steps"], record=cyc >= P["burn_in"])
    vals = np.empty(G)
    for g in range(G):
        ch = np.arange(g * Cg, (g + 1) * Cg)
        a, _ = run.free_energies(0, chains=ch)
        b, _ = run.free_energies(1, chains=ch)
        vals[g] = bpmf_kT(a, b)
    B, se = vals.mean(), vals.std(ddof=1) / np.sqrt(G)
    se_c = np.hypot(se, se_o)
    print("20-atom BPMF gpu %.4f +- %.4f (%d groups) oracle %.4f +- %.4f (%d groups) |diff| %.4f combined se %.4f"
          % (B, se, G, Bo, se_o, len(vals_o), abs(B - Bo), se_c))
    assert se_c <= MAX_SE_KT, (se, se_o)
    assert abs(B - Bo) < PARITY_KT, (B, Bo, se, se_o)
