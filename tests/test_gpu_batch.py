"""GPU parity of multi-ligand batches: every replica of every ligand in one HMC launch per
atoms-per-lane class ("Sampling": velocity Verlet + Metropolis, as for one ligand).

- Against the FP64 oracle, ligand by ligand, with the tolerances of the one-ligand HMC test: dH to
  2e-3 kcal/mol + 1e-4 relative after 10 steps of 2 fs; decisions bit-exact given the kernel's dH,
  and equal to the oracle's wherever its log-acceptance margin exceeds the dH tolerance; positions
  of trials both accept to 1e-3 A; rejected replicas unchanged bit for bit.
- Against the one-ligand kernel: where both stage the per-pair table, or neither does, the batch
  gives the same bits (the replica's Philox counter is its global index in both; replicas per
  block do not enter a replica's arithmetic).
- The uniform layout (every replica in the 65-96-atom shape), the autotuned shapes and a captured
  CUDA graph give results that pass the same checks; graph replays equal eager launches bit for
  bit.
Ligands of 10, 20, 31, 33, 47, 64, 65 and 70 atoms cover the three classes and their edges; the
soft electrostatic cap is the batch's smallest (every ligand keeps |q_i| v_e <= sqrt(A_i) v_r)."""
import math

import numpy as np
import pytest

import oracle
from paper_1507_03703_gb300 import synthetic as S

from systems import raw_grids32, state_table

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SIZES = [10, 20, 31, 33, 47, 64, 65, 70]
STRIDE = 70


@pytest.fixture(scope="module")
def batch():
    """A receptor with an 11 A pocket in a 28 A lattice (0.5 A), 8 + 8 states, clash-free
    ligands: the largest ligands fit without steric blow-ups, so 10-step trials stay stable."""
    from paper_1507_03703_gb300.algdock import Context
    site = np.zeros(3)
    rec = S.make_receptor(2000, site, seed=3, pocket_radius=11.0)
    sys_ = S.System(ligand=None, receptor=rec, grid=S.cube_grid(site, 0.5, 57), site=site,
                    legs=[S.bc_ladder(8), S.cd_ladder(8)])
    g32 = raw_grids32(sys_)
    T, alpha, dt = state_table(sys_)
    ligs = [S.make_ligand(n, seed=100 + n, min_sep=2.6) for n in SIZES]
    cap = min(oracle.soft_elec_cap(l) for l in ligs)
    ctx = Context(0)
    ctx.grids_load(sys_.grid, *g32, vmax_e=cap)
    ctx.states_set(T, alpha, dt)
    ctx.batch_load(ligs, sys_.site)
    K = len(T)
    lig_of = np.repeat(np.arange(len(ligs)), K).astype(np.int32)
    ctx.batch_layout(lig_of, STRIDE)
    x = np.zeros((len(lig_of), STRIDE, 3), dtype=np.float32)
    for l, lig in enumerate(ligs):
        pos = S.place_ligand(lig, sys_.receptor, sys_.site, K, seed=200 + l, n_tries=16)
        pos = pos + np.random.default_rng(300 + l).normal(scale=0.1, size=pos.shape).astype(np.float32)
        x[l * K:(l + 1) * K, :lig.n_atoms] = pos
    states = np.tile(np.arange(K), len(ligs)).astype(np.int32)
    return sys_, g32, T, alpha, dt, ligs, cap, ctx, lig_of, x, states


def _run(ctx, x, states, n_steps, seed, cycle):
    R = x.shape[0]
    xd = torch.from_numpy(x.copy()).cuda()
    sd = torch.from_numpy(states).cuda()
    comps = torch.empty((R, 4), dtype=torch.float64, device="cuda")
    dH = torch.empty(R, dtype=torch.float64, device="cuda")
    acc = torch.empty(R, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    ctx.batch_hmc_cycle(sd, xd, comps, dH, acc, n_steps=n_steps, seed=seed, cycle=cycle, counters=cnt)
    torch.cuda.synchronize()
    return xd.cpu().numpy(), comps.cpu().numpy(), dH.cpu().numpy(), acc.cpu().numpy(), cnt.cpu().numpy()


def _uniform(seed, rep, cycle):
    o = oracle.philox4x32_10([0, rep & 0xFFFFFFFF, cycle & 0xFFFFFFFF, 2], [seed & 0xFFFFFFFF, seed >> 32])
    return oracle.u53(int(o[0]), int(o[1]))


def _check_against_oracle(b, out, seed, cycle, n_steps):
    sys_, g32, T, alpha, dt, ligs, cap, ctx, lig_of, x, states = b
    xg, cg, dHg, ag, cnt = out
    K = len(T)
    assert cnt[0] == ag.sum()
    for l, lig in enumerate(ligs):
        sl = slice(l * K, (l + 1) * K)
        na = lig.n_atoms
        osys = oracle.OracleSystem(sys_.grid, *[a.astype(np.float64) for a in g32], lig, T, alpha, dt,
                                   site=sys_.site, vmax_e=cap)
        xo, co, dHo, ao, _ = osys.hmc(x[sl, :na].astype(np.float64), states[sl], n_steps, seed, cycle,
                                      rep_offset=l * K)
        kT = oracle.KB * T[states[sl]]
        for j in range(K):
            u = _uniform(seed, l * K + j, cycle)
            assert bool(ag[sl][j]) == (u < math.exp(-dHg[sl][j] / kT[j])), (l, j)
        tol = 2e-3 + 1e-4 * np.abs(dHo)
        assert np.all(np.abs(dHg[sl] - dHo) <= tol), (na, np.max(np.abs(dHg[sl] - dHo) - tol))
        margin = np.array([abs(math.log(max(_uniform(seed, l * K + j, cycle), 1e-300)) + dHo[j] / kT[j])
                           for j in range(K)])
        clear = margin > 2 * tol / kT
        assert np.array_equal(ag[sl][clear], ao[clear]), na
        both = (ag[sl] == 1) & (ao == 1)
        if both.any():
            assert np.max(np.abs(xg[sl][both, :na] - xo[both])) < 1e-3, na
        rej = ag[sl] == 0
        assert np.array_equal(xg[sl][rej], x[sl][rej])
        # the padding beyond each ligand's atoms is never written
        assert np.array_equal(xg[sl][:, na:], x[sl][:, na:])


def test_batch_matches_the_oracle_per_ligand(batch):
    out = _run(batch[7], batch[9], batch[10], 10, seed=0xBA7C4, cycle=3)
    _check_against_oracle(batch, out, 0xBA7C4, 3, 10)


def test_batch_equals_the_one_ligand_kernel(batch):
    from paper_1507_03703_gb300.algdock import Context
    sys_, g32, T, alpha, dt, ligs, cap, ctx, lig_of, x, states = batch
    K = len(T)
    xg, cg, dHg, ag, _ = _run(ctx, x, states, 10, seed=77, cycle=5)
    one = Context(0)
    one.grids_load(sys_.grid, *g32, vmax_e=cap)
    one.states_set(T, alpha, dt)
    shapes = ctx.batch_shapes()
    compared = 0
    for l, lig in enumerate(ligs):
        one.ligand_load(lig, sys_.site)
        table = one.hmc_shape()[1]
        cls = 0 if lig.n_atoms <= 32 else (3 if lig.n_atoms > 64 else (1 if table else 2))
        if table != shapes[cls][1]:
            continue  # pair-table and pair-type kernels round differently (checked against the oracle)
        compared += 1
        sl = slice(l * K, (l + 1) * K)
        xd = torch.from_numpy(np.ascontiguousarray(x[sl, :lig.n_atoms])).cuda()
        c1 = torch.empty((K, 4), dtype=torch.float64, device="cuda")
        d1 = torch.empty(K, dtype=torch.float64, device="cuda")
        a1 = torch.empty(K, dtype=torch.uint8, device="cuda")
        one.hmc_cycle(torch.from_numpy(states[sl]).cuda(), xd, c1, d1, a1, n_steps=10, seed=77, cycle=5,
                      rep_offset=l * K)
        torch.cuda.synchronize()
        assert np.array_equal(xd.cpu().numpy(), xg[sl, :lig.n_atoms]), lig.n_atoms
        assert np.array_equal(d1.cpu().numpy(), dHg[sl]) and np.array_equal(a1.cpu().numpy(), ag[sl])
        assert np.array_equal(c1.cpu().numpy(), cg[sl])
    assert compared >= 6


def test_uniform_layout_and_tuned_shapes(batch):
    sys_, g32, T, alpha, dt, ligs, cap, ctx, lig_of, x, states = batch
    try:
        ctx.batch_layout(lig_of, STRIDE, uniform=True)
        out = _run(ctx, x, states, 10, seed=0xBA7C4, cycle=3)
        _check_against_oracle(batch, out, 0xBA7C4, 3, 10)
        ctx.batch_layout(lig_of, STRIDE)
        xd = torch.from_numpy(x).cuda()
        chosen, ms = ctx.batch_tune(torch.from_numpy(states).cuda(), xd, n_steps=10, n_timed=2)
        assert np.array_equal(xd.cpu().numpy(), x)  # the tuner works on a copy
        assert ms > 0
        for k, (wpb, table) in enumerate(chosen):
            assert wpb in (0, 4, 8, 16)
            assert not (k == 3 and table)
        assert chosen == ctx.batch_shapes()
        out = _run(ctx, x, states, 10, seed=0xBA7C4, cycle=3)
        _check_against_oracle(batch, out, 0xBA7C4, 3, 10)
    finally:
        ctx.batch_layout(lig_of, STRIDE)


def test_graph_replay_equals_eager_launches(batch):
    sys_, g32, T, alpha, dt, ligs, cap, ctx, lig_of, x, states = batch
    R = x.shape[0]
    eager = _run(ctx, x, states, 10, seed=5, cycle=9)
    xd = torch.from_numpy(x.copy()).cuda()
    sd = torch.from_numpy(states).cuda()
    comps = torch.empty((R, 4), dtype=torch.float64, device="cuda")
    dH = torch.empty(R, dtype=torch.float64, device="cuda")
    acc = torch.empty(R, dtype=torch.uint8, device="cuda")
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        ctx.set_stream(s)
        try:
            with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
                ctx.batch_hmc_cycle(sd, xd, comps, dH, acc, n_steps=10, seed=5, cycle=9)
        finally:
            ctx.set_stream(None)
    torch.cuda.current_stream().wait_stream(s)
    xd.copy_(torch.from_numpy(x))
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(xd.cpu().numpy(), eager[0])
    assert np.array_equal(dH.cpu().numpy(), eager[2]) and np.array_equal(acc.cpu().numpy(), eager[3])


def test_layout_errors(batch):
    from paper_1507_03703_gb300.algdock import AlgdockError
    sys_, g32, T, alpha, dt, ligs, cap, ctx, lig_of, x, states = batch
    with pytest.raises(AlgdockError):
        ctx.batch_layout(lig_of, 64)  # a 65- and a 70-atom ligand do not fit
    with pytest.raises(AlgdockError):
        ctx.batch_layout(np.array([0, len(ligs)], dtype=np.int32), STRIDE)
    ctx.batch_layout(lig_of, STRIDE)


def test_layout_counts_the_kernels_static_shared_memory():
    """The 33-64-atom ligands of the 256-ligand workload include one whose 16-replica table block
    asks for 16 bytes less dynamic shared memory than 227 KB; with the batch kernel's own static
    shared memory (its copy of the ligand layout) that is over the per-block limit.  That ligand
    joins the class of 8-replica table blocks, with the 63-64-atom ligands that exceed the limit
    outright, and the rest keep 16-replica blocks: the layout sets every launch attribute."""
    from paper_1507_03703_gb300.algdock import Context
    sys_, ligs = S.config_batch(3)
    mid = [l for l in ligs if 33 <= l.n_atoms <= 64]
    ctx = Context(0)
    ctx.batch_load(mid, sys_.site)
    lig_of = np.repeat(np.arange(len(mid)), 2).astype(np.int32)
    ctx.batch_layout(lig_of, 64)
    shapes = ctx.batch_shapes()
    assert shapes[1] == (16, True)
    assert shapes[2] == (8, True)
