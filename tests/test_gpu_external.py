"""GPU parity of the external-coordinate moves ("Sampling": a uniformly random rotation about the
centre of mass, a 0.6 A Gaussian translation, the Metropolis test, at states with alpha < 0.01)
against the FP64 oracle on the same seeded inputs and random streams.

- one move per replica: the accept decision agrees wherever the oracle's log-acceptance margin
  exceeds 1e-3 (the kernel's FP32 grid terms differ from FP64 by ~1e-6 relative); positions of
  moves both accept agree to 1e-4 A and their components to 1e-5 relative; rejected replicas and
  replicas at other states are unchanged bit for bit; U_L is carried over exactly;
- the random streams are indexed by the global replica (rep_offset): two halves equal the whole;
- GPU chains sample a harmonic well (3 kT/k) and a dipole in a uniform field (Langevin)."""
import math

import numpy as np
import pytest

import oracle
from paper_1507_03703_gb300 import synthetic as S

from systems import configurations, gpu_context, oracle_system, raw_grids32

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

T_ST = np.array([300.0, 300.0, 400.0, 350.0, 300.0])
A_ST = np.array([np.nan, 0.0, 0.003, 0.008, 0.5])  # moves at states 1..3 only
DT_ST = np.full(5, 2.0)


@pytest.fixture(scope="module")
def small():
    sys_ = S.config_small(1)
    g32 = raw_grids32(sys_)
    ctx = gpu_context(sys_, g32, T_ST, A_ST, DT_ST)
    osys = oracle_system(sys_, g32, T_ST, A_ST, DT_ST)
    return sys_, ctx, osys


def _start(sys_, osys, R, seed):
    x = configurations(sys_, R, seed=seed, jitter=0.05)
    comps = np.array([osys.energy_force(xi.astype(np.float64))[0] for xi in x])
    states = (np.arange(R) % len(T_ST)).astype(np.int32)
    return x, comps, states


def test_one_move_matches_the_oracle(small):
    sys_, ctx, osys = small
    R, seed, cycle = 200, 31, 4
    x, comps, states = _start(sys_, osys, R, 40)
    xd, cd = torch.from_numpy(x.copy()).cuda(), torch.from_numpy(comps.copy()).cuda()
    acc = torch.zeros(R, dtype=torch.int32, device="cuda")
    ctx.external_moves(torch.from_numpy(states).cuda(), xd, cd, 1, seed=seed, cycle=cycle, accepted=acc)
    torch.cuda.synchronize()
    xg, cg, ag = xd.cpu().numpy(), cd.cpu().numpy(), acc.cpu().numpy()
    xo, co, ao, lr = osys.external_moves(x.astype(np.float64), comps, states, 1, seed, cycle, logratio=True)
    moving = np.isin(states, [1, 2, 3])
    # replicas at other states: untouched
    assert np.array_equal(xg[~moving], x[~moving]) and np.array_equal(cg[~moving], comps[~moving])
    assert np.all(ag[~moving] == 0) and np.all(ao[~moving] == 0)
    u = np.array([oracle.u53(*[int(v) for v in oracle.philox4x32_10([2, r, cycle, 5],
                                                                     [seed & 0xFFFFFFFF, seed >> 32])[:2]])
                  for r in range(R)])
    margin = np.abs(lr - np.log(np.maximum(u, 1e-300)))
    clear = moving & (margin > 1e-3)
    assert clear.sum() > 0.9 * moving.sum()
    assert np.array_equal(ag[clear], ao[clear])
    both = moving & (ag == 1) & (ao == 1)
    rej = moving & (ag == 0)
    assert both.sum() > 10
    assert np.max(np.abs(xg[both] - xo[both])) < 1e-4
    assert np.array_equal(cg[both, 0], comps[both, 0])  # U_L carried over
    err = np.abs(cg[both, 1:] - co[both, 1:]) / np.maximum(np.abs(co[both, 1:]), 1.0)
    assert err.max() < 1e-5, err.max()
    assert np.array_equal(xg[rej], x[rej]) and np.array_equal(cg[rej], comps[rej])


def test_replica_offsets_index_the_streams(small):
    sys_, ctx, osys = small
    R = 64
    x, comps, states = _start(sys_, osys, R, 41)
    st = torch.from_numpy(states).cuda()
    xa, ca = torch.from_numpy(x.copy()).cuda(), torch.from_numpy(comps.copy()).cuda()
    ctx.external_moves(st, xa, ca, 20, seed=5, cycle=2)
    xb, cb = torch.from_numpy(x.copy()).cuda(), torch.from_numpy(comps.copy()).cuda()
    h = R // 2
    ctx.external_moves(st[:h], xb[:h], cb[:h], 20, seed=5, cycle=2)
    ctx.external_moves(st[h:], xb[h:], cb[h:], 20, seed=5, cycle=2, rep_offset=h)
    torch.cuda.synchronize()
    assert torch.equal(xa, xb) and torch.equal(ca, cb)
    assert not torch.equal(xa, torch.from_numpy(x).cuda())


def _flat_context(lig, elec, T, alpha, k=oracle.K_RESTRAINT, d0=oracle.D0):
    from paper_1507_03703_gb300.algdock import Context
    grid = S.cube_grid(np.zeros(3), 0.5, 33)
    zero = np.zeros((33, 33, 33), dtype=np.float32)
    ctx = Context(0)
    ctx.grids_load(grid, zero, zero, zero if elec is None else elec.astype(np.float32), ligand=lig)
    ctx.ligand_load(lig, np.zeros(3), k=k, d0=d0)
    ctx.states_set([T], [alpha], [2.0])
    return ctx


def test_gpu_chain_samples_a_harmonic_well():
    k = 5.0
    ctx = _flat_context(S.one_atom_ligand(charge=0.0), None, 300.0, 0.0, k=k, d0=0.0)
    R = 4096
    rng = np.random.default_rng(12)
    x = torch.from_numpy(rng.normal(scale=0.3, size=(R, 1, 3)).astype(np.float32)).cuda()
    comps = torch.empty((R, 4), dtype=torch.float64, device="cuda")
    ctx.reduced_energies(R, x=x, comps=comps)
    st = torch.zeros(R, dtype=torch.int32, device="cuda")
    vals = []
    for cyc in range(60):
        ctx.external_moves(st, x, comps, 5, seed=13, cycle=cyc)
        if cyc >= 10:
            vals.append((x[:, 0, :].double() ** 2).sum(-1).cpu().numpy())
    per = np.array(vals).mean(0)
    exact = 3 * oracle.KB * 300.0 / k
    assert abs(per.mean() - exact) < 4 * per.std(ddof=1) / math.sqrt(R), (per.mean(), exact)


def test_gpu_dipole_in_a_uniform_field_follows_the_langevin_function():
    q, bond, E0, T = 0.5, 1.5, 1.2, 300.0
    lig = S.Ligand(mass=np.array([12.0, 12.0]), charge=np.array([q, -q]), rstar=np.array([1.8, 1.8]),
                   eps=np.array([0.1, 0.1]), bonds=np.array([[0, 1]], dtype=np.int32), bond_k=np.array([400.0]),
                   bond_r0=np.array([bond]), angles=np.zeros((0, 3), dtype=np.int32), angle_k=np.zeros(0),
                   angle_theta0=np.zeros(0), torsions=np.zeros((0, 4), dtype=np.int32),
                   torsion_V=np.zeros((0, 3)), torsion_gamma=np.zeros((0, 3)),
                   x0=np.array([[0.0, 0.0, 0.5 * bond], [0.0, 0.0, -0.5 * bond]]))
    ax = -8.0 + 0.5 * np.arange(33)
    elec = np.broadcast_to(-E0 * ax[:, None, None], (33, 33, 33)).copy()
    ctx = _flat_context(lig, elec, T, 1.0)  # alpha = 1: the hard grids only
    R = 4096
    x = torch.from_numpy(np.repeat(lig.x0[None], R, axis=0).astype(np.float32)).cuda()
    comps = torch.empty((R, 4), dtype=torch.float64, device="cuda")
    ctx.reduced_energies(R, x=x, comps=comps)
    st = torch.zeros(R, dtype=torch.int32, device="cuda")
    vals = []
    for cyc in range(40):
        ctx.external_moves(st, x, comps, 4, seed=14, cycle=cyc, alpha_max=1.5)
        if cyc >= 5:
            u = (x[:, 0] - x[:, 1]).double()
            vals.append((u[:, 2] / u.norm(dim=1)).cpu().numpy())
    per = np.array(vals).mean(0)
    a = q * bond * E0 / (oracle.KB * T)
    exact = 1.0 / math.tanh(a) - 1.0 / a
    assert abs(per.mean() - exact) < 4 * per.std(ddof=1) / math.sqrt(R), (per.mean(), exact)
