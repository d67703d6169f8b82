"""Edge cases of the C ABI on the GPU: error codes for bad arguments and call order, empty
inputs, and the ligand-size boundaries of the warp layout (1, 32, 33, 64, 65 and 96 atoms)."""
import math

import numpy as np
import pytest

import oracle
from paper_1507_03703_gb300 import synthetic as S

from systems import configurations, gpu_context, oracle_system, raw_grids32, state_table

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def base():
    sys_ = S.config_small(1)
    return sys_, raw_grids32(sys_), state_table(sys_)


def test_call_order_and_argument_errors(base):
    from paper_1507_03703_gb300 import algdock as A
    sys_, g32, (T, alpha, dt) = base
    ctx = A.Context(0)
    x = torch.zeros((4, sys_.ligand.n_atoms, 3), dtype=torch.float32, device="cuda")
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    comps = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(A.AlgdockError) as e:
        ctx.hmc_cycle(st, x, comps, n_steps=5)
    assert e.value.status == A.E_STATE
    ctx.grids_load(sys_.grid, *g32, ligand=sys_.ligand)
    ctx.ligand_load(sys_.ligand, sys_.site)
    ctx.states_set(T, alpha, dt)
    # a host array where a device pointer is required
    L = A.load_library()
    host = np.zeros(4 * sys_.ligand.n_atoms * 3, dtype=np.float32)
    r = L.algdock_hmc_cycle(ctx.h, 4, st.data_ptr(), host.ctypes.data, comps.data_ptr(), None, None, 5, 0, 0, 0, None)
    assert r == A.E_INVALID and "device" in ctx.last_error()
    # empty inputs are no-ops
    ctx.hmc_cycle(st[:0], x[:0], comps[:0], n_steps=5)
    ctx.reduced_energies(0, x=x[:0], comps=comps[:0])
    # bad exchange sizes
    cfg = torch.zeros((1, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(A.AlgdockError) as e:
        ctx.exchange(8, 0, torch.zeros((1, 8, 4), dtype=torch.float64, device="cuda"), cfg, max_sep=0)
    assert e.value.status == A.E_INVALID
    with pytest.raises(A.AlgdockError) as e:
        ctx.exchange(8, 12, torch.zeros((1, 8, 4), dtype=torch.float64, device="cuda"), cfg)
    assert e.value.status == A.E_INVALID  # states 12..19 are outside the 16-state table
    # MBAR: counts must sum to N
    with pytest.raises(A.AlgdockError) as e:
        ctx.mbar(torch.zeros((2, 10), dtype=torch.float64, device="cuda"), np.array([5, 4]))
    assert e.value.status == A.E_INVALID


def test_ligand_validation():
    from paper_1507_03703_gb300 import algdock as A
    ctx = A.Context(0)
    big = S.make_ligand(97, seed=1)
    with pytest.raises(A.AlgdockError) as e:
        ctx.ligand_load(big, np.zeros(3))
    assert e.value.status == A.E_INVALID
    lig = S.make_ligand(10, seed=2)
    lig.charge = lig.charge.copy()
    lig.charge[3] = math.nan
    with pytest.raises(A.AlgdockError) as e:
        ctx.ligand_load(lig, np.zeros(3))
    assert e.value.status == A.E_NUMERIC
    lig = S.make_ligand(10, seed=2)
    lig.bonds = lig.bonds.copy()
    lig.bonds[0, 1] = 10
    with pytest.raises(A.AlgdockError) as e:
        ctx.ligand_load(lig, np.zeros(3))
    assert e.value.status == A.E_INVALID


@pytest.mark.parametrize("n_atoms", [1, 32, 33, 64, 65, 96])
def test_forces_at_layout_boundaries(base, n_atoms):
    sys0, g32, (T, alpha, dt) = base
    lig = S.one_atom_ligand() if n_atoms == 1 else S.make_ligand(n_atoms, seed=n_atoms)
    sys_ = S.System(ligand=lig, receptor=sys0.receptor, grid=sys0.grid, site=sys0.site, legs=sys0.legs)
    ctx = gpu_context(sys_, g32, T, alpha, dt)
    osys = oracle_system(sys_, g32, T, alpha, dt)
    K = len(T)
    x = configurations(sys_, 2 * K, seed=n_atoms, jitter=0.2)
    states = np.arange(2 * K) % K
    xd = torch.from_numpy(x).cuda()
    F = torch.empty_like(xd)
    comps = torch.empty((2 * K, 4), dtype=torch.float64, device="cuda")
    ctx.energy_force(torch.from_numpy(states.astype(np.int32)).cuda(), xd, F, comps)
    torch.cuda.synchronize()
    F = F.cpu().numpy().astype(np.float64)
    w_sg, w_g, _ = osys.state_weights()
    for n in range(2 * K):
        c_o, F_o = osys.energy_force(x[n].astype(np.float64), w_sg[states[n]], w_g[states[n]])
        ref = np.linalg.norm(F_o)
        if ref == 0.0:  # e.g. one atom, no grid weight, inside the flat bottom: no force at all
            assert np.all(F[n] == 0.0)
        else:
            assert np.linalg.norm(F[n] - F_o) / ref <= 1e-5


def test_gather_probe_runs_and_keeps_its_sink(base):
    """The gather-roofline probe (not a step of the method): it needs loaded lattices, reads only,
    and leaves its sink untouched (the folded sum never takes the impossible value)."""
    from paper_1507_03703_gb300 import algdock as A
    sys_, g32, (T, alpha, dt) = base
    ctx = A.Context(0)
    sink = torch.zeros(1, dtype=torch.float32, device="cuda")
    with pytest.raises(A.AlgdockError) as e:
        ctx.gather_probe(1000, sink=sink)
    assert e.value.status == A.E_STATE
    ctx.grids_load(sys_.grid, *g32, ligand=sys_.ligand)
    for soft in (False, True):
        ctx.gather_probe(100_000, soft=soft, seed=3, sink=sink)
        ctx.gather_probe(0, soft=soft, sink=sink)
    torch.cuda.synchronize()
    assert sink.item() == 0.0
