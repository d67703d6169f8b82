"""Checkpoint and resume on the GPU: the paper stores each stage's data between cycles so that an
interrupted calculation restarts where it stopped ("Stages"; "Equilibration and production").
N cycles, a checkpoint, a fresh context that loads it, and M more cycles must repeat the
uninterrupted N + M cycles bit for bit: positions, components, state permutations, exchange and
trial counters, and every recorded snapshot.  The fresh context starts with other time steps, so
the test also shows that the checkpoint restores each state's time step."""
import numpy as np
import pytest

from paper_1507_03703_gb300 import synthetic as S

from systems import configurations, gpu_context, raw_grids32, state_table

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _run(ctx, legs, C, x0, seed):
    from paper_1507_03703_gb300.sampler import Leg, ReplicaExchange
    return ReplicaExchange(ctx, [Leg(l.K, o) for l, o in legs], C, x0, seed=seed, n_external=20)


def _state(run):
    out = {"x": run.x, "comps": run.comps, "state_of": run.state_of, "counters": run.counters,
           "history": torch.stack(run.history)}
    for li in range(len(run.legs)):
        out["config_of_%d" % li] = run.config_of[li]
        out["attempts_%d" % li] = run.attempts[li]
        out["accepts_%d" % li] = run.accepts[li]
    return out


def test_resume_repeats_the_uninterrupted_run_bit_for_bit(tmp_path):
    from paper_1507_03703_gb300.algdock import E_STATE, AlgdockError
    sys_ = S.config_small(1)
    g32 = raw_grids32(sys_)
    T, alpha, dt = state_table(sys_)
    bc, cd = sys_.legs
    legs = [(bc, 0), (cd, bc.K)]
    C, N, M, steps = 6, 7, 5, 15
    x0 = configurations(sys_, C * (bc.K + cd.K), seed=71)
    ref = _run(gpu_context(sys_, g32, T, alpha, dt), legs, C, x0, seed=9)
    for cyc in range(N + M):
        ref.cycle(cyc, steps, record=cyc >= 2)
    first = _run(gpu_context(sys_, g32, T, alpha, dt), legs, C, x0, seed=9)
    for cyc in range(N):
        first.cycle(cyc, steps, record=cyc >= 2)
    path = tmp_path / "run.ckpt"
    first.save(path, N)
    # a fresh context whose state table has other time steps, and a run built with another seed
    ctx = gpu_context(sys_, g32, T, alpha, np.full_like(dt, 0.5))
    resumed = _run(ctx, legs, C, configurations(sys_, C * (bc.K + cd.K), seed=72), seed=1234)
    nxt = resumed.load(path)
    assert nxt == N and resumed.seed == 9
    for cyc in range(nxt, N + M):
        resumed.cycle(cyc, steps, record=cyc >= 2)
    a, b = _state(ref), _state(resumed)
    for k in a:
        assert torch.equal(a[k], b[k]), k
    assert int(ref.counters[0].item()) > 0
    # a context holding another ligand refuses the checkpoint
    other = gpu_context(sys_, g32, T, alpha, dt, ligand=S.make_ligand(12, seed=5))
    with pytest.raises(AlgdockError) as ei:
        _run(other, legs, C, configurations(sys_, C * (bc.K + cd.K), seed=73, ligand=S.make_ligand(12, seed=5)),
             seed=9).load(path)
    assert ei.value.status == E_STATE
