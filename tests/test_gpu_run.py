"""The context's own run ("Equilibration and production"): replicas held by the context
(algdock_replicas_init), cycles with the context's seed and params (algdock_run), copy-out,
checkpoint and resume of those replicas (algdock_replicas_save / load), the device-side checks of
a cycle's results (params.checks), the external-coordinate moves inside algdock_cycle ("Sampling"),
and MBAR's defaults from the params.  Each composed path must repeat, bit for bit, the same cycles
made of algdock_cycle on caller-owned arrays or of the separate calls."""
import numpy as np
import pytest

from paper_1507_03703_gb300 import synthetic as S

from systems import configurations, raw_grids32, state_table

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def small():
    sys_ = S.config_small(1)
    return sys_, raw_grids32(sys_), state_table(sys_)


def _ctx(small, seed=0, **params):
    from paper_1507_03703_gb300.algdock import Context
    sys_, g32, (T, alpha, dt) = small
    ctx = Context(0, seed=seed, **params)
    ctx.grids_load(sys_.grid, *g32, ligand=sys_.ligand)
    ctx.ligand_load(sys_.ligand, sys_.site)
    ctx.states_set(T, alpha, dt)
    bc, cd = sys_.legs
    return ctx, [(bc.K, 0), (cd.K, bc.K)]


def _identity(legs, C):
    st = np.concatenate([np.tile(off + np.arange(K), C) for K, off in legs]).astype(np.int32)
    cfg = np.concatenate([np.tile(np.arange(K), C) for K, _ in legs]).astype(np.int32)
    return st, cfg


def _get(ctx, R, na):
    out = {"x": np.zeros((R, na, 3), np.float32), "comps": np.zeros((R, 4)), "state_of": np.zeros(R, np.int32),
           "config_of": np.zeros(R, np.int32), "counters": np.zeros(4, np.int64)}
    ctx.replicas_get(**out)
    return out


def test_params_round_trip_and_validation(small):
    from paper_1507_03703_gb300.algdock import AlgdockError, E_INVALID, Context
    ctx, _ = _ctx(small, seed=123456789012345, n_steps=7, max_sep=3, checks=1)
    p = ctx.params()
    assert (p["seed"], p["n_steps"], p["n_sweeps"], p["max_sep"], p["checks"]) == (123456789012345, 7, 25, 3, 1)
    ctx.set_params(n_sweeps=4, n_external=20)
    p = ctx.params()
    assert (p["n_sweeps"], p["n_external"], p["n_steps"]) == (4, 20, 7)
    for bad in ({"max_sep": 0}, {"n_sweeps": 20000, "max_sep": 5}, {"sigma_ext": float("nan")},
                {"mbar_precision": 3}, {"mbar_tol": 0.0}):
        with pytest.raises(AlgdockError) as e:
            ctx.set_params(**bad)
        assert e.value.status == E_INVALID
        with pytest.raises(AlgdockError):
            Context(0, **bad)
    assert ctx.params()["n_sweeps"] == 4  # a rejected set changes nothing


def test_run_repeats_cycle_on_caller_arrays(small):
    sys_ = small[0]
    steps, sweeps, sep, seed, first, n_cyc, C = 12, 10, 3, 77, 3, 5, 4
    ctx, legs = _ctx(small, seed=seed, n_steps=steps, n_sweeps=sweeps, max_sep=sep)
    R = C * sum(K for K, _ in legs)
    na = sys_.ligand.n_atoms
    x0 = configurations(sys_, R, seed=5)
    x = torch.from_numpy(x0.copy()).cuda()
    comps = torch.empty((R, 4), dtype=torch.float64, device="cuda")
    ctx.reduced_energies(R, x=x, comps=comps)
    st0, cfg0 = _identity(legs, C)
    st, cfg = torch.from_numpy(st0).cuda(), torch.from_numpy(cfg0).cuda()
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    words = sum(K * K * C for K, _ in legs)
    u_ref = torch.zeros(n_cyc * words, dtype=torch.float64, device="cuda")
    for i in range(n_cyc):
        ctx.cycle(legs, C, first + i, x, comps, st, cfg, n_steps=steps, n_sweeps=sweeps, max_sep=sep, seed=seed,
                  counters=cnt, u_kn=u_ref[i * words:(i + 1) * words])
    ctx.replicas_init(legs, C, x0)  # host positions
    assert ctx.ukn_words() == words
    u = np.zeros(n_cyc * words)  # host snapshots
    ctx.run(n_cyc, first_cycle=first, u_kn=u)
    got = _get(ctx, R, na)
    torch.cuda.synchronize()
    assert np.array_equal(got["x"], x.cpu().numpy())
    assert np.array_equal(got["comps"], comps.cpu().numpy())
    assert np.array_equal(got["state_of"], st.cpu().numpy())
    assert np.array_equal(got["config_of"], cfg.cpu().numpy())
    assert np.array_equal(got["counters"], cnt.cpu().numpy())
    assert np.array_equal(u, u_ref.cpu().numpy())
    assert got["counters"][0] > 0 and not np.array_equal(got["config_of"], cfg0)


def test_replicas_resume_from_checkpoint_is_bit_identical(small, tmp_path):
    sys_ = small[0]
    C = 3
    a, legs = _ctx(small, seed=4242, n_steps=10, n_sweeps=6)
    R = C * sum(K for K, _ in legs)
    na = sys_.ligand.n_atoms
    x0 = torch.from_numpy(configurations(sys_, R, seed=9)).cuda()  # device positions
    a.replicas_init(legs, C, x0)
    a.run(3, first_cycle=0)
    path = tmp_path / "replicas.ckpt"
    a.replicas_save(path, 3)
    a.run(4, first_cycle=3)
    want = _get(a, R, na)
    b, _ = _ctx(small, seed=1, n_steps=10, n_sweeps=6)  # another seed: the checkpoint's is restored
    assert b.replicas_load(path) == 3
    assert b.params()["seed"] == 4242
    assert b.ukn_words() == a.ukn_words()
    b.run(4, first_cycle=3)
    got = _get(b, R, na)
    for k in want:
        assert np.array_equal(got[k], want[k]), k


def test_device_checks_flag_nonfinite_and_broken_permutations(small):
    from paper_1507_03703_gb300.algdock import AlgdockError, E_NUMERIC, E_STATE
    sys_ = small[0]
    C = 2
    ctx, legs = _ctx(small, seed=3, n_steps=5, n_sweeps=2, checks=1)
    R = C * sum(K for K, _ in legs)
    x0 = configurations(sys_, R, seed=13)
    bad = x0.copy()
    bad[5, 1, 2] = np.nan
    with pytest.raises(AlgdockError) as e:
        ctx.replicas_init(legs, C, bad)
    assert e.value.status == E_NUMERIC and "non-finite" in str(e.value)
    ctx.replicas_init(legs, C, x0)
    ctx.run(2)
    # a ladder whose config_of repeats a slot: the exchange leaves it as it is, the check reports it
    x = torch.from_numpy(x0.copy()).cuda()
    comps = torch.empty((R, 4), dtype=torch.float64, device="cuda")
    ctx.reduced_energies(R, x=x, comps=comps)
    st0, cfg0 = _identity(legs, C)
    cfg0[1] = cfg0[0]
    args = (legs, C, 0, x, comps, torch.from_numpy(st0).cuda(), torch.from_numpy(cfg0).cuda())
    with pytest.raises(AlgdockError) as e:
        ctx.cycle(*args, n_steps=5, n_sweeps=2)
    assert e.value.status == E_STATE and "permutation" in str(e.value)
    ctx.set_params(checks=0)
    ctx.cycle(*args, n_steps=5, n_sweeps=2)  # unchecked: no error
    # non-finite positions with the checks off: the run goes on; on again: the cycle reports them
    ctx.replicas_init(legs, C, bad)
    ctx.run(1)
    ctx.set_params(checks=1)
    with pytest.raises(AlgdockError) as e:
        ctx.run(1, first_cycle=1)
    assert e.value.status == E_NUMERIC


def test_cycle_external_moves_repeat_the_separate_calls(small):
    sys_ = small[0]
    C, steps, sweeps, sep, seed, n_ext = 3, 8, 5, 4, 99, 6
    ctx, legs = _ctx(small)
    R = C * sum(K for K, _ in legs)
    x0 = configurations(sys_, R, seed=21)
    st0, cfg0 = _identity(legs, C)
    runs = []
    for composed, moves in ((False, n_ext), (True, n_ext), (True, 0)):
        x = torch.from_numpy(x0.copy()).cuda()
        comps = torch.empty((R, 4), dtype=torch.float64, device="cuda")
        ctx.reduced_energies(R, x=x, comps=comps)
        st, cfg = torch.from_numpy(st0.copy()).cuda(), torch.from_numpy(cfg0.copy()).cuda()
        cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
        for cyc in range(4):
            if composed:
                ctx.cycle(legs, C, cyc, x, comps, st, cfg, n_steps=steps, n_sweeps=sweeps, max_sep=sep, seed=seed,
                          counters=cnt, n_external=moves)
                continue
            ctx.hmc_cycle(st, x, comps, n_steps=steps, seed=seed, cycle=cyc, counters=cnt)
            ctx.external_moves(st, x, comps, n_moves=moves, seed=seed, cycle=cyc, counters=cnt)
            base = 0
            for li, (K, off) in enumerate(legs):
                n = C * K
                ctx.exchange(K, off, comps[base:base + n], cfg[base:base + n], st[base:base + n], n_sweeps=sweeps,
                             max_sep=sep, seed=seed, cycle=cyc, ladder_offset=li * C)
                base += n
        torch.cuda.synchronize()
        runs.append([t.cpu().numpy() for t in (x, comps, st, cfg, cnt)])
    for a, b in zip(runs[0], runs[1]):
        assert np.array_equal(a, b)
    # the moves took part: the same cycles without them end elsewhere
    assert not np.array_equal(runs[1][0], runs[2][0])


def test_mbar_takes_the_context_defaults(small):
    ctx, _ = _ctx(small, mbar_tol=1e-9, mbar_max_iter=500, mbar_precision=1)
    rng = np.random.default_rng(4)
    K, n = 5, 300
    mu = np.linspace(0, 2, K)
    xs = np.concatenate([rng.normal(m, 1.0, n) for m in mu])
    u = torch.from_numpy(0.5 * (xs[None, :] - mu[:, None]) ** 2).cuda()
    Nk = np.full(K, n)
    f_def, it_def = ctx.mbar(u, Nk, tol=0.0, max_iter=0, precision_mode=-1)
    f_exp, it_exp = ctx.mbar(u, Nk, tol=1e-9, max_iter=500, precision_mode=1)
    assert it_def == it_exp and np.array_equal(f_def, f_exp)
