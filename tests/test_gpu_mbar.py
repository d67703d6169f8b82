"""GPU parity of MBAR ("Estimation"; Shirts & Chodera 2008) on identical u_kn: FP64 mode within
1e-8 kT of the oracle with the same iteration count (+-1: the stopping test compares a change
near the tolerance); the FP32-exponential mode within 2e-6 kT (each exponential carries ~2 ulp of
FP32 error, i.e. ~2.4e-7 relative per term, which moves f by at most a few times that)."""
import numpy as np
import pytest

import oracle
from paper_1507_03703_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _ukn(K, Nper, seed, D=2):
    bk, mu, x, N_k = S.harmonic_oscillator_samples(K, Nper, seed=seed, D=D)
    u = 0.5 * bk[:, None] * ((x[None, :, :] - mu[:, None, :]) ** 2).sum(-1)
    return u, N_k


@pytest.fixture(scope="module")
def ctx():
    from paper_1507_03703_gb300.algdock import Context
    return Context(0)


@pytest.mark.parametrize("K,Nper", [(2, 3000), (7, 1537), (24, 800)])
def test_mbar_fp64_matches_oracle(ctx, K, Nper):
    u, N_k = _ukn(K, Nper, seed=K)
    f_o, it_o = oracle.mbar(u, N_k, tol=1e-10)
    f, it = ctx.mbar(torch.from_numpy(u).cuda(), N_k, tol=1e-10, max_iter=10000)
    assert np.max(np.abs(f - f_o)) < 1e-8
    assert abs(it - it_o) <= 1


def test_mbar_fp32_exponentials(ctx):
    u, N_k = _ukn(6, 4000, seed=5)
    f_o, _ = oracle.mbar(u, N_k, tol=1e-10)
    f, it = ctx.mbar(torch.from_numpy(u).cuda(), N_k, tol=1e-9, max_iter=10000, precision_mode=1)
    assert np.max(np.abs(f - f_o)) < 2e-6


def test_mbar_fp32_compensated(ctx):
    """Precision mode 2: columns shifted by their minimum in FP64 (exact in the result), then FP32
    arguments, exponentials and Kahan-compensated sums.  The arguments carry FP32 rounding of
    values of a few kT (~1e-7 kT each), so f agrees with the FP64 oracle within 1e-6 kT."""
    u, N_k = _ukn(6, 4000, seed=6)
    f_o, _ = oracle.mbar(u, N_k, tol=1e-10)
    f, it = ctx.mbar(torch.from_numpy(u).cuda(), N_k, tol=1e-9, max_iter=10000, precision_mode=2)
    # measured: about 3e-8 kT; the bound is the 1e-6 kT stated for the FP32 modes
    assert np.max(np.abs(f - f_o)) < 1e-6


def test_mbar_unsampled_states_and_nonconvergence(ctx):
    from paper_1507_03703_gb300.algdock import AlgdockError, E_NOT_CONVERGED
    u, N_k = _ukn(5, 1000, seed=9)
    # move all samples of state 2 to state 1's count: state 2 becomes an unsampled target state
    N_k = N_k.copy()
    N_k[1] += N_k[2]
    N_k[2] = 0
    f_o, it_o = oracle.mbar(u, N_k, tol=1e-10)
    f, it = ctx.mbar(torch.from_numpy(u).cuda(), N_k, tol=1e-10)
    assert np.max(np.abs(f - f_o)) < 1e-8
    with pytest.raises(AlgdockError) as e:
        ctx.mbar(torch.from_numpy(u).cuda(), N_k, tol=1e-14, max_iter=3)
    assert e.value.status == E_NOT_CONVERGED
    f3, it3 = ctx.mbar(torch.from_numpy(u).cuda(), N_k, tol=1e-14, max_iter=3, raise_on_nonconvergence=False)
    f3_o, _ = oracle.mbar(u, N_k, tol=1e-14, max_iter=3)
    assert np.max(np.abs(f3 - f3_o)) < 1e-10


def test_mbar_identical_states(ctx):
    row = np.random.default_rng(1).normal(size=700)
    u = np.tile(row, (3, 1))
    f, it = ctx.mbar(torch.from_numpy(u).cuda(), np.array([200, 0, 500]), tol=1e-12)
    assert np.allclose(f, 0.0, atol=1e-12)


def test_mbar_precision_study_K256_N1e6(ctx, capsys):
    """MBAR at K = 256 states and N = 1e6 samples (harmonic wells in 2-D, exact samples built on
    the device): the FP64 mode against the closed form f_k = -ln(2 pi / (beta k_k)) (relative to
    state 0) within the statistical error, and the FP32-exponential mode against the FP64 mode.
    Prints the errors and the iteration rates (pytest -s)."""
    import time
    K, Nper, D = 256, 3907, 2
    g = torch.Generator(device="cuda").manual_seed(31)
    bk = torch.rand(K, device="cuda", dtype=torch.float64, generator=g) * 3.5 + 0.5
    mu = torch.rand((K, D), device="cuda", dtype=torch.float64, generator=g) * 0.6 - 0.3
    x = (mu[:, None, :] + torch.randn((K, Nper, D), device="cuda", dtype=torch.float64, generator=g)
         / torch.sqrt(bk)[:, None, None]).reshape(-1, D)
    N = x.shape[0]
    u = torch.empty((K, N), device="cuda", dtype=torch.float64)
    for k in range(K):
        u[k] = 0.5 * bk[k] * ((x - mu[k]) ** 2).sum(-1)
    N_k = np.full(K, Nper, dtype=np.int64)
    exact = -(D / 2) * np.log(2 * np.pi / bk.cpu().numpy())
    exact -= exact[0]
    t = time.perf_counter()
    f64, it64 = ctx.mbar(u, N_k, tol=1e-9, max_iter=20000, precision_mode=0)
    t64 = (time.perf_counter() - t) / it64
    t = time.perf_counter()
    f32, it32 = ctx.mbar(u, N_k, tol=1e-9, max_iter=20000, precision_mode=1)
    t32 = (time.perf_counter() - t) / it32
    ctx.mbar(u, N_k, tol=1e-9, max_iter=2, precision_mode=2, raise_on_nonconvergence=False)  # scratch
    t = time.perf_counter()
    fc, itc = ctx.mbar(u, N_k, tol=1e-9, max_iter=20000, precision_mode=2)
    tc = (time.perf_counter() - t) / itc
    err = np.abs(f64 - exact)
    d = np.abs(f32 - f64)
    dc = np.abs(fc - f64)
    with capsys.disabled():
        print("\nMBAR precision, K = %d, N = %d:" % (K, N))
        print("  FP64 mode vs closed form: max %.3f kT, rms %.3f kT (%d iterations, %.2f ms each)"
              % (err.max(), np.sqrt((err ** 2).mean()), it64, 1e3 * t64))
        print("  FP32 exponentials vs FP64: max %.2e kT (%d iterations, %.2f ms each)" % (d.max(), it32, 1e3 * t32))
        print("  FP32 compensated vs FP64: max %.2e kT (%d iterations, %.2f ms each, incl. the shift)"
              % (dc.max(), itc, 1e3 * tc))
    assert err.max() < 0.1
    assert d.max() < 1e-6   # measured 1.0e-8 kT
    assert dc.max() < 1e-6  # measured 3.0e-8 kT


def test_mbar_partials_match_the_oracle_and_a_sharded_solve_matches_one_process(ctx):
    """MBAR sharded over samples: the device's (max, sum) state pairs of one iteration equal the
    oracle's FP64 state sums of the same columns (1e-12 relative), and a solve whose samples sit in
    three uneven shards (launched one after another on this GPU, merged on the host by the library's
    update, as the ranks of a multi-GPU run do) equals the one-process device solve within 1e-10 kT."""
    from paper_1507_03703_gb300.algdock import mbar_update
    u, N_k = _ukn(8, 5000, seed=12)
    ud = torch.from_numpy(u).cuda()
    f = np.linspace(0.0, 1.5, 8)
    p_dev = ctx.mbar_partials(ud, N_k, f)
    p_ora = oracle.mbar_partials(u, N_k, f)
    assert np.max(np.abs(p_dev[:, 0] - p_ora[:, 0])) < 1e-12
    assert np.max(np.abs(p_dev[:, 1] / p_ora[:, 1] - 1)) < 1e-12
    cuts = [0, 7000, 7001, u.shape[1]]
    shards = [ud[:, a:b].contiguous() for a, b in zip(cuts, cuts[1:])]
    g, it = np.zeros(8), 0
    for it in range(1, 10001):
        g, d = mbar_update(np.stack([ctx.mbar_partials(s, N_k, g) for s in shards]), g)
        if d < 1e-12:
            break
    f_one, _ = ctx.mbar(ud, N_k, tol=1e-12)
    assert np.max(np.abs(g - f_one)) < 1e-10
    empty = ctx.mbar_partials(ud[:, :0], N_k, f)
    assert np.all(empty[:, 0] == -np.inf) and np.all(empty[:, 1] == 0)
