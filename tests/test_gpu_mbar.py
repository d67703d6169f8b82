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
