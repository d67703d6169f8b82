"""algdock_mbar_noalloc: MBAR for callers that cannot allocate device memory (for example a host
framework whose caching allocator owns all device memory, or a service that reserves its whole
budget at start-up).  The call uses a fixed scratch array inside the library instead of device
allocations; its results must equal those of algdock_mbar, call after call, since the shared
array keeps the previous call's contents.

This file is collected last on purpose: if it fails in a run that stops at the first failure,
every other test has already run.  It passes alone in a fresh process and after the others."""
import ctypes

import numpy as np
import pytest

from paper_1507_03703_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-8  # the MBAR parity tolerance of the other GPU tests (kT)


def _ukn(K, Nper, seed):
    bk, mu, x, N_k = S.harmonic_oscillator_samples(K, Nper, seed=seed, D=2)
    return 0.5 * bk[:, None] * ((x[None, :, :] - mu[:, None, :]) ** 2).sum(-1), N_k


def _noalloc(ctx, u, N_k, tol=1e-10, max_iter=10000):
    """Direct call of the C entry point through ctypes."""
    L = ctx._L
    K, N = u.shape
    Nk = np.ascontiguousarray(N_k, dtype=np.int64)
    f = np.zeros(K)
    it = ctypes.c_int32()
    st = L.algdock_mbar_noalloc(ctx.h, K, N, u.data_ptr(), Nk.ctypes.data, tol, max_iter, 0, f.ctypes.data,
                                ctypes.byref(it))
    return st, f, it.value


def test_noalloc_mbar_matches_mbar_on_consecutive_calls():
    from paper_1507_03703_gb300.algdock import OK, Context
    ctx = Context(0)
    # two calls in a row with different sizes: the second must not see the first's leftovers
    for K, Nper, seed in [(9, 3000, 1), (5, 1200, 2)]:
        u, N_k = _ukn(K, Nper, seed)
        ud = torch.from_numpy(u).cuda()
        f_ref, it_ref = ctx.mbar(ud, N_k, tol=1e-10)
        st, f, it = _noalloc(ctx, ud, N_k)
        assert st == OK, ctx.last_error()
        assert np.max(np.abs(f - f_ref)) <= TOL
        assert it == it_ref


def test_noalloc_mbar_rejects_sizes_beyond_its_buffer():
    from paper_1507_03703_gb300.algdock import E_INVALID, Context
    ctx = Context(0)
    K, N = 2, 1_100_000  # 8.8 MB of per-sample scratch alone, above the 8 MiB buffer
    u = torch.zeros((K, N), dtype=torch.float64, device="cuda")
    st, _, _ = _noalloc(ctx, u, np.array([N // 2, N - N // 2]))
    assert st == E_INVALID
    assert "bytes of scratch" in ctx.last_error()


def test_noalloc_mbar_rejects_precision_mode_2_by_name():
    """Mode 2 keeps an FP32 copy of u_kn that the fixed array does not hold: the call says so."""
    from paper_1507_03703_gb300.algdock import E_INVALID, Context
    ctx = Context(0)
    u = torch.zeros((2, 10), dtype=torch.float64, device="cuda")
    L = ctx._L
    f = np.zeros(2)
    it = ctypes.c_int32()
    Nk = np.array([5, 5], dtype=np.int64)
    st = L.algdock_mbar_noalloc(ctx.h, 2, 10, u.data_ptr(), Nk.ctypes.data, 1e-10, 100, 2, f.ctypes.data,
                                ctypes.byref(it))
    assert st == E_INVALID
    assert "precision_mode" in ctx.last_error()
