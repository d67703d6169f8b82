"""The tcgen05 GEMM of the learned proposal's network (tensor-memory accumulators, TMA operand
tiles): C = epi(A . B^T) against the FP64 product of the same BF16 values, over one tile, ragged
M / N / K edges (the TMA zero fill and the masked epilogue), a K longer than the stage ring, every
epilogue and the split reduction.  Then the network's forward pass and loss gradient at row counts
where they run on this GEMM (from 8192 rows for the forward pass, from 4096 for the gradient),
against the FP64 oracle with the same BF16 roundings."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    from paper_1507_03703_gb300.algdock import Context
    return Context(0)


def _ab(M, N, K, seed):
    g = torch.Generator().manual_seed(seed)
    A = torch.randn(M, K, generator=g).bfloat16()
    B = torch.randn(N, K, generator=g).bfloat16()
    return A, B, A.double() @ B.double().T


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (128, 256, 64), (64, 48, 64), (300, 360, 256), (4096, 256, 256),
                                   (129, 200, 328), (512, 64, 1000)])
def test_gemm_fp32_epilogue(ctx, M, N, K):
    A, B, ref = _ab(M, N, K, M + N + K)
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    ctx.gemm_bf16(A.cuda(), B.cuda(), C, epilogue=0)
    got = C.cpu().double()
    # FP32 accumulation of K products of BF16 values: relative to the largest entry
    assert torch.isfinite(got).all()
    assert (got - ref).abs().max().item() <= 1e-5 * ref.abs().max().item() * max(1.0, K / 256)


def test_gemm_epilogues_and_split(ctx):
    M, N, K = 520, 264, 256
    A, B, ref = _ab(M, N, K, 7)
    bias = torch.randn(N, generator=torch.Generator().manual_seed(8))
    mask = torch.randn(M, N, generator=torch.Generator().manual_seed(9)).bfloat16()
    tol = 1e-5 * ref.abs().max().item()
    C = torch.empty((M, N), dtype=torch.float32, device="cuda")
    ctx.gemm_bf16(A.cuda(), B.cuda(), C, epilogue=1, bias=bias.cuda())
    assert (C.cpu().double() - (ref + bias.double())).abs().max().item() <= tol
    H = torch.empty((M, N), dtype=torch.bfloat16, device="cuda")
    ctx.gemm_bf16(A.cuda(), B.cuda(), H, epilogue=2, bias=bias.cuda())
    want = torch.clamp(ref + bias.double(), min=0.0)
    assert (H.cpu().double() - want).abs().max().item() <= tol + 2 ** -8 * want.abs().max().item()
    assert torch.all(((H.cpu() == 0) == (want <= 0)) | (want.abs() < tol))
    ctx.gemm_bf16(A.cuda(), B.cuda(), H, epilogue=3, mask=mask.cuda())
    want = torch.where(mask.double() > 0, ref, torch.zeros_like(ref))
    assert (H.cpu().double() - want).abs().max().item() <= tol + 2 ** -8 * want.abs().max().item()
    # split reduction over a long K: the slices' partial products sum to the product
    M2, N2, K2 = 360, 256, 4104  # a row stride of 16-byte multiples (TMA), not a multiple of the 64-wide stage
    A2, B2, ref2 = _ab(M2, N2, K2, 10)
    P = torch.zeros((16, M2, N2), dtype=torch.float32, device="cuda")
    ctx.gemm_bf16(A2.cuda(), B2.cuda(), P, epilogue=0, n_split=16)
    assert (P.sum(0).cpu().double() - ref2).abs().max().item() <= 2e-5 * ref2.abs().max().item() * (K2 / 256)


def _params(seed):
    from paper_1507_03703_gb300 import synthetic as S
    p = S.mlp_init(seed, out_scale=0.5)
    rng = np.random.default_rng(seed)
    for k in ("b1", "b2", "b3", "b4"):  # nonzero biases, so the epilogues' bias terms count
        p[k] = rng.normal(scale=0.1, size=p[k].shape)
    return p


def _device(p):
    from paper_1507_03703_gb300.algdock import bf16_values, pack_mlp
    flat, w16 = pack_mlp(p)
    return torch.from_numpy(flat).cuda(), torch.from_numpy(w16.view(np.int16)).cuda()


def _bf16_params(p):
    from paper_1507_03703_gb300.algdock import bf16_values
    return {k: (bf16_values(v) if k.startswith("W") else np.asarray(v, dtype=np.float32)).astype(np.float64)
            for k, v in p.items()}


@pytest.mark.parametrize("N", [8192, 8200])
def test_network_forward_on_the_tensor_cores(ctx, N):
    p = _params(21)
    pd, wd = _device(p)
    X = np.random.default_rng(22).normal(size=(N, 64)).astype(np.float32)
    out = torch.empty((N, 360), dtype=torch.float32, device="cuda")
    ctx.mlp_forward(pd, wd, torch.from_numpy(X).cuda(), out)
    oracle.set_bf16_activations(True)
    try:
        ref = oracle.mlp_forward(_bf16_params(p), X.astype(np.float64))[0]
    finally:
        oracle.set_bf16_activations(False)
    g = out.cpu().numpy()
    rel = np.linalg.norm(g - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.median(rel) < 1e-3 and rel.max() < 2e-2, (np.median(rel), rel.max())


def test_network_gradient_on_the_tensor_cores(ctx):
    from paper_1507_03703_gb300.algdock import unpack_mlp
    p = _params(31)
    pd, wd = _device(p)
    rng = np.random.default_rng(32)
    N, D = 4099, 15
    X = rng.normal(size=(N, 64)).astype(np.float32)
    tgt = np.zeros((N, 22), dtype=np.float32)
    tgt[:, :D] = rng.normal(scale=0.3, size=(N, D))
    grad = torch.empty(pd.numel(), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    ctx.mlp_grad(pd, wd, torch.from_numpy(X).cuda(), torch.from_numpy(tgt).cuda(), D, grad, loss)
    g = unpack_mlp(grad.cpu().numpy())
    q = _bf16_params(p)
    oracle.set_bf16_activations(True)
    try:
        out, h1, h2, h3 = oracle.mlp_forward(q, X.astype(np.float64))
    finally:
        oracle.set_bf16_activations(False)
    dout = np.zeros_like(out)
    lq = np.zeros(N)
    for n in range(N):
        lq[n], gn = oracle.mixture_logq(out[n], D, tgt[n, :D].astype(np.float64), grad=True)
        dout[n] = -gn / N
    go = oracle.mlp_backward(q, X.astype(np.float64), h1, h2, h3, dout)
    for k in g:
        rel = np.linalg.norm(g[k] - go[k]) / max(np.linalg.norm(go[k]), 1e-30)
        assert rel < 3e-2, (k, rel)
    assert float(loss.item()) == pytest.approx(-lq.mean(), rel=2e-3)
