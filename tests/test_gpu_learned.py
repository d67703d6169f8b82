"""GPU parity of the learned pose proposal (an extension of the paper's external-coordinate moves,
"Sampling") against the FP64 oracle.

- features and training targets: FP32/FP64 arithmetic on the same float poses, 1e-5 absolute;
- network outputs: the oracle runs in FP64 with the same BF16 weights and with its input and
  hidden activations rounded to BF16 where the tensor-core path stores them, so the two differ
  by FP32 accumulation and the rare activation that rounds to the neighbouring BF16 value:
  median per-row relative error < 1e-3, every row < 2e-2;
- gradients of the mean negative log-density: the backward pass also rounds the propagated
  gradients to BF16 (relative 2^-9 each), so per tensor ||dg|| / ||g|| < 3e-2;
- one Adam step against the published update rule (Kingma & Ba), 1e-6 relative;
- the learned Metropolis-Hastings move: decisions agree wherever the oracle's log-acceptance
  margin exceeds 0.05, positions of moves both accept agree to 1e-3 A, rejected poses are kept
  bit for bit; and on its own, a chain of learned moves on the GPU samples a harmonic well."""
import math

import numpy as np
import pytest

import oracle
from paper_1507_03703_gb300 import synthetic as S

from systems import configurations, gpu_context, oracle_system, raw_grids32, state_table

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def small():
    sys_ = S.config_small(1)
    g32 = raw_grids32(sys_)
    T, alpha, dt = state_table(sys_)
    ctx = gpu_context(sys_, g32, T, alpha, dt)
    osys = oracle_system(sys_, g32, T, alpha, dt)
    return sys_, g32, T, alpha, dt, ctx, osys


def _params(seed, sigma_bias=0.0):
    p = S.mlp_init(seed, out_scale=0.5)
    p["b4"][8 + 8 * 22:] = sigma_bias
    return p


def _device_params(p):
    from paper_1507_03703_gb300.algdock import pack_mlp
    flat, w = pack_mlp(p)
    return torch.from_numpy(flat).cuda(), torch.from_numpy(w.view(np.int16)).cuda()


def _bf16_params(p):
    """The parameters the GPU actually uses: BF16 weights, FP32 biases (as float64)."""
    from paper_1507_03703_gb300.algdock import bf16_values
    q = {}
    for k, v in p.items():
        q[k] = bf16_values(v).astype(np.float64) if k.startswith("W") else np.asarray(v, np.float32).astype(np.float64)
    return q


def _comps_of(osys, x):
    return np.array([osys.energy_force(xi.astype(np.float64))[0] for xi in x])


def test_features_and_targets(small):
    sys_, g32, T, alpha, dt, ctx, osys = small
    assert ctx.learned_ntorsions() == osys.learned_ntorsions()
    N = 70
    x = configurations(sys_, N, seed=21, jitter=0.3)
    y = configurations(sys_, N, seed=22, jitter=0.3)
    comps = _comps_of(osys, x)
    states = (np.arange(N) % len(T)).astype(np.int32)
    feat = torch.empty((N, 64), dtype=torch.float32, device="cuda")
    ctx.learned_features(torch.from_numpy(states).cuda(), torch.from_numpy(x).cuda(), torch.from_numpy(comps).cuda(),
                         feat)
    delta = torch.empty((N, 22), dtype=torch.float32, device="cuda")
    ctx.pose_delta(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), delta)
    torch.cuda.synchronize()
    f, d = feat.cpu().numpy(), delta.cpu().numpy()
    D = 6 + osys.learned_ntorsions()
    for n in range(N):
        fo = osys.features(x[n].astype(np.float64), comps[n], states[n])
        assert np.max(np.abs(f[n] - fo)) < 1e-5, n
        do = osys.pose_delta(x[n].astype(np.float64), y[n].astype(np.float64))
        err = d[n, :D] - do
        err[6:] = (err[6:] + np.pi) % (2 * np.pi) - np.pi
        assert np.max(np.abs(err)) < 1e-5, n
        assert np.all(d[n, D:] == 0.0)


def test_network_forward(small):
    ctx = small[5]
    p = _params(3)
    pd, wd = _device_params(p)
    rng = np.random.default_rng(4)
    N = 300  # several 64-row tiles and a ragged one
    X = rng.normal(size=(N, 64)).astype(np.float32)
    out = torch.empty((N, 360), dtype=torch.float32, device="cuda")
    ctx.mlp_forward(pd, wd, torch.from_numpy(X).cuda(), out)
    torch.cuda.synchronize()
    oracle.set_bf16_activations(True)
    try:
        ref = oracle.mlp_forward(_bf16_params(p), X.astype(np.float64))[0]
    finally:
        oracle.set_bf16_activations(False)
    g = out.cpu().numpy()
    rel = np.linalg.norm(g - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.median(rel) < 1e-3 and rel.max() < 2e-2, (np.median(rel), rel.max())


def test_fused_forward_matches_layer_by_layer(small):
    """The fused one-kernel forward pass (16-byte aligned operands) and the layer-by-layer GEMM path
    (taken for a misaligned feature pointer) round at the same places, so they agree to FP32
    accumulation order and the rare BF16 activation that rounds the other way."""
    ctx = small[5]
    p = _params(12)
    pd, wd = _device_params(p)
    rng = np.random.default_rng(13)
    N = 1000
    X = torch.from_numpy(rng.normal(size=(N, 64)).astype(np.float32)).cuda()
    store = torch.empty(N * 64 + 1, dtype=torch.float32, device="cuda")
    Xm = store[1:].view(N, 64)
    Xm.copy_(X)
    assert Xm.data_ptr() % 16 != 0
    a = torch.empty((N, 360), dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    ctx.mlp_forward(pd, wd, X, a)
    ctx.mlp_forward(pd, wd, Xm, b)
    torch.cuda.synchronize()
    a, b = a.cpu().numpy(), b.cpu().numpy()
    rel = np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)
    assert np.median(rel) < 1e-4 and rel.max() < 2e-2, (np.median(rel), rel.max())


def test_network_gradient_and_loss(small):
    ctx = small[5]
    p = _params(5)
    pd, wd = _device_params(p)
    rng = np.random.default_rng(6)
    N, D = 200, 17
    X = rng.normal(size=(N, 64)).astype(np.float32)
    tgt = np.zeros((N, 22), dtype=np.float32)
    tgt[:, :D] = rng.normal(scale=0.3, size=(N, D))
    grad = torch.empty(pd.numel(), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    ctx.mlp_grad(pd, wd, torch.from_numpy(X).cuda(), torch.from_numpy(tgt).cuda(), D, grad, loss)
    torch.cuda.synchronize()
    from paper_1507_03703_gb300.algdock import unpack_mlp
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


def test_adam_step_follows_the_published_rule(small):
    ctx = small[5]
    p = _params(7)
    pd, wd = _device_params(p)
    flat0 = pd.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(8)
    g = rng.normal(size=flat0.size).astype(np.float32)
    m = torch.from_numpy((0.1 * rng.normal(size=flat0.size)).astype(np.float32)).cuda()
    v = torch.from_numpy(np.abs(0.01 * rng.normal(size=flat0.size)).astype(np.float32)).cuda()
    m0, v0 = m.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
    step, lr = 3, 1e-3
    ctx.mlp_adam(pd, wd, torch.from_numpy(g).cuda(), m, v, step, lr)
    torch.cuda.synchronize()
    mm = 0.9 * m0 + 0.1 * g
    vv = 0.999 * v0 + 0.001 * g.astype(np.float64) ** 2
    new = flat0 - lr * (mm / (1 - 0.9 ** step)) / (np.sqrt(vv / (1 - 0.999 ** step)) + 1e-8)
    got = pd.cpu().numpy()
    assert np.allclose(got, new, rtol=1e-5, atol=1e-7)
    from paper_1507_03703_gb300.algdock import bf16_bits, unpack_mlp
    w = np.concatenate([unpack_mlp(got)[k].ravel() for k in ("W1", "W2", "W3", "W4")])
    assert np.array_equal(wd.cpu().numpy().view(np.uint16), bf16_bits(w))


def test_learned_move_matches_oracle(small):
    sys_, g32, T, alpha, dt, ctx, osys = small
    p = _params(9, sigma_bias=1.0)
    pd, wd = _device_params(p)
    R = 128
    x = configurations(sys_, R, seed=23, jitter=0.05)
    comps = _comps_of(osys, x)
    states = (np.arange(R) % len(T)).astype(np.int32)
    xd = torch.from_numpy(x.copy()).cuda()
    cd = torch.from_numpy(comps.copy()).cuda()
    acc = torch.zeros(R, dtype=torch.int32, device="cuda")
    seed, cycle = 77, 5
    ctx.propose_learned(pd, wd, torch.from_numpy(states).cuda(), xd, cd, 1, seed=seed, cycle=cycle, accepted=acc)
    torch.cuda.synchronize()
    xg, ag = xd.cpu().numpy(), acc.cpu().numpy()
    oracle.set_bf16_activations(True)
    try:
        xo, co, ao, lr = osys.learned_mh(_bf16_params(p), x.astype(np.float64), comps, states, 1, seed, cycle)
    finally:
        oracle.set_bf16_activations(False)
    u = np.array([oracle.u53(*[int(v) for v in oracle.philox4x32_10([101, r, cycle, 4],
                                                                     [seed & 0xFFFFFFFF, seed >> 32])[:2]])
                  for r in range(R)])
    margin = np.abs(lr - np.log(np.maximum(u, 1e-300)))
    clear = margin > 0.05
    assert clear.sum() > R // 2
    assert np.array_equal(ag[clear], ao[clear])
    both = (ag == 1) & (ao == 1)
    assert both.sum() > 0
    assert np.max(np.abs(xg[both] - xo[both])) < 1e-3
    rej = ag == 0
    assert np.array_equal(xg[rej], x[rej])


def test_learned_chain_samples_a_harmonic_well_on_the_gpu():
    """One atom in a pure harmonic restraint (d0 = 0) on zero grids: a chain of learned moves with
    a random network gives <|r - c|^2> = 3 kT / k."""
    from paper_1507_03703_gb300.algdock import Context
    k = 5.0
    grid = S.cube_grid(np.zeros(3), 1.0, 5)
    zero = np.zeros((5, 5, 5), dtype=np.float32)
    lig = S.one_atom_ligand(charge=0.0)
    ctx = Context(0)
    ctx.grids_load(grid, zero, zero, zero, ligand=lig)
    ctx.ligand_load(lig, np.zeros(3), k=k, d0=0.0)
    ctx.states_set([300.0], [np.nan], [2.0])
    p = _params(10)
    pd, wd = _device_params(p)
    R = 2048
    rng = np.random.default_rng(11)
    x = torch.from_numpy(rng.normal(scale=0.3, size=(R, 1, 3)).astype(np.float32)).cuda()
    comps = torch.empty((R, 4), dtype=torch.float64, device="cuda")
    ctx.reduced_energies(R, x=x, comps=comps)
    st = torch.zeros(R, dtype=torch.int32, device="cuda")
    vals = []
    for cyc in range(60):
        ctx.propose_learned(pd, wd, st, x, comps, 4, seed=12, cycle=cyc)
        if cyc >= 10:
            vals.append((x[:, 0, :] ** 2).sum(-1).cpu().numpy())
    per = np.array(vals).mean(0)
    exact = 3 * oracle.KB * 300.0 / k
    assert abs(per.mean() - exact) < 4 * per.std(ddof=1) / math.sqrt(R), (per.mean(), exact)
