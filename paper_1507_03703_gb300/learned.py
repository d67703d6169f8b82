"""Training and use of the learned pose proposal through the C ABI.

The proposal network is trained on poses that plain HMC itself sampled: for random pairs (x_i,
x_j) of samples at one state, the target is the move that takes x_i to x_j, and the loss is the
mean negative log-density of those moves under the network's mixture.  Every step (features,
targets, forward and backward passes, Adam) runs in the library; this module only picks pairs and
orders the calls.
"""
from __future__ import annotations

import numpy as np
import torch

from . import synthetic
from .algdock import MLP_DMAX, MLP_NFEAT, MLP_NPARAMS, pack_mlp


class LearnedProposal:
    """Device-resident network parameters (FP32 master + BF16 copy) and Adam moments."""

    def __init__(self, ctx, seed: int = 0, device="cuda", n_torsions: int = -1):
        """n_torsions: moved torsions (negative: all the ligand's, 0: rigid-body moves only)."""
        self.ctx = ctx
        flat, w = pack_mlp(synthetic.mlp_init(seed))
        dev = torch.device(device)
        self.params = torch.from_numpy(flat).to(dev)
        self.wbf16 = torch.from_numpy(w.view(np.int16)).to(dev)
        self.m = torch.zeros(MLP_NPARAMS, dtype=torch.float32, device=dev)
        self.v = torch.zeros_like(self.m)
        self.grad = torch.zeros_like(self.m)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.step = 0
        T = ctx.learned_ntorsions()
        self.T = T if n_torsions < 0 else min(T, n_torsions)

    def train(self, x, comps, state, n_iter: int, batch: int = 4096, lr: float = 1e-3, seed: int = 0,
              pairs=None):
        """Adam on the mean negative log-density of moves between pairs of the samples
        x [S][n_atoms][3] (float32, device) with components comps [S][4].  state: one state index
        for all samples, or an array of S state indices (pairs are then drawn within a state).
        Pairs: random, or the given (I, J) index arrays (e.g. the same chain a few cycles apart).
        Returns the loss after each iteration."""
        S = x.shape[0]
        dev = x.device
        rng = np.random.default_rng(seed)
        if pairs is not None:
            PI = torch.as_tensor(np.asarray(pairs[0]), device=dev)
            PJ = torch.as_tensor(np.asarray(pairs[1]), device=dev)
        per_sample = np.ndim(state) > 0
        if per_sample:
            st_all = np.asarray(state, dtype=np.int32).ravel()
            order = np.argsort(st_all, kind="stable")
            counts = np.bincount(st_all)
            starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
            st_dev = torch.from_numpy(st_all).to(dev)
            order_dev = torch.from_numpy(order).to(dev)
        else:
            st = torch.full((batch,), int(state), dtype=torch.int32, device=dev)
        feat = torch.empty((batch, MLP_NFEAT), dtype=torch.float32, device=dev)
        delta = torch.empty((batch, MLP_DMAX), dtype=torch.float32, device=dev)
        losses = []
        D = 6 + self.T
        for _ in range(n_iter):
            if pairs is not None:
                sel = torch.from_numpy(rng.integers(0, PI.numel(), size=batch)).to(dev)
                i, j = PI[sel], PJ[sel]
            elif per_sample:
                ii = rng.integers(0, S, size=batch)
                k = st_all[ii]
                jj = starts[k] + (rng.random(batch) * counts[k]).astype(np.int64)
                i = torch.from_numpy(ii).to(dev)
                j = order_dev[torch.from_numpy(jj).to(dev)]
            else:
                i = torch.from_numpy(rng.integers(0, S, size=batch)).to(dev)
                j = torch.from_numpy(rng.integers(0, S, size=batch)).to(dev)
            if per_sample:
                st = st_dev[i].contiguous()
            xi, xj = x[i].contiguous(), x[j].contiguous()
            self.ctx.learned_features(st, xi, comps[i].contiguous(), feat)
            self.ctx.pose_delta(xi, xj, delta)
            self.ctx.mlp_grad(self.params, self.wbf16, feat, delta, D, self.grad, self.loss)
            self.step += 1
            self.ctx.mlp_adam(self.params, self.wbf16, self.grad, self.m, self.v, self.step, lr)
            losses.append(self.loss.clone())
        return [float(l.item()) for l in losses]

    def propose(self, state_of, x, comps, n_moves, seed, cycle, accepted=None, counters=None, rep_offset=0):
        self.ctx.propose_learned(self.params, self.wbf16, state_of, x, comps, n_moves, seed=seed, cycle=cycle,
                                 rep_offset=rep_offset, accepted=accepted, counters=counters, n_torsions=self.T)
