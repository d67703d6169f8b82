"""Replica-exchange HMC runs and BPMF estimation on the GPU, through the C ABI.

Bookkeeping only (device buffers, call order, history of components); every step of the method
runs in libalgdock's kernels.  Replicas are stored leg-major: for each leg (ladder of K states),
n_chains independent chains of K configuration slots, so slot r = leg_base + c*K + i.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from .algdock import N_COUNTERS, Context


@dataclass
class Leg:
    K: int
    state_offset: int  # first state of this leg in the context's state table


class ReplicaExchange:
    """All legs of one ligand: HMC for every slot in one launch, then exchange per leg."""

    def __init__(self, ctx: Context, legs, n_chains: int, x0, seed: int, n_sweeps: int = 25, max_sep: int = 5,
                 device="cuda", rep_offset: int = 0, ladder_offset: int = 0, n_external: int = 0,
                 alpha_max: float = 0.01, sigma: float = 0.6, batched: bool = False):
        """rep_offset / ladder_offset: global index of this run's first replica slot and first
        ladder in the Philox counters (a rank's share of a sharded run; see ranks.Shard).
        n_external: external-coordinate moves per replica after each HMC move at states with
        alpha < alpha_max (the paper: 20, 0.01, sigma 0.6 A); 0 leaves them out.
        batched: chain c runs ligand c of the context's multi-ligand batch (x0 holds each slot's
        positions padded to a common atom stride; call ctx.batch_layout(self.lig_of(), stride)
        before the first cycle)."""
        self.ctx, self.legs, self.C = ctx, list(legs), int(n_chains)
        self.seed, self.n_sweeps, self.max_sep = int(seed), int(n_sweeps), int(max_sep)
        self.rep_offset, self.ladder_offset = int(rep_offset), int(ladder_offset)
        self.n_external, self.alpha_max, self.sigma = int(n_external), float(alpha_max), float(sigma)
        self.batched = bool(batched)
        if self.batched and self.n_external:
            raise ValueError("external-coordinate moves run on single-ligand contexts only")
        self.R = self.C * sum(l.K for l in self.legs)
        x0 = np.asarray(x0, dtype=np.float32)
        if x0.shape[0] != self.R:
            raise ValueError("x0 must hold n_chains * sum(K) configurations")
        self.n_atoms = x0.shape[1]
        dev = torch.device(device)
        self.x = torch.from_numpy(np.ascontiguousarray(x0)).to(dev)
        self.comps = torch.zeros((self.R, 4), dtype=torch.float64, device=dev)
        self.dH = torch.zeros(self.R, dtype=torch.float64, device=dev)
        self.acc = torch.zeros(self.R, dtype=torch.uint8, device=dev)
        self.ext_acc = torch.zeros(self.R, dtype=torch.int32, device=dev)
        self.counters = torch.zeros(N_COUNTERS, dtype=torch.int64, device=dev)
        self.base = []
        state = np.empty(self.R, dtype=np.int32)
        b = 0
        self.config_of, self.attempts, self.accepts = [], [], []
        for leg in self.legs:
            self.base.append(b)
            for c in range(self.C):
                state[b + c * leg.K: b + (c + 1) * leg.K] = leg.state_offset + np.arange(leg.K)
            self.config_of.append(torch.arange(leg.K, dtype=torch.int32, device=dev).repeat(self.C).contiguous())
            self.attempts.append(torch.zeros((self.max_sep, leg.K), dtype=torch.int64, device=dev))
            self.accepts.append(torch.zeros((self.max_sep, leg.K), dtype=torch.int64, device=dev))
            b += self.C * leg.K
        self.state_of = torch.from_numpy(state).to(dev)
        self.history = []

    def leg_slice(self, li):
        b = self.base[li]
        return slice(b, b + self.C * self.legs[li].K)

    def lig_of(self):
        """Chain (batch ligand) of every slot, host int32 [R]."""
        out = np.empty(self.R, dtype=np.int32)
        for li, leg in enumerate(self.legs):
            b = self.base[li]
            out[b:b + self.C * leg.K] = np.repeat(np.arange(self.C, dtype=np.int32), leg.K)
        return out

    def hmc(self, cycle: int, n_steps: int):
        run = self.ctx.batch_hmc_cycle if self.batched else self.ctx.hmc_cycle
        run(self.state_of, self.x, self.comps, self.dH, self.acc, n_steps=n_steps, seed=self.seed, cycle=cycle,
            rep_offset=self.rep_offset, counters=self.counters)

    def external(self, cycle: int):
        if self.n_external > 0:
            self.ctx.external_moves(self.state_of, self.x, self.comps, self.n_external, seed=self.seed, cycle=cycle,
                                    alpha_max=self.alpha_max, sigma=self.sigma, rep_offset=self.rep_offset,
                                    accepted=self.ext_acc)

    def _exchange_leg(self, li, cycle):
        leg = self.legs[li]
        sl = self.leg_slice(li)
        self.ctx.exchange(leg.K, leg.state_offset, self.comps[sl], self.config_of[li], self.state_of[sl],
                          n_sweeps=self.n_sweeps, max_sep=self.max_sep, seed=self.seed, cycle=cycle,
                          ladder_offset=self.ladder_offset + li * self.C, attempts=self.attempts[li],
                          accepts=self.accepts[li])

    def exchange(self, cycle: int):
        """Exchange sweeps on every ladder.  The legs' ladders are independent; with the context on a
        torch stream, legs after the first run on side streams (ordered by events), so that the
        one-block-per-ladder launches of the two legs share the GPU instead of taking turns."""
        main = getattr(self.ctx, "stream", None)
        if len(self.legs) < 2 or main is None:
            for li in range(len(self.legs)):
                self._exchange_leg(li, cycle)
            return
        if not hasattr(self, "_side"):
            self._side = [torch.cuda.Stream(device=main.device) for _ in self.legs[1:]]
        ready = torch.cuda.Event()
        ready.record(main)
        for li, side in enumerate(self._side, 1):
            side.wait_event(ready)
            self.ctx.set_stream(side)
            self._exchange_leg(li, cycle)
        self.ctx.set_stream(main)
        self._exchange_leg(0, cycle)
        for side in self._side:
            done = torch.cuda.Event()
            done.record(side)
            main.wait_event(done)

    def cycle(self, cycle: int, n_steps: int, record: bool = False):
        """One iteration ("Equilibration and production"): an HMC move and the external-coordinate
        moves for every replica, then the exchange sweeps."""
        self.hmc(cycle, n_steps)
        self.external(cycle)
        self.exchange(cycle)
        if record:
            self.history.append(self.comps.clone())

    def free_energies(self, li: int, tol=1e-10, max_iter=10000, precision_mode=0, chains=None):
        """MBAR over the recorded components of leg li (optionally a subset of chains)."""
        leg = self.legs[li]
        sl = self.leg_slice(li)
        H = torch.stack([h[sl] for h in self.history], 0).reshape(len(self.history), self.C, leg.K, 4)
        if chains is not None:
            H = H[:, chains]
        comps = H.reshape(-1, 4).contiguous()
        N = comps.shape[0]
        u = torch.empty((leg.K, N), dtype=torch.float64, device=comps.device)
        self.ctx.reduced_energies(N, comps=comps, k_begin=leg.state_offset, k_count=leg.K, u_kn=u)
        N_k = np.full(leg.K, N // leg.K, dtype=np.int64)
        return self.ctx.mbar(u, N_k, tol=tol, max_iter=max_iter, precision_mode=precision_mode)


def bpmf_kT(f_bc, f_cd):
    """beta_T B = f_BC,L + f'_CD: last-minus-first reduced free energy of each ladder ("Estimation")."""
    return (f_bc[-1] - f_bc[0]) + (f_cd[-1] - f_cd[0])
