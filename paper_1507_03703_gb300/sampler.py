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

    def acceptance(self, li: int):
        """Neighbour-pair exchange acceptance of leg li since its counters were last reset, [K - 1]."""
        att = self.attempts[li][0, :-1].double().cpu().numpy()
        acc = self.accepts[li][0, :-1].double().cpu().numpy()
        return np.divide(acc, att, out=np.full_like(att, np.nan), where=att > 0)

    def insert_states(self, T, alpha, dt, threshold=0.4, seed=0, counter=0):
        """Between cycles ("Equilibration and production"): where a leg's neighbour exchange
        acceptance over the cycles since the last insertion fell below the threshold, insert a
        state (protocol.insertions) and populate it by sampling importance resampling: each chain's
        configuration for the new state is drawn from the configurations at its lower neighbour,
        all chains pooled, with weights exp(u_lower - u_new) (the library's resample kernel).
        T, alpha, dt: the context's whole state table, which this run's legs make up in order.
        Rebuilds the state table, the replica buffers (identity permutations), zeroes the exchange
        counters and clears the recorded history (a sharded run renumbers its replicas: its rank
        offsets follow the new ladder sizes).  Returns the new (T, alpha, dt) and, per leg, the
        indices of the inserted states within the leg."""
        from .protocol import insertions
        T, alpha, dt = np.asarray(T, float), np.asarray(alpha, float), np.asarray(dt, float)
        if T.size != sum(l.K for l in self.legs) or any(
                l.state_offset != sum(m.K for m in self.legs[:i]) for i, l in enumerate(self.legs)):
            raise ValueError("insert_states needs the run's legs to make up the whole state table, in order")
        dev = self.x.device
        plans, nT, nA, nD = [], [], [], []
        for li, leg in enumerate(self.legs):
            o = leg.state_offset
            att = self.attempts[li][0, :leg.K - 1].cpu().numpy()
            acc = self.accepts[li][0, :leg.K - 1].cpu().numpy()
            lt, la, ld, new = insertions(T[o:o + leg.K], alpha[o:o + leg.K], dt[o:o + leg.K], att, acc, threshold)
            plans.append((lt.size, new))
            nT.append(lt)
            nA.append(la)
            nD.append(ld)
        if all(not new for _, new in plans):
            return T, alpha, dt, [[] for _ in self.legs]
        newT, newA, newD = np.concatenate(nT), np.concatenate(nA), np.concatenate(nD)
        self.ctx.states_set(newT, newA, newD)
        C, na = self.C, self.n_atoms
        xs_legs, cs_legs, legs, off = [], [], [], 0
        for li, (leg, (K2, new)) in enumerate(zip(self.legs, plans)):
            sl = self.leg_slice(li)
            # configurations and components by state: slot config_of[c, k] of chain c holds state k
            cfg = self.config_of[li].view(C, leg.K).long()
            rows = (torch.arange(C, device=dev)[:, None] * leg.K + cfg).reshape(-1)
            xk = self.x[sl][rows].view(C, leg.K, na, 3)
            ck = self.comps[sl][rows].view(C, leg.K, 4)
            old_pos = [k2 for k2 in range(K2) if k2 not in {n for n, _ in new}]
            x2 = torch.empty((C, K2, na, 3), dtype=self.x.dtype, device=dev)
            c2 = torch.empty((C, K2, 4), dtype=torch.float64, device=dev)
            x2[:, old_pos] = xk
            c2[:, old_pos] = ck
            for j, (n, lower) in enumerate(new):
                k_lower = old_pos.index(lower)
                pool_c = ck[:, k_lower].contiguous()
                pool_x = xk[:, k_lower].contiguous()
                idx = torch.empty(C, dtype=torch.int64, device=dev)
                xo = torch.empty((C, na, 3), dtype=self.x.dtype, device=dev)
                self.ctx.resample(pool_c, off + lower, off + n, C, seed, counter + 1000 * li + j, x_in=pool_x,
                                  x_out=xo, idx=idx)
                x2[:, n] = xo
                c2[:, n] = pool_c[idx]
            xs_legs.append(x2.reshape(-1, na, 3))
            cs_legs.append(c2.reshape(-1, 4))
            legs.append(Leg(K2, off))
            off += K2
        self.legs = legs
        self.R = C * sum(l.K for l in legs)
        self.x = torch.cat(xs_legs).contiguous()
        self.comps = torch.cat(cs_legs).contiguous()
        self.dH = torch.zeros(self.R, dtype=torch.float64, device=dev)
        self.acc = torch.zeros(self.R, dtype=torch.uint8, device=dev)
        self.ext_acc = torch.zeros(self.R, dtype=torch.int32, device=dev)
        self.base, state = [], np.empty(self.R, dtype=np.int32)
        self.config_of, self.attempts, self.accepts = [], [], []
        b = 0
        for leg in legs:
            self.base.append(b)
            for c in range(C):
                state[b + c * leg.K: b + (c + 1) * leg.K] = leg.state_offset + np.arange(leg.K)
            self.config_of.append(torch.arange(leg.K, dtype=torch.int32, device=dev).repeat(C).contiguous())
            self.attempts.append(torch.zeros((self.max_sep, leg.K), dtype=torch.int64, device=dev))
            self.accepts.append(torch.zeros((self.max_sep, leg.K), dtype=torch.int64, device=dev))
            b += C * leg.K
        self.state_of = torch.from_numpy(state).to(dev)
        self.history = []
        if self.batched:
            self.ctx.batch_layout(self.lig_of(), na)
        return newT, newA, newD, [[n for n, _ in new] for _, new in plans]

    # ---------------------------------------------------------------- checkpoint and resume
    def _buffers(self):
        a = {"legs": np.array([[l.K, l.state_offset] for l in self.legs], dtype=np.int32).ravel(),
             "x": self.x, "comps": self.comps, "state_of": self.state_of, "dH": self.dH, "acc": self.acc,
             "ext_acc": self.ext_acc, "counters": self.counters}
        for li in range(len(self.legs)):
            a["config_of_%d" % li] = self.config_of[li]
            a["attempts_%d" % li] = self.attempts[li]
            a["accepts_%d" % li] = self.accepts[li]
        return a

    def save(self, path, next_cycle: int):
        """Checkpoint of the run through algdock_checkpoint_save: the context's state table (with
        every state's time step), the seed, the next cycle and every buffer the run keeps between
        cycles, the recorded components included."""
        from .algdock import checkpoint_save
        a = self._buffers()
        a["history"] = (torch.stack(self.history).contiguous() if self.history else
                        torch.zeros((0, self.R, 4), dtype=torch.float64, device=self.x.device))
        checkpoint_save(self.ctx, path, self.seed, next_cycle, a)

    def load(self, path) -> int:
        """Restores a checkpoint written by save (on a context holding the same ligand and lattice;
        the legs may differ from the constructor's, e.g. after state insertion).  The context's state
        table is restored too.  Returns the cycle to run next."""
        from .algdock import checkpoint_load, checkpoint_query
        q = checkpoint_query(self.ctx, path, ["legs", "x", "history"])
        if q["legs"][1] < 2 or q["x"][1] < 0:
            raise ValueError("not a replica-exchange checkpoint: " + str(path))
        la = np.zeros(q["legs"][1], dtype=np.int32)
        checkpoint_load(None, path, {"legs": la})
        legs = [Leg(int(la[2 * i]), int(la[2 * i + 1])) for i in range(la.size // 2)]
        R = q["x"][1] // (self.n_atoms * 3)
        C = R // sum(l.K for l in legs)
        dev = self.x.device
        self.legs, self.C, self.R = legs, C, R
        self.x = torch.empty((R, self.n_atoms, 3), dtype=torch.float32, device=dev)
        self.comps = torch.empty((R, 4), dtype=torch.float64, device=dev)
        self.dH = torch.empty(R, dtype=torch.float64, device=dev)
        self.acc = torch.empty(R, dtype=torch.uint8, device=dev)
        self.ext_acc = torch.empty(R, dtype=torch.int32, device=dev)
        self.state_of = torch.empty(R, dtype=torch.int32, device=dev)
        self.base, b = [], 0
        for leg in legs:
            self.base.append(b)
            b += C * leg.K
        self.config_of = [torch.empty(C * l.K, dtype=torch.int32, device=dev) for l in legs]
        self.attempts = [torch.empty((self.max_sep, l.K), dtype=torch.int64, device=dev) for l in legs]
        self.accepts = [torch.empty((self.max_sep, l.K), dtype=torch.int64, device=dev) for l in legs]
        a = self._buffers()
        hist = torch.empty((q["history"][1] // (R * 4), R, 4), dtype=torch.float64, device=dev)
        a["history"] = hist
        seed, cycle = checkpoint_load(self.ctx, path, a)
        self.counters = a["counters"]
        self.seed = int(seed)
        self.history = [h for h in hist]
        if self.batched:
            self.ctx.batch_layout(self.lig_of(), self.n_atoms)
        return int(cycle)

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


def effective_samples(ctx, series):
    """Effective sample size of series [cycles][chains] (device float64): the sum over chains of
    N / g, with g the statistical inefficiency of each chain's whole series from the library's
    equilibration kernel (its first candidate start, t0 = 0)."""
    T = int(series.shape[0])
    s = series.reshape(T, -1).contiguous()
    if T < 2:
        return float(s.shape[1] * T)
    g, _, _ = ctx.detect_equilibration(s, n_cand=1)
    return float((T / g[:, 0]).sum().item())
