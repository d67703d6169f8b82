"""Protocol initialization on the GPU ("Initialization"): one leg's states placed one after another.

For each new state:
1. the next parameter is one thermodynamic-length step from the current state; the step uses the
   standard deviations of the current state's samples (warming leg: T; coupling leg: alpha);
2. seeds are resampled from the current state's samples with weights exp(u_k - u_{k+1});
3. the seeds are sampled (HMC trials) at the new state, and the time step is adapted until the
   acceptance lies in [0.4, 0.8];
4. the spacing is checked by the mean exchange probability between the two states' samples.
   Below 0.4 the speed shrinks by 4/5 and the state is placed again; above 0.99 the new state
   replaces the current one.

The sampling, the statistics, the resampling and the exchange probabilities run in the library's
kernels, and the scalar steps (the parameter steps, the time-step rule, the insertion rule) in its
host entry points.  This module holds the state-by-state control flow.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def _lib():
    from .algdock import load_library
    return load_library()


def _call(name, *args):
    import ctypes
    from .algdock import AlgdockError
    out = ctypes.c_double()
    st = getattr(_lib(), name)(*[float(a) for a in args], ctypes.byref(out))
    if st != 0:
        raise AlgdockError(st, name + ": bad arguments")
    return out.value


def next_temperature(T, sigma_U, speed, T_end=600.0):
    """Warming leg, one thermodynamic-length step (algdock_next_temperature)."""
    return _call("algdock_next_temperature", T, sigma_U, speed, T_end)


def next_alpha(a, sigma_sg, sigma_g, sigma_u, speed, T_T=300.0, T_H=600.0):
    """Coupling leg, one thermodynamic-length step (algdock_next_alpha)."""
    return _call("algdock_next_alpha", a, sigma_sg, sigma_g, sigma_u, speed, T_T, T_H)


def adapt_dt(dt, acc):
    """The time-step rule (algdock_adapt_dt)."""
    return _call("algdock_adapt_dt", dt, acc)


def insertions(T, alpha, dt, attempts, accepts, threshold=0.4, T_T=300.0, T_H=600.0):
    """Between cycles ("Equilibration and production"), through algdock_insert_states: a state
    goes between every neighbour pair whose exchange acceptance is below the threshold.
    attempts / accepts: neighbour-pair counts [K - 1].  Returns the new (T, alpha, dt) and, for
    each new state, (its index, the index of its lower neighbour)."""
    import ctypes
    from .algdock import AlgdockError
    T, alpha, dt = (np.ascontiguousarray(v, dtype=np.float64) for v in (T, alpha, dt))
    K = T.size
    att = np.zeros(max(K, 1), dtype=np.int64)
    acc = np.zeros(max(K, 1), dtype=np.int64)
    att[:K - 1] = np.asarray(attempts, dtype=np.int64)[:K - 1]
    acc[:K - 1] = np.asarray(accepts, dtype=np.int64)[:K - 1]
    cap = 2 * K - 1
    oT, oA, oD = np.empty(cap), np.empty(cap), np.empty(cap)
    low = np.empty(cap, dtype=np.int32)
    n = ctypes.c_int32()
    st = _lib().algdock_insert_states(K, T.ctypes.data, alpha.ctypes.data, dt.ctypes.data, att.ctypes.data, acc.ctypes.data, float(threshold),
            float(T_T), float(T_H), cap, ctypes.byref(n), oT.ctypes.data, oA.ctypes.data, oD.ctypes.data,
            low.ctypes.data)
    if st != 0:
        raise AlgdockError(st, "insert_states: bad arguments")
    m = n.value
    new = [(j, int(low[j])) for j in range(m) if low[j] >= 0]
    return oT[:m].copy(), oA[:m].copy(), oD[:m].copy(), new


class ProtocolBuilder:
    """Builds the states of one leg on a context whose grids and ligand are loaded; the context's
    state table is replaced as states are added."""

    def __init__(self, ctx, n_trials=40, n_steps=50, T_T=300.0, T_H=600.0, device="cuda"):
        self.ctx, self.n_trials, self.n_steps = ctx, int(n_trials), int(n_steps)
        self.T_T, self.T_H = float(T_T), float(T_H)
        self.dev = torch.device(device)
        self.cycle = 0
        self.hmc_trials = 0

    def _set(self, T, A, D):
        self.ctx.states_set(np.array(T, dtype=np.float64), np.array(A, dtype=np.float64),
                            np.array(D, dtype=np.float64))

    def _sample(self, T, A, D, k, seeds, seed, max_attempts=20):
        """Sampling and adaptation at state k from the seeds [n][na][3] (device float32).
        Returns (comps [n_trials*n, 4], x [n_trials*n, na, 3], acceptance, dt)."""
        n = seeds.shape[0]
        st = torch.full((n,), k, dtype=torch.int32, device=self.dev)
        acc = torch.zeros(n, dtype=torch.uint8, device=self.dev)
        for _ in range(max_attempts):
            x = seeds.clone()
            comps = torch.empty((n, 4), dtype=torch.float64, device=self.dev)
            cs, xs, n_acc = [], [], torch.zeros((), dtype=torch.int64, device=self.dev)
            for _t in range(self.n_trials):
                self.ctx.hmc_cycle(st, x, comps, accepted=acc, n_steps=self.n_steps, seed=seed, cycle=self.cycle)
                self.cycle += 1
                self.hmc_trials += 1
                cs.append(comps.clone())
                xs.append(x.clone())
                n_acc += acc.sum()
            rate = float(n_acc.item()) / (self.n_trials * n)
            if 0.4 <= rate <= 0.8:
                break
            new = adapt_dt(D[k], rate)
            if new == D[k]:
                break
            D[k] = new
            self._set(T, A, D)
        return torch.cat(cs), torch.cat(xs), rate, D[k]

    def build_leg(self, leg, seeds, seed, speed=None, dt0=2.0, max_states=400, max_reselect=40):
        """leg "bc" (300 -> 600 K, no grids) or "cd" (alpha 0 -> 1, T from 600 to 300 K); seeds
        [n][na][3] float32 (numpy or device).  Returns dict(T, alpha, dt, pacc, acceptance, speed,
        hmc_trials)."""
        bc = leg == "bc"
        speed = (20.0 if bc else 0.2) if speed is None else float(speed)
        seeds = torch.as_tensor(np.asarray(seeds, dtype=np.float32)).to(self.dev)
        n = seeds.shape[0]
        T, A, D = ([self.T_T], [math.nan], [dt0]) if bc else ([self.T_H], [0.0], [dt0])
        self._set(T, A, D)
        comps_k, x_k, rate, _ = self._sample(T, A, D, 0, seeds, seed)
        pacc, rates = [], [rate]
        prev = None
        for _ in range(max_states):
            k = len(T) - 1
            if (bc and T[k] >= 600.0) or (not bc and A[k] >= 1.0):
                break
            sig = self.ctx.state_statistics(comps_k, k)
            for _try in range(max_reselect):
                if bc:
                    Tn, An = next_temperature(T[k], sig[0], speed), math.nan
                else:
                    An = next_alpha(A[k], sig[1], sig[2], sig[3], speed, self.T_T, self.T_H)
                    Tn = (self.T_T - self.T_H) * An + self.T_H
                Tc, Ac, Dc = T + [Tn], A + [An], D + [D[k]]
                self._set(Tc, Ac, Dc)
                new_seeds = torch.empty_like(seeds)
                self.ctx.resample(comps_k, k, k + 1, n, seed, 1_000_000 + self.cycle, x_in=x_k, x_out=new_seeds)
                comps_n, x_n, rate_n, dt_n = self._sample(Tc, Ac, Dc, k + 1, new_seeds, seed)
                p = self.ctx.mean_pacc(comps_k, comps_n, k, k + 1)
                if p >= 0.4:
                    break
                speed *= 0.8
            if p > 0.99 and k > 0:  # the current state is too close to its successor: replaced
                T[k], A[k], D[k] = Tn, An, dt_n
                self._set(T, A, D)
                pacc[-1] = self.ctx.mean_pacc(prev, comps_n, k - 1, k)
            else:
                T.append(Tn)
                A.append(An)
                D.append(dt_n)
                pacc.append(p)
            rates.append(rate_n)
            prev = comps_k
            comps_k, x_k = comps_n, x_n
            self._set(T, A, D)
        return {"T": np.array(T), "alpha": np.array(A), "dt": np.array(D), "pacc": np.array(pacc),
                "acceptance": np.array(rates), "speed": speed, "hmc_trials": self.hmc_trials}
