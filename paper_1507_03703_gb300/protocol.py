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
kernels. This module holds the state-by-state control flow and the scalar arithmetic of the
parameter steps and the time-step rule.
"""
from __future__ import annotations

import math

import numpy as np
import torch

KB = 0.0019872043  # kcal/(mol K)


def _logistic(z):
    return 1.0 / (1.0 + math.exp(-z)) if z >= 0 else math.exp(z) / (1.0 + math.exp(z))


def d_alpha_sg(a):
    """d alpha_sg / d alpha for alpha_sg = 1 - (2 alpha - 1)^2 (Eq. (protocol))."""
    return -4.0 * (2.0 * a - 1.0)


def d_alpha_g(a):
    """d alpha_g / d alpha for alpha_g = (2 alpha - 1)^2 logistic(1000 (alpha - 1/2)) (Eq. (protocol))."""
    s = 2.0 * a - 1.0
    L = _logistic(1000.0 * (a - 0.5))
    return 4.0 * s * L + s * s * 1000.0 * L * (1.0 - L)


def next_temperature(T, sigma_U, speed, T_end=600.0):
    """Warming leg: sigma[dl/dT] = sigma[U_S] / (k_B T^2), so T + speed k_B T^2 / sigma[U_S]."""
    if sigma_U <= 0.0:  # no fluctuation: the step is unbounded, so the leg's end is next
        return T_end
    return min(T_end, T + speed * KB * T * T / sigma_U)


def next_alpha(a, sigma_sg, sigma_g, sigma_u, speed, T_T=300.0, T_H=600.0):
    """Coupling leg: alpha + speed / (|alpha_sg'| sigma[Psi_sg]/(k_B T) + |alpha_g'| sigma[Psi_g]/(k_B T)
    + |T_T - T_H| sigma[u]/T), T = T(alpha), not past 1."""
    T = (T_T - T_H) * a + T_H
    rate = (abs(d_alpha_sg(a)) * sigma_sg / (KB * T) + abs(d_alpha_g(a)) * sigma_g / (KB * T)
            + abs(T_T - T_H) * sigma_u / T)
    if rate <= 0.0:  # no fluctuation: the step is unbounded, so the leg's end is next
        return 1.0
    return min(1.0, a + speed / rate)


def adapt_dt(dt, acc):
    """Acceptance > 0.8: +0.125 fs; < 0.1: -0.5 fs; < 0.4: -0.25 fs; kept in [0.1, 5] fs."""
    if acc > 0.8:
        dt += 0.125
    elif acc < 0.1:
        dt -= 0.5
    elif acc < 0.4:
        dt -= 0.25
    return min(5.0, max(0.1, dt))


def insertions(T, alpha, dt, attempts, accepts, threshold=0.4, T_T=300.0, T_H=600.0):
    """Between cycles ("Equilibration and production"): a state goes between every neighbour
    pair (a, a+1) whose exchange acceptance over the cycle is below the threshold (pairs never
    attempted are left alone), at the midpoint of the leg's control parameter (the geometric mean
    temperature on the warming leg, the mean alpha with T(alpha) on the coupling leg) and with the
    smaller time step.  attempts / accepts: neighbour-pair counts [K - 1].  Returns the new
    (T, alpha, dt) and, for each new state, (its index, the index of its lower neighbour)."""
    T, alpha, dt = np.asarray(T, float), np.asarray(alpha, float), np.asarray(dt, float)
    att, acc = np.asarray(attempts, float), np.asarray(accepts, float)
    nT, nA, nD, new = [], [], [], []
    for k in range(T.size):
        nT.append(T[k])
        nA.append(alpha[k])
        nD.append(dt[k])
        if k + 1 < T.size and att[k] > 0 and acc[k] / att[k] < threshold:
            if math.isnan(alpha[k]):
                t, a = math.sqrt(T[k] * T[k + 1]), math.nan
            else:
                a = 0.5 * (alpha[k] + alpha[k + 1])
                t = T_H + (T_T - T_H) * a
            new.append((len(nT), len(nT) - 1))
            nT.append(t)
            nA.append(a)
            nD.append(min(dt[k], dt[k + 1]))
    return np.array(nT), np.array(nA), np.array(nD), new


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
