#!/usr/bin/env python
"""Benchmark of the plain BPMF hot path at paper scale on GB300.

Workload (one GPU): a 48-atom synthetic ligand (seed 2), a 4000-atom receptor, three 129^3 grids at
0.25 A, 32 warming + 96 coupling states, 64 independent chains (8192 replicas).  One step = one HMC
trial of 50 velocity-Verlet steps for every replica, 25 replica-exchange sweeps on each of the 128
ladders, and the u_kn of the step's snapshot (every replica at every state of its leg, from the
energy components of the trial's final evaluation).  Metric: ligand atom-force
evaluations per second (replicas x atoms x VV steps / time).  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ligand atom-force evals/s"
N_STATES_BC, N_STATES_CD, N_CHAINS, N_VV = 32, 96, 64, 50
FP32_LANES_PER_SM = 128


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--clocks-csv", default=None,
                   help="keep the nvidia-smi samples of the timed region in this file (default: a temporary file)")
    p.add_argument("--no-mbar", action="store_true")
    p.add_argument("--no-learned", action="store_true")
    p.add_argument("--no-fep", action="store_true", help="skip the end-point (f_DE) measurement")
    p.add_argument("--fep-only", action="store_true", help="only the end-point (f_DE) measurement, after warm-up")
    p.add_argument("--no-batch", action="store_true", help="skip the multi-ligand batch measurement")
    p.add_argument("--batch-only", action="store_true", help="only the multi-ligand batch measurement")
    p.add_argument("--no-bpmf", action="store_true", help="skip the BPMF effective-samples comparison")
    p.add_argument("--no-protocol", action="store_true", help="skip the protocol-initialization measurement")
    p.add_argument("--protocol-only", action="store_true",
                   help="set up the workload and run only the protocol-initialization measurement")
    p.add_argument("--bpmf-only", action="store_true",
                   help="set up the workload and run only the BPMF effective-samples comparison")
    p.add_argument("--paper-cycles", type=int, default=8000)
    p.add_argument("--learned-cycles", type=int, default=8000)
    p.add_argument("--bpmf-window", type=int, default=1000)
    p.add_argument("--learned-only", action="store_true",
                   help="set up the workload and run only the learned-vs-plain comparison (for profiling)")
    return p.parse_args()


def workload():
    from paper_1507_03703_gb300 import synthetic as S
    sys_ = S.config_paper_scale(2)
    return sys_


def workload_config(sys_, n_gpus):
    lig = sys_.ligand
    return {"workload": "plain BPMF hot path, paper scale",
            "ligand_atoms": lig.n_atoms, "receptor_atoms": sys_.receptor.n_atoms,
            "grid": "3 x 129^3 at 0.25 A (+2 soft)", "states": N_STATES_BC + N_STATES_CD,
            "chains_per_gpu": N_CHAINS, "replicas_per_gpu": N_CHAINS * (N_STATES_BC + N_STATES_CD),
            "vv_steps": N_VV, "exchange_sweeps": 25, "max_sep": 5, "parallelism": "chains sharded, dp%d" % n_gpus,
            "l2": "flushed between steps (256 MB write); steps timed individually"}


def flops_per_replica_eval(lig):
    """Algorithmic FP32 work of one force evaluation of one replica (the roofline's unit):
    26 per unique nonbonded pair (LJ + Coulomb energy and force on both atoms), 20 per bond,
    60 per angle, 100 per torsion, 170 per atom for the five interpolated channels and 12 per
    atom for the velocity-Verlet update."""
    na = lig.n_atoms
    nbr = [[] for _ in range(na)]
    for a, b in lig.bonds:
        nbr[a].append(b)
        nbr[b].append(a)
    n_pairs = 0
    for i in range(na):
        dist = {i: 0}
        frontier = [i]
        for d in (1, 2):
            nxt = []
            for u in frontier:
                for v in nbr[u]:
                    if v not in dist:
                        dist[v] = d
                        nxt.append(v)
            frontier = nxt
        n_pairs += sum(1 for j in range(i + 1, na) if j not in dist)
    return 26 * n_pairs + 20 * len(lig.bonds) + 60 * len(lig.angles) + 100 * len(lig.torsions) + 182 * na


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index, path=None):
        self.index = index
        self.proc = None
        self.keep = path is not None
        if path is None:
            import tempfile
            fd, path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
        self.path = path

    def start(self):
        try:
            if os.path.dirname(self.path):
                os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        try:
            return self._summary()
        finally:
            if not self.keep and os.path.exists(self.path):
                os.remove(self.path)

    def _summary(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            w = [t.strip() for t in line.split(",")]
            if len(w) < 9:
                continue
            try:
                sm.append(float(w[1]))
                mx = float(w[2])
            except ValueError:
                continue
            for n, v in zip(names, w[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def mbar_seconds_per_iteration(ctx, u, N_k, mode, stream, short=4, long=14):
    """Seconds per MBAR iteration: two solves stopped after short and long iterations (tolerance
    zero, so neither stops on its own unless the iterates stop changing), timed with CUDA events,
    the time difference over the difference of the iterations each solve reports.  The
    difference cancels the per-solve setup (the shift of mode 2, the first launches)."""
    import torch
    ctx.mbar(u, N_k, tol=1e-300, max_iter=2, precision_mode=mode, raise_on_nonconvergence=False)
    t, it = {}, {}
    for m in (short, long):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        _, n_it = ctx.mbar(u, N_k, tol=1e-300, max_iter=m, precision_mode=mode, raise_on_nonconvergence=False)
        it[m] = m if n_it < 0 else n_it  # -1: stopped at max_iter, not converged
        e1.record(stream)
        torch.cuda.synchronize()
        t[m] = e0.elapsed_time(e1) * 1e-3
    if it[long] <= it[short]:
        raise RuntimeError("MBAR stopped before %d iterations; cannot time an iteration" % long)
    return (t[long] - t[short]) / (it[long] - it[short])


def mbar_hbm_roofline(ctx, dev, K=256, n_per=3907, short=4, long=14):
    """MBAR precision mode 2 against HBM at the precision study's size (K = 256 harmonic wells in
    2-D, about 1e6 exact samples built on the device, u_kn of 2 GB in FP64, 1 GB as the shifted
    FP32 copy): each iteration reads the FP32 u_kn twice (2 K N 4 bytes) and writes and reads the
    log denominators (2 N 4 bytes).  Seconds per iteration from two solves of fixed lengths, timed
    with CUDA events on the context's stream (the difference cancels the shift and the setup)."""
    import torch
    g = torch.Generator(device=dev).manual_seed(31)
    bk = torch.rand(K, device=dev, dtype=torch.float64, generator=g) * 3.5 + 0.5
    mu = torch.rand((K, 2), device=dev, dtype=torch.float64, generator=g) * 0.6 - 0.3
    x = (mu[:, None, :] + torch.randn((K, n_per, 2), device=dev, dtype=torch.float64, generator=g)
         / torch.sqrt(bk)[:, None, None]).reshape(-1, 2)
    N = x.shape[0]
    u = torch.empty((K, N), device=dev, dtype=torch.float64)
    for k in range(K):
        u[k] = 0.5 * bk[k] * ((x - mu[k]) ** 2).sum(-1)
    N_k = np.full(K, n_per, dtype=np.int64)
    per_it = mbar_seconds_per_iteration(ctx, u, N_k, 2, torch.cuda.current_stream(dev), short, long)
    bytes_it = 2.0 * K * N * 4 + 2.0 * N * 4
    peak = measured_peaks().get("hbm_gbs")
    achieved = bytes_it / per_it / 1e9
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak if peak else None, "kernel": "MBAR iteration, precision mode 2",
           "workload": "K = %d, N = %d" % (K, N), "ms_per_iteration": per_it * 1e3,
           "bytes_per_iteration": bytes_it, "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)"}
    del u, x
    torch.cuda.empty_cache()
    return out


def gather_bytes_per_launch(alpha, R_per_state, n_atoms, n_steps):
    """Useful lattice bytes of one HMC launch, 32 B per active grid per atom and evaluation (8
    corners x 4 B): the three full grids (96 B) where the state's FP32 weight alpha_g is nonzero and
    the two soft grids (64 B) where alpha_sg is, in each of the n_steps - 1 force-only evaluations,
    and all five in the two energy evaluations (first and last).  The padding lane of the stored
    full-grid records is not counted.  Weights of Eq. (protocol)."""
    out = 0.0
    for a in alpha:
        if np.isnan(a):
            w_sg = w_g = 0.0
        else:
            s_ = 2.0 * a - 1.0
            z = 1000.0 * (a - 0.5)
            lg = 1.0 / (1.0 + np.exp(-z)) if z >= 0 else np.exp(z) / (1.0 + np.exp(z))
            w_sg, w_g = 1.0 - s_ * s_, s_ * s_ * lg
        gated = 96.0 * (np.float32(w_g) != 0) + 64.0 * (np.float32(w_sg) != 0)
        out += R_per_state * n_atoms * (2 * 160.0 + (n_steps - 1) * gated)
    return out


def gather_peak(ctx, stream, n_cells=8 * 1024 * 1024, reps=5):
    """Measured rate of random 8-corner gathers from both loaded lattices, in the useful bytes of
    gather_bytes_per_launch (160 B per cell: five grids x 8 corners x 4 B)."""
    import torch
    sink = ctx.gather_probe(n_cells, soft=True, seed=1)
    ms = []
    for r in range(reps + 2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.gather_probe(n_cells, soft=True, seed=2 + r, sink=sink)
        e1.record(stream)
        torch.cuda.synchronize()
        if r >= 2:
            ms.append(e0.elapsed_time(e1))
    return n_cells * 160.0 / (float(np.median(ms)) * 1e-3) / 1e9


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# DRAM bytes (read + write) and warp instructions per launch of a kernel from one ncu capture of
# the bench command, with a fingerprint of the sources the kernel was built from at the time: the
# figures are reported only while those sources are unchanged.
NCU_TRAFFIC = {
    "hmc_kernel": {"bytes_per_launch": 11305984, "warp_instructions_per_launch": 1310285150,
                   "sources": ("hmc.cu", "internal.cuh", "grids.cu"),
                   "sha256": "4534b47f86cbe5ae0b75a683b4845996a3f3f4ea7aad13c7c2c1e305a693bec0"},
}


def captured_traffic(kernel, field="bytes_per_launch"):
    """A per-launch figure of `kernel` from its ncu capture (DRAM bytes by default), or None if its
    sources changed."""
    import hashlib
    rec = NCU_TRAFFIC.get(kernel)
    if rec is None:
        return None
    h = hashlib.sha256()
    for f in rec["sources"]:
        with open(os.path.join(ROOT, "paper_1507_03703_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return rec.get(field) if h.hexdigest() == rec["sha256"] else None


def learned_vs_plain(ctx, sys_, stream, dev, chains=2048, burn=20, data_cycles=489, train_iter=500, cmp_cycles=200,
                     n_moves=4, lag=1, mixed=True, seed=7, target=N_STATES_BC, n_torsions=-1):
    """Effective samples per second at one state of plain HMC and of HMC plus learned proposals,
    after training the proposal on the plain run's own samples: moves between random pairs of
    samples (lag None), between poses of the same chain `lag` cycles apart, or (mixed) as many of
    each, so that the mixture learns both long jumps and local moves.  The default state
    is the decoupled end of the coupling leg (alpha = 0, 600 K), where the paper applies its own
    external-coordinate moves.  ESS: sum over chains of N / g of the Psi_g series."""
    import torch

    from paper_1507_03703_gb300 import synthetic as S
    from paper_1507_03703_gb300.learned import LearnedProposal
    from paper_1507_03703_gb300.sampler import effective_samples
    lig = sys_.ligand
    base = S.place_ligand(lig, sys_.receptor, sys_.site, 128, seed=seed, n_tries=8).astype(np.float32)
    x = torch.from_numpy(base[np.arange(chains) % 128]).to(dev)
    comps = torch.empty((chains, 4), dtype=torch.float64, device=dev)
    st = torch.full((chains,), target, dtype=torch.int32, device=dev)
    ctx.reduced_energies(chains, x=x, comps=comps)
    xs, cs = [], []
    for cyc in range(burn + data_cycles):
        ctx.hmc_cycle(st, x, comps, n_steps=N_VV, seed=seed, cycle=cyc)
        if cyc >= burn:
            xs.append(x.clone())
            cs.append(comps.clone())
    X = torch.cat(xs)
    Cm = torch.cat(cs)
    lp = LearnedProposal(ctx, seed=seed, n_torsions=n_torsions)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    pairs = None
    if lag is not None:
        t_idx = np.arange(data_cycles - lag)
        I = (t_idx[:, None] * chains + np.arange(chains)[None, :]).ravel()
        pairs = (I, I + lag * chains)
        if mixed:  # as many random pairs again, so the mixture learns long jumps and local moves
            rng_p = np.random.default_rng(seed)
            S_ = data_cycles * chains
            pairs = (np.concatenate([I, rng_p.integers(0, S_, size=I.size)]),
                     np.concatenate([I + lag * chains, rng_p.integers(0, S_, size=I.size)]))
    losses = lp.train(X, Cm, target, n_iter=train_iter, batch=4096, lr=1e-3, seed=seed, pairs=pairs)
    ev[1].record(stream)
    torch.cuda.synchronize()
    train_ms = ev[0].elapsed_time(ev[1])
    x0, c0 = x.clone(), comps.clone()
    st_tab = np.concatenate([[(l.T[k], l.alpha[k]) for k in range(l.K)] for l in sys_.legs])
    out = {"state": "index %d: T %.0f K, alpha %s" % (target, st_tab[target][0], st_tab[target][1]),
           "chains": chains, "training_poses": int(X.shape[0]), "train_iters": train_iter, "train_ms": train_ms,
           "loss_first": losses[0], "loss_last": losses[-1], "moves_per_cycle": n_moves,
           "moved_torsions": lp.T,
           "training_pairs": ("random pairs" if lag is None else
                              ("half random pairs, half the same chain %d cycles apart" % lag if mixed
                               else "same chain, %d cycles apart" % lag))}
    for mode in ("plain", "learned"):
        x.copy_(x0)
        comps.copy_(c0)
        acc = torch.zeros(chains, dtype=torch.int32, device=dev)
        series = []
        t = 0.0
        for cyc in range(cmp_cycles):
            ev[0].record(stream)
            ctx.hmc_cycle(st, x, comps, n_steps=N_VV, seed=seed + 1, cycle=1000 + cyc)
            if mode == "learned":
                lp.propose(st, x, comps, n_moves, seed=seed + 2, cycle=cyc, accepted=acc)
            ev[1].record(stream)
            series.append(comps[:, 3].clone())
            torch.cuda.synchronize()
            t += ev[0].elapsed_time(ev[1])
        ess = effective_samples(ctx, torch.stack(series))
        out[mode] = {"ess": ess, "ms": t, "ess_per_s": ess / (t * 1e-3)}
        if mode == "learned":
            out[mode]["move_acceptance"] = float(acc.sum().item()) / (chains * cmp_cycles * n_moves)
    out["ess_per_s_ratio"] = out["learned"]["ess_per_s"] / out["plain"]["ess_per_s"]
    return out


def _target_psi_g(run, li, k_local):
    """Psi_g of the configuration at state k_local of leg li, one value per chain."""
    import torch
    leg = run.legs[li]
    sl = run.leg_slice(li)
    st = run.state_of[sl].view(run.C, leg.K)
    slot = (st == leg.state_offset + k_local).int().argmax(dim=1)
    return run.comps[sl].view(run.C, leg.K, 4)[torch.arange(run.C, device=st.device), slot, 3].clone()


BPMF_REFERENCE = os.path.join(ROOT, "bpmf_reference.json")


def bpmf_reference():
    """The converged BPMF of the paper-scale workload from bpmf_reference.json (written by
    bpmf_reference.py from independent long realizations of both iterations), or None."""
    try:
        return json.load(open(BPMF_REFERENCE))
    except Exception:
        return None


def bpmf_warm(ctx, sys_, seed, warm=200, n_external=20, train_iter=300):
    """The common start of the BPMF study's arms: `warm` cycles of the paper's iteration from seeded
    placements (both legs, 64 chains x 128 states), and a learned proposal (rigid-body moves)
    trained on that run's poses at every state.  Returns (run, proposal, training summary)."""
    import torch

    from paper_1507_03703_gb300 import synthetic as S
    from paper_1507_03703_gb300.learned import LearnedProposal
    from paper_1507_03703_gb300.sampler import Leg, ReplicaExchange
    legs = [Leg(N_STATES_BC, 0), Leg(N_STATES_CD, N_STATES_BC)]
    R = N_CHAINS * (N_STATES_BC + N_STATES_CD)
    base = S.place_ligand(sys_.ligand, sys_.receptor, sys_.site, 128, seed=seed, n_tries=8).astype(np.float32)
    pre = ReplicaExchange(ctx, legs, N_CHAINS, base[np.arange(R) % base.shape[0]], seed=seed, n_external=n_external)
    ctx.reduced_energies(R, x=pre.x, comps=pre.comps)
    xs, cs, ss = [], [], []
    for cyc in range(warm):
        pre.cycle(cyc, N_VV)
        if cyc >= warm // 2 and cyc % 10 == 0:
            xs.append(pre.x.clone())
            cs.append(pre.comps.clone())
            ss.append(pre.state_of.clone())
    lp = LearnedProposal(ctx, seed=seed, n_torsions=0)
    losses = lp.train(torch.cat(xs), torch.cat(cs), torch.cat(ss).cpu().numpy(), n_iter=train_iter, seed=seed)
    return pre, lp, {"poses": int(sum(x.shape[0] for x in xs)), "iters": train_iter, "loss_first": losses[0],
                     "loss_last": losses[-1]}


def bpmf_arm(ctx, stream, dev, pre, lp, n_cyc, window, seed, n_external=20, n_learned=4):
    """One arm from the warm state: the paper's iteration (lp None: an HMC move and the
    external-coordinate moves at alpha < 0.01 per replica, then 25 exchange sweeps) or the same plus
    n_learned learned moves per replica.  Every `window` cycles: the window's BPMF (MBAR per leg
    over snapshots every 10 cycles), the effective samples of the Psi_g series at the target state
    (alpha = 1, 300 K) per chain (N / g from the library's estimator) and the GPU time."""
    import torch

    from paper_1507_03703_gb300.sampler import ReplicaExchange, bpmf_kT, effective_samples
    legs = pre.legs
    R = pre.R
    run = ReplicaExchange(ctx, legs, N_CHAINS, pre.x.cpu().numpy(), seed=seed, n_external=n_external)
    run.comps.copy_(pre.comps)
    run.state_of.copy_(pre.state_of)
    for li in range(len(legs)):
        run.config_of[li].copy_(pre.config_of[li])
    acc = torch.zeros(R, dtype=torch.int32, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    wins, series, full, ms = [], [], [], 0.0
    torch.cuda.synchronize()
    ev[0].record(stream)
    for cyc in range(n_cyc):
        run.hmc(cyc, N_VV)
        run.external(cyc)
        if lp is not None:
            lp.propose(run.state_of, run.x, run.comps, n_learned, seed=seed + 1, cycle=cyc, accepted=acc)
        run.exchange(cyc)
        if cyc % 10 == 0:
            run.history.append(run.comps.clone())
        series.append(_target_psi_g(run, 1, N_STATES_CD - 1))
        full.append(series[-1])
        if (cyc + 1) % window == 0:
            ev[1].record(stream)
            torch.cuda.synchronize()
            w_ms = ev[0].elapsed_time(ev[1])
            ms += w_ms
            S_ = torch.stack(series)
            g, _, _ = ctx.detect_equilibration(S_, n_cand=1)
            ess_chain = (S_.shape[0] / g[:, 0]).cpu().numpy()
            f = [run.free_energies(li, max_iter=20000)[0] for li in range(len(legs))]
            run.history = []
            wins.append({"cycles": cyc + 1, "bpmf_kT": float(bpmf_kT(f[0], f[1])), "ess": float(ess_chain.sum()),
                         "ess_chain": ess_chain.tolist(), "gpu_ms": w_ms})
            series = []
            ev[0].record(stream)
    _, t0s, neffs = ctx.detect_equilibration(torch.stack(full), stride=max(1, n_cyc // 40))
    out = {"cycles": n_cyc, "gpu_ms_per_cycle": ms / max(1, n_cyc), "windows": wins,
           "equilibration_cycles_median": float(t0s.double().median().item()),
           "n_eff_after_equilibration": float(neffs.sum().item()),
           "external_acceptance": float(run.ext_acc.sum().item()) / max(1, n_external * n_cyc * N_CHAINS)}
    if lp is not None:
        out["learned_acceptance"] = float(acc.sum().item()) / (R * n_learned * n_cyc)
    return out


def in_band_from(windows, b_ref, criterion):
    """Index of the first window from which every later window's BPMF stays within `criterion` of
    b_ref (None if the last window is outside)."""
    first = None
    for i in range(len(windows) - 1, -1, -1):
        if abs(windows[i]["bpmf_kT"] - b_ref) <= criterion:
            first = i
        else:
            break
    return first


def bpmf_convergence(ctx, sys_, stream, dev, paper_cycles=8000, learned_cycles=8000, window=1000, warm=200,
                     n_external=20, n_learned=4, train_iter=300, seed=11, criterion=0.2, n_boot=2000):
    """BPMF effective samples per second of the paper's iteration and of the same plus learned
    moves, at the criterion of `criterion` kT from the reference BPMF of bpmf_reference.json.  An
    arm is credited only with the windows from the last entry into the band on, and only if it stays
    there to the end.  The learned/plain ratio comes with a 95 % bootstrap interval over chains (the
    per-chain effective samples of the credited windows resampled)."""
    pre, lp, training = bpmf_warm(ctx, sys_, seed, warm, n_external, train_iter)
    out = {"workload": "both legs, %d chains x %d states, %d VV steps" % (N_CHAINS, N_STATES_BC + N_STATES_CD, N_VV),
           "target_state": "alpha = 1, 300 K", "warm_cycles": warm, "window_cycles": window,
           "criterion_kT": criterion, "learned_training": training}
    ref = bpmf_reference()
    if ref is None:
        out["reference"] = None
        out["note"] = "no bpmf_reference.json: no arm is credited"
    else:
        out["reference"] = {k: ref[k] for k in ("bpmf_kT", "spread_kT", "sem_kT", "realizations", "source")}
    arms = {"paper": bpmf_arm(ctx, stream, dev, pre, None, paper_cycles, window, seed + 1, n_external, n_learned),
            "learned": bpmf_arm(ctx, stream, dev, pre, lp, learned_cycles, window, seed + 1, n_external, n_learned)}
    rng = np.random.default_rng(seed)
    boot = {}
    for name, a in arms.items():
        a["final_bpmf_kT"] = a["windows"][-1]["bpmf_kT"] if a["windows"] else None
        first = in_band_from(a["windows"], ref["bpmf_kT"], criterion) if ref else None
        if first is None:
            a["credited_from_cycles"] = None
            a["bpmf_eff_samples_per_s"] = 0.0
        else:
            done = a["windows"][first:]
            a["credited_from_cycles"] = a["windows"][first]["cycles"] - window
            gpu_s = sum(w["gpu_ms"] for w in done) * 1e-3
            per_chain = np.sum([w["ess_chain"] for w in done], axis=0)
            a["bpmf_eff_samples_per_s"] = float(per_chain.sum() / gpu_s)
            idx = rng.integers(0, per_chain.size, size=(n_boot, per_chain.size))
            boot[name] = per_chain[idx].sum(axis=1) / gpu_s
        if ref:
            a["final_abs_err_kT"] = abs(a["final_bpmf_kT"] - ref["bpmf_kT"])
        for w in a["windows"]:
            w.pop("ess_chain")
        out[name] = a
    if "paper" in boot and "learned" in boot:
        r = boot["learned"] / boot["paper"]
        out["learned_vs_paper"] = {"ratio": arms["learned"]["bpmf_eff_samples_per_s"] /
                                            arms["paper"]["bpmf_eff_samples_per_s"],
                                   "ci95": [float(np.percentile(r, 2.5)), float(np.percentile(r, 97.5))]}
    else:
        out["learned_vs_paper"] = {"ratio": None, "note": "an arm is not within the criterion at its end: "
                                                           "no ratio"}
    return out


def protocol_build(ctx, sys_, stream, n_seeds=50, seed=21):
    """Protocol initialization ("Initialization") of both legs for the paper-scale ligand with the
    paper's settings: 50 seeds, 2000 steps (40 HMC trials of 50 steps) per state and attempt,
    speeds s_bc = 20 and s_cd = 0.2, time steps adapted into [0.1, 5] fs.  The seeds of both legs
    are placements of the ligand in the binding site (the coupling leg starts unbound, at alpha = 0
    and 600 K)."""
    import torch

    from paper_1507_03703_gb300 import synthetic as S
    from paper_1507_03703_gb300.protocol import ProtocolBuilder
    lig = sys_.ligand
    seeds = S.place_ligand(lig, sys_.receptor, sys_.site, n_seeds, seed=seed, n_tries=8).astype(np.float32)
    out = {}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for leg in ("bc", "cd"):
        pb = ProtocolBuilder(ctx)
        torch.cuda.synchronize()
        t = time.perf_counter()
        ev[0].record(stream)
        r = pb.build_leg(leg, seeds, seed=seed)
        ev[1].record(stream)
        torch.cuda.synchronize()
        out[leg] = {"states": int(len(r["T"])), "wall_s": time.perf_counter() - t,
                    "gpu_s": ev[0].elapsed_time(ev[1]) * 1e-3, "hmc_trials": r["hmc_trials"],
                    "final_speed": r["speed"], "pacc_min": float(r["pacc"].min()) if len(r["pacc"]) else None,
                    "pacc_mean": float(r["pacc"].mean()) if len(r["pacc"]) else None,
                    "dt_fs_min": float(r["dt"].min()), "dt_fs_max": float(r["dt"].max()),
                    "acceptance_mean": float(r["acceptance"].mean())}
        if leg == "bc":
            out[leg]["T_K"] = [round(float(v), 1) for v in r["T"]]
        else:
            out[leg]["alpha_first"] = [round(float(v), 4) for v in r["alpha"][:8]]
    return out


def padded_ligand(lig, n, site):
    """The ligand padded to n atoms with inert atoms: no charge, no Lennard-Jones well, no bonded
    term, a mass of 1e9 amu (they stay where they are put) at distinct points of a 1 A lattice
    around the site.  Every pair and grid term of an n-atom ligand is evaluated; the real atoms'
    forces are unchanged except for the restraint (the heavy atoms hold the centre of mass at the
    site), which is immaterial to throughput."""
    from paper_1507_03703_gb300 import synthetic as S
    k = n - lig.n_atoms
    side = int(np.ceil(k ** (1.0 / 3.0))) if k > 0 else 1
    g = np.stack(np.meshgrid(*[np.arange(side)] * 3, indexing="ij"), -1).reshape(-1, 3)[:k]
    pad = g - 0.5 * (side - 1) + 0.25
    return S.Ligand(mass=np.concatenate([lig.mass, np.full(k, 1e9)]), charge=np.concatenate([lig.charge, np.zeros(k)]),
                    rstar=np.concatenate([lig.rstar, np.full(k, 1.5)]), eps=np.concatenate([lig.eps, np.zeros(k)]),
                    bonds=lig.bonds, bond_k=lig.bond_k, bond_r0=lig.bond_r0, angles=lig.angles, angle_k=lig.angle_k,
                    angle_theta0=lig.angle_theta0, torsions=lig.torsions, torsion_V=lig.torsion_V,
                    torsion_gamma=lig.torsion_gamma, x0=np.concatenate([lig.x0, pad + np.asarray(site)]))


def batching(dev, stream, steps=10, warmup=3, seed=3):
    """Many ligands in one launch per atoms-per-lane class: 256 ligands of U[10, 70] atoms, 64
    states each (16 BC + 48 CD), one chain each (16384 replicas), 50 VV steps, against one
    129^3 x 3 grid set.  Ligand atom-force evals/s (real atoms) of the HMC launches with the
    default shapes, the autotuned shapes, the uniform layout (every replica in the 65-96-atom
    shape) and the padded-uniform baseline (every ligand padded to 70 atoms, uniform shape); then a
    whole cycle (HMC + exchange on both legs) captured as one CUDA graph, replayed, against the
    same cycle launched eagerly.  L2 is flushed between timed launches."""
    import torch
    from paper_1507_03703_gb300 import algdock
    from paper_1507_03703_gb300 import synthetic as S
    from paper_1507_03703_gb300.algdock import Context
    from paper_1507_03703_gb300.sampler import Leg, ReplicaExchange
    sys_, ligs = S.config_batch(seed)
    T = np.concatenate([l.T for l in sys_.legs])
    alpha = np.concatenate([l.alpha for l in sys_.legs])
    dt = np.concatenate([l.dt_fs for l in sys_.legs])
    ctx = Context(dev.index or 0)
    ctx.set_stream(stream)
    nx, ny, nz = sys_.grid.n
    raw = [torch.empty((nz, ny, nx), dtype=torch.float32, device=dev) for _ in range(3)]
    ctx.grids_build(sys_.grid, sys_.receptor, *raw)
    ctx.grids_load(sys_.grid, *raw, vmax_e=min(algdock.soft_elec_cap(l) for l in ligs))
    del raw
    ctx.states_set(T, alpha, dt)
    ctx.batch_load(ligs, sys_.site)
    L, stride = len(ligs), max(l.n_atoms for l in ligs)
    legs = [Leg(sys_.legs[0].K, 0), Leg(sys_.legs[1].K, sys_.legs[0].K)]
    Ktot = sum(l.K for l in legs)
    # one placement per ligand and state slot (4 placements per ligand, reused)
    place = [S.place_ligand(l, sys_.receptor, sys_.site, 4, seed=50 + i, n_tries=8) for i, l in enumerate(ligs)]
    x0 = np.zeros((L * Ktot, stride, 3), dtype=np.float32)
    b = 0
    for leg in legs:
        for c in range(L):
            for k in range(leg.K):
                x0[b + c * leg.K + k, :ligs[c].n_atoms] = place[c][k % 4]
        b += L * leg.K
    run = ReplicaExchange(ctx, legs, L, x0, seed=4321, batched=True)
    lig_of = run.lig_of()
    ctx.batch_layout(lig_of, stride)
    evals = float(sum(ligs[c].n_atoms for c in lig_of)) * N_VV
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def time_hmc(tag, first):
        for w in range(warmup):
            run.hmc(first + w, N_VV)
        ms = []
        for s_ in range(steps):
            flush.fill_(float(s_))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run.hmc(first + warmup + s_, N_VV)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        m = float(np.median(ms))
        return {"ms_per_launch": m, "evals_per_s": evals / (m * 1e-3)}

    out = {"workload": "%d ligands of %d-%d atoms (mean %.1f), %d states each, 1 chain, %d VV steps, 129^3 x 3 grids"
                       % (L, min(l.n_atoms for l in ligs), stride, np.mean([l.n_atoms for l in ligs]), Ktot, N_VV),
           "replicas": int(len(lig_of)), "ligands_per_atoms_per_lane": [int(sum(1 for l in ligs if (l.n_atoms + 31) // 32 == k))
                                                        for k in (1, 2, 3)]}
    out["default"] = time_hmc("default", 0)
    chosen, tms = ctx.batch_tune(run.state_of, run.x, n_steps=N_VV, n_timed=5)
    out["tuned_shapes"] = [{"class": k, "replicas_per_block": w, "pair_table": t} for k, (w, t) in enumerate(chosen)]
    out["tuner_ms_per_launch"] = tms
    out["tuned"] = time_hmc("tuned", 100)
    ctx.batch_layout(lig_of, stride, uniform=True)
    out["uniform"] = time_hmc("uniform", 200)
    out["tuned_vs_uniform"] = out["tuned"]["evals_per_s"] / out["uniform"]["evals_per_s"]
    # padded-uniform: every ligand padded to the largest size with inert atoms, one shape for all
    x_real = run.x.clone()
    padded = [padded_ligand(l, stride, sys_.site) for l in ligs]
    ctx.batch_load(padded, sys_.site)
    ctx.batch_layout(lig_of, stride, uniform=True)
    xp = x_real.cpu().numpy()
    for r, c in enumerate(lig_of):
        xp[r, ligs[c].n_atoms:] = padded[c].x0[ligs[c].n_atoms:]
    run.x.copy_(torch.from_numpy(xp))
    out["padded_uniform"] = time_hmc("padded", 250)
    out["padded_uniform"]["acceptance"] = float(run.acc.float().mean().item())
    out["tuned_vs_padded_uniform"] = out["tuned"]["evals_per_s"] / out["padded_uniform"]["evals_per_s"]
    ctx.batch_load(ligs, sys_.site)
    run.x.copy_(x_real)
    ctx.batch_layout(lig_of, stride)
    ctx.batch_tune(run.state_of, run.x, n_steps=N_VV, n_timed=5)
    # the whole cycle, eager and as one graph, timed in alternation (three rounds of 10 cycles
    # each) so that both arms run on the same evolving configurations
    for w in range(warmup):
        run.hmc(300 + w, N_VV)
        run.exchange(300 + w)
    g = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream(device=dev)
    cap.wait_stream(stream)
    with torch.cuda.stream(cap):
        ctx.set_stream(cap)
        try:
            with torch.cuda.graph(g, stream=cap, capture_error_mode="relaxed"):
                run.hmc(500, N_VV)
                run.exchange(500)
        finally:
            ctx.set_stream(stream)
    stream.wait_stream(cap)
    for w in range(warmup):
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    eager, graph = [], []
    for rnd in range(3):
        e0.record(stream)
        for s_ in range(steps):
            run.hmc(400 + 100 * rnd + s_, N_VV)
            run.exchange(400 + 100 * rnd + s_)
        e1.record(stream)
        torch.cuda.synchronize()
        eager.append(e0.elapsed_time(e1) / steps)
        e0.record(stream)
        for s_ in range(steps):
            g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        graph.append(e0.elapsed_time(e1) / steps)
    eager_ms, graph_ms = float(np.median(eager)), float(np.median(graph))
    out["cycle_eager_ms"] = eager_ms
    out["cycle_graph_ms"] = graph_ms
    out["cycle_graph_evals_per_s"] = evals / (graph_ms * 1e-3)
    out["hmc_acceptance"] = float(run.acc.float().mean().item())
    return out


FLOPS_PER_TARGET_PAIR = 18  # 3 differences, r^2 (3 mul + 2 add), 1 reciprocal, 3 powers, 3 multiply-adds


def fep_endpoint(ctx, run, sys_, stream, sm_max, n_samples=16384, first_cycle=30_000):
    """f_DE ("Estimation": Zwanzig perturbation of milestone D samples into the target force field,
    whose receptor-ligand energies are computed directly).  The configuration at milestone D
    (alpha = 1, 300 K) of every chain is taken each cycle until n_samples are gathered; then the
    target interaction (one launch over all samples) and the FEP reduction are timed with CUDA
    events on the launching stream."""
    import torch
    lig, rec = sys_.ligand, sys_.receptor
    ctx.receptor_load(rec)
    kD = N_STATES_BC + N_STATES_CD - 1
    dev = run.x.device
    xs = torch.empty((n_samples, lig.n_atoms, 3), dtype=torch.float32, device=dev)
    psi_g = torch.empty(n_samples, dtype=torch.float64, device=dev)
    filled, cyc = 0, first_cycle
    while filled < n_samples:
        run.cycle(cyc, N_VV)
        slots = torch.nonzero(run.state_of == kD).flatten()
        take = min(int(slots.numel()), n_samples - filled)
        xs[filled:filled + take] = run.x[slots[:take]]
        psi_g[filled:filled + take] = run.comps[slots[:take], 3]
        filled += take
        cyc += 1
    psi_t = torch.empty(n_samples, dtype=torch.float64, device=dev)
    beta = 1.0 / (0.0019872043 * 300.0)
    for _ in range(3):
        ctx.target_interaction(xs, psi_t)
        ctx.fep(psi_t, psi_g, beta=beta)
    torch.cuda.synchronize()
    ti, fe = [], []
    for _ in range(10):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        ctx.target_interaction(xs, psi_t)
        e[1].record(stream)
        r = ctx.fep(psi_t, psi_g, beta=beta)
        e[2].record(stream)
        torch.cuda.synchronize()
        ti.append(e[0].elapsed_time(e[1]))
        fe.append(e[1].elapsed_time(e[2]))
    ti_ms, fe_ms = float(np.median(ti)), float(np.median(fe))
    pairs = n_samples * lig.n_atoms * rec.n_atoms
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak = n_sm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = pairs * FLOPS_PER_TARGET_PAIR / (ti_ms * 1e-3) / 1e12
    return {"samples": n_samples, "milestone": "D (alpha = 1, 300 K)", "f_DE_kT": r["f"], "sigma_kT": r["sigma"],
            "n_eff": r["n_eff"], "min_target_interaction_kcal": float(psi_t.min().item()),
            "target_interaction_ms": ti_ms, "fep_reduction_ms_incl_result_copy": fe_ms, "pairs_per_s": pairs / (ti_ms * 1e-3),
            "configurations_per_s": n_samples / ((ti_ms + fe_ms) * 1e-3),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "kernel": "target_interaction_kernel",
                         "traffic": None, "traffic_ncu_summary": "profiles/target_interaction_paper_scale.md",
                         "flops_per_launch": pairs * FLOPS_PER_TARGET_PAIR,
                         "peak_source": "%d SMs x 128 FP32 lanes x 2 x %.0f MHz (derived)" % (n_sm, sm_max)}}


def oracle_cpu_baseline(sys_, n_rep=65536, n_threads=0):
    """The FP64 oracle as it stands on this host's cores: one HMC trial of 50 VV steps for a
    bounded sample of replicas spread over all states (about 10-30 s on a 16-core host)."""
    import oracle
    T = np.concatenate([l.T for l in sys_.legs])
    alpha = np.concatenate([l.alpha for l in sys_.legs])
    dt = np.concatenate([l.dt_fs for l in sys_.legs])
    ljr, lja, elec = oracle.grid_direct_sum(sys_.receptor, sys_.grid)
    osys = oracle.OracleSystem(sys_.grid, ljr, lja, elec, sys_.ligand, T, alpha, dt, site=sys_.site)
    from paper_1507_03703_gb300 import synthetic as S
    base = S.place_ligand(sys_.ligand, sys_.receptor, sys_.site, 64, seed=9, n_tries=4).astype(np.float64)
    x = base[np.arange(n_rep) % base.shape[0]]
    states = (np.arange(n_rep) % len(T)).astype(np.int32)
    t = time.perf_counter()
    _, _, _, _, used = osys.hmc(x, states, N_VV, 1, 0, n_threads=n_threads)
    el = time.perf_counter() - t
    evals = n_rep * sys_.ligand.n_atoms * N_VV
    return {"value": evals / el, "unit": METRIC, "cores": int(used), "kind": "oracle",
            "sample": "%d replicas x 1 HMC trial of %d VV steps (all 128 states), %.1f s" % (n_rep, N_VV, el)}


def run_reference(args):
    """The oracle timed as the reference arm: each step is one bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sys_ = workload()
    import oracle
    T = np.concatenate([l.T for l in sys_.legs])
    alpha = np.concatenate([l.alpha for l in sys_.legs])
    dt = np.concatenate([l.dt_fs for l in sys_.legs])
    ljr, lja, elec = oracle.grid_direct_sum(sys_.receptor, sys_.grid)
    osys = oracle.OracleSystem(sys_.grid, ljr, lja, elec, sys_.ligand, T, alpha, dt, site=sys_.site)
    from paper_1507_03703_gb300 import synthetic as S
    n_rep = 128
    x = S.place_ligand(sys_.ligand, sys_.receptor, sys_.site, n_rep, seed=9, n_tries=4).astype(np.float64)
    states = (np.arange(n_rep) % len(T)).astype(np.int32)
    used = 1
    for w in range(args.warmup):
        x, _, _, _, used = osys.hmc(x, states, N_VV, 1, w)
    t = time.perf_counter()
    for s in range(args.steps):
        x, _, _, _, used = osys.hmc(x, states, N_VV, 1, 1000 + s)
    el = time.perf_counter() - t
    evals = n_rep * sys_.ligand.n_atoms * N_VV * args.steps
    v = evals / el
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "evals/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(sys_, 1), sample="%d replicas per step (all states)" % n_rep),
        "cpu_baseline": {"value": v, "unit": "evals/s", "cores": int(used), "kind": "oracle",
                         "sample": "%d replicas x 1 HMC trial of %d VV steps per step" % (n_rep, N_VV)},
        "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    from paper_1507_03703_gb300 import build as B
    B.build()
    from paper_1507_03703_gb300 import synthetic as S
    from paper_1507_03703_gb300.algdock import Context
    from paper_1507_03703_gb300.ranks import max_over_ranks, shard_per_rank
    from paper_1507_03703_gb300.sampler import Leg, ReplicaExchange

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sys_ = workload()
    lig = sys_.ligand
    T = np.concatenate([l.T for l in sys_.legs])
    alpha = np.concatenate([l.alpha for l in sys_.legs])
    dt = np.concatenate([l.dt_fs for l in sys_.legs])

    stream = torch.cuda.current_stream(dev)
    ctx = Context(local)
    ctx.set_stream(stream)
    nx, ny, nz = sys_.grid.n
    raw = [torch.empty((nz, ny, nx), dtype=torch.float32, device=dev) for _ in range(3)]
    ctx.grids_build(sys_.grid, sys_.receptor, *raw)
    ctx.grids_load(sys_.grid, *raw, ligand=lig)
    ctx.ligand_load(lig, sys_.site)
    ctx.states_set(T, alpha, dt)
    del raw
    legs = [Leg(N_STATES_BC, 0), Leg(N_STATES_CD, N_STATES_BC)]
    R = N_CHAINS * (N_STATES_BC + N_STATES_CD)
    # weak scaling: N_CHAINS chains per rank, numbered globally so that ranks draw disjoint streams
    sh = shard_per_rank(N_CHAINS, world, rank)
    base = S.place_ligand(lig, sys_.receptor, sys_.site, 128, seed=100 + rank, n_tries=8).astype(np.float32)
    x0 = base[np.arange(R) % base.shape[0]]
    run = ReplicaExchange(ctx, legs, N_CHAINS, x0, seed=1000, rep_offset=sh.rep_offset(N_STATES_BC + N_STATES_CD),
                          ladder_offset=sh.ladder_offset(len(legs)))
    u_leg = [torch.empty((l.K, N_CHAINS * l.K), dtype=torch.float64, device=dev) for l in legs]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    snap_stream = torch.cuda.Stream(device=dev)

    def step(cyc, ev=None):
        if ev is not None:
            ev[0].record(stream)
        run.hmc(cyc, N_VV)
        if ev is not None:
            ev[1].record(stream)
        # the snapshot (u_kn per leg from the components the trial's final energy evaluation left)
        # reads only the components, which the exchange does not move: it runs beside the sweeps
        hmc_done = torch.cuda.Event()
        hmc_done.record(stream)
        snap_stream.wait_event(hmc_done)
        ctx.set_stream(snap_stream)
        for li, leg in enumerate(legs):
            sl = run.leg_slice(li)
            ctx.reduced_energies(N_CHAINS * leg.K, comps=run.comps[sl], k_begin=leg.state_offset, k_count=leg.K,
                                 u_kn=u_leg[li])
        snap_done = torch.cuda.Event()
        snap_done.record(snap_stream)
        ctx.set_stream(stream)
        run.exchange(cyc)
        if ev is not None:
            ev[2].record(stream)
        stream.wait_event(snap_done)
        if ev is not None:
            ev[3].record(stream)

    if args.learned_only:
        r = learned_vs_plain(ctx, sys_, stream, dev, target=N_STATES_BC + 28, cmp_cycles=20, train_iter=20)
        print(json.dumps({"learned_vs_plain": r}))
        return
    if args.protocol_only:
        print(json.dumps({"protocol_initialization": protocol_build(ctx, sys_, stream)}))
        return
    if args.bpmf_only:
        r = bpmf_convergence(ctx, sys_, stream, dev, paper_cycles=args.paper_cycles,
                             learned_cycles=args.learned_cycles, window=args.bpmf_window)
        print(json.dumps({"bpmf_eff_samples": r}))
        return
    if args.batch_only:
        print(json.dumps({"batching": batching(dev, stream)}))
        return
    if args.fep_only:
        for w in range(args.warmup):
            step(w)
        print(json.dumps({"fep_endpoint": fep_endpoint(ctx, run, sys_, stream, measured_peaks().get("sm_max_mhz")
                                                       or 2070.0)}))
        return
    launches_per_step = 1 + len(legs) + len(legs)  # hmc, exchange per leg, u_kn per leg
    for w in range(args.warmup):
        step(w)
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    clocks = Clocks(local, args.clocks_csv)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    for s in range(args.steps):
        flush.fill_(float(s))
        step(args.warmup + s, evs[s])
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    hmc_ms = [e[0].elapsed_time(e[1]) for e in evs]
    ex_ms = [e[1].elapsed_time(e[2]) for e in evs]
    ukn_ms = [e[2].elapsed_time(e[3]) for e in evs]
    step_ms = [e[0].elapsed_time(e[3]) for e in evs]
    ms_per_step = sum(step_ms) / args.steps
    ms_per_step = max_over_ranks(ms_per_step, device=dev)
    evals_per_step = world * R * lig.n_atoms * N_VV
    value = evals_per_step / (ms_per_step * 1e-3)

    # roofline of the dominant kernel (the fused HMC trial), FP32 ALU bound
    peaks = measured_peaks()
    sm_max = (clk or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_tflops = n_sm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    # algorithmic work: the measurement plan's 15 N_a + 60 flop per atom evaluation (pairs plus
    # bonded terms), times the atom evaluations of a launch (n_steps + 1 force evaluations)
    fl = (15 * lig.n_atoms + 60) * lig.n_atoms * R * (N_VV + 1)
    fl_detail = flops_per_replica_eval(lig) * R * (N_VV + 1)
    hmc_avg = sum(hmc_ms) / len(hmc_ms)
    achieved = fl / (hmc_avg * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": captured_traffic("hmc_kernel"),
                "traffic_ncu_summary": "profiles/hmc_kernel_paper_scale.md",
                "kernel": "hmc_kernel", "kernel_ms": hmc_avg,
                "peak_source": "%d SMs x 128 FP32 lanes x 2 x %.0f MHz (derived)" % (n_sm, sm_max),
                "flops_per_launch": fl, "flops_rule": "(15 N_a + 60) per atom evaluation",
                "frac_with_term_by_term_count": fl_detail / (hmc_avg * 1e-3) / 1e12 / peak_tflops}

    # the same kernel against the SMs' issue rate (four warp instructions per cycle per SM): the
    # instructions of its ncu capture over the launch time, while the kernel's sources are unchanged
    inst = captured_traffic("hmc_kernel", "warp_instructions_per_launch")
    issue_peak = 4 * n_sm * sm_max * 1e6
    roofline_issue = None
    if inst:
        roofline_issue = {"bound": "issue", "achieved": inst / (hmc_avg * 1e-3), "peak": issue_peak,
                          "unit": "warp instructions/s", "frac": inst / (hmc_avg * 1e-3) / issue_peak,
                          "kernel": "hmc_kernel", "warp_instructions_per_launch": inst,
                          "peak_source": "%d SMs x 4 schedulers x %.0f MHz" % (n_sm, sm_max)}

    # the same kernel against the L2 gather roofline: useful lattice bytes per launch over the
    # measured rate of random 8-corner gathers from the same lattices
    gbytes = gather_bytes_per_launch(alpha, N_CHAINS, lig.n_atoms, N_VV)
    g_peak = gather_peak(ctx, stream)
    g_ach = gbytes / (hmc_avg * 1e-3) / 1e9
    roofline_gather = {"bound": "l2_gather", "achieved": g_ach, "peak": g_peak, "unit": "GB/s",
                       "frac": g_ach / g_peak, "kernel": "hmc_kernel", "useful_bytes_per_launch": gbytes,
                       "peak_source": "random 8-corner cell gathers of both lattices (algdock_gather_probe), "
                                      "measured in this run"}

    # end to end through the C ABI with host buffers: algdock_cycle takes the run's arrays in pinned
    # host memory, copies them in, runs the step (HMC trial, exchange of both legs, snapshot u_kn
    # into a device buffer) and copies them back before it returns
    legs_desc = [(l.K, l.state_offset) for l in legs]
    h_x = run.x.cpu().pin_memory()
    h_c = run.comps.cpu().pin_memory()
    h_s = run.state_of.cpu().pin_memory()
    h_cfg = torch.cat(run.config_of).cpu().pin_memory()
    u_all = torch.empty(sum(l.K * N_CHAINS * l.K for l in legs), dtype=torch.float64, device=dev)
    e2e_steps = max(2, min(args.steps, 10))
    # one untimed call first: the context allocates its staging buffer and side stream on the first
    # call with host arrays
    ctx.cycle(legs_desc, N_CHAINS, 9_999, h_x, h_c, h_s, h_cfg, n_steps=N_VV, seed=run.seed,
              rep_offset=run.rep_offset, ladder_offset=run.ladder_offset, counters=run.counters, u_kn=u_all)
    torch.cuda.synchronize()
    es, ee = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    es.record(stream)
    for s in range(e2e_steps):
        ctx.cycle(legs_desc, N_CHAINS, 10_000 + s, h_x, h_c, h_s, h_cfg, n_steps=N_VV, seed=run.seed,
                  rep_offset=run.rep_offset, ladder_offset=run.ladder_offset, counters=run.counters, u_kn=u_all)
    ee.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(es.elapsed_time(ee) / e2e_steps, device=dev)
    io_bytes = int(h_x.numel() * 4 + h_c.numel() * 8 + h_s.numel() * 4 + h_cfg.numel() * 4)
    e2e = {"value": world * R * lig.n_atoms * N_VV / (e2e_ms * 1e-3), "unit": "evals/s",
           "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes, "call": "algdock_cycle, pinned host arrays"}

    acc = run.counters.cpu().numpy()
    n_trials = R * (args.warmup + args.steps + e2e_steps + 1)  # the counters include the e2e steps
    extra = {}
    if not args.no_mbar and rank == 0:
        # MBAR over K = 128 states and ~1e5 samples recorded from the run
        n_snap = (100_000 + R - 1) // R
        comps_hist = torch.empty((n_snap, R, 4), dtype=torch.float64, device=dev)
        for s in range(n_snap):
            run.cycle(20_000 + s, N_VV)
            comps_hist[s].copy_(run.comps)
        N = n_snap * R
        u = torch.empty((len(T), N), dtype=torch.float64, device=dev)
        ctx.reduced_energies(N, comps=comps_hist.reshape(N, 4), k_begin=0, k_count=len(T), u_kn=u)
        N_k = np.full(len(T), N // len(T), dtype=np.int64)
        for mode, key in ((0, "fp64"), (1, "fp32exp"), (2, "fp32")):
            extra["mbar_%s_iters_per_s" % key] = 1.0 / mbar_seconds_per_iteration(ctx, u, N_k, mode, stream)
        f, it = ctx.mbar(u, N_k, tol=1e-10, max_iter=20000)
        extra["mbar_K"], extra["mbar_N"], extra["mbar_iters_to_1e-10"] = len(T), N, it
        del u, comps_hist
        extra["mbar_roofline"] = mbar_hbm_roofline(ctx, dev)
    if not args.no_fep and rank == 0:
        extra["fep_endpoint"] = fep_endpoint(ctx, run, sys_, stream, sm_max)
    if not args.no_batch and rank == 0 and world == 1:
        extra["batching"] = batching(dev, stream)
    if not args.no_learned and rank == 0:
        # the learned proposal at the sizes of its configuration: a network trained on 2048 chains x
        # 489 cycles = 1,001,472 plain-HMC poses of the state, batches of 4096 (the tensor-core
        # path), moves of the rigid body and of every torsion; at the paper's own regime of
        # external-coordinate moves (alpha ~ 0.01), mid-leg, and the fully coupled end
        # Two move sets: rigid body and every torsion (the configuration's), and rigid body only
        # (the paper's external-coordinate moves with a learned proposal).
        extra["learned_vs_plain"] = [learned_vs_plain(ctx, sys_, stream, dev, target=k, n_torsions=nt)
                                     for nt in (-1, 0)
                                     for k in (N_STATES_BC + 1, N_STATES_BC + 28, N_STATES_BC + N_STATES_CD - 1)]
    if not args.no_protocol and world == 1:
        extra["protocol_initialization"] = protocol_build(ctx, sys_, stream)
        ctx.states_set(T, alpha, dt)
    if not args.no_bpmf and world == 1:
        extra["bpmf_eff_samples"] = bpmf_convergence(ctx, sys_, stream, dev)

    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(sys_, world),
        "roofline": roofline, "roofline_gather": roofline_gather, "roofline_issue": roofline_issue, "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk, "breakdown_ms": {"hmc": hmc_avg, "exchange_both_legs_beside_snapshot": sum(ex_ms) / len(ex_ms),
                                        "snapshot_tail_after_exchange": sum(ukn_ms) / len(ukn_ms),
                                        "wall_per_step_incl_flush":
                                        1e3 * wall / args.steps},
        "hmc_cycles_per_s": 1e3 / ms_per_step,
        "hmc_acceptance": float(acc[0]) / max(1, n_trials),
    }
    line.update(extra)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_cpu_baseline(sys_)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
