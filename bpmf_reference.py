#!/usr/bin/env python
"""Reference BPMF of the paper-scale workload, for the BPMF effective-samples measurement of
bench.py.  Writes bpmf_reference.json.

The BPMF ("Estimation": beta_T B = f_BC,L + f'_CD, MBAR per leg) of the paper-scale system is
estimated by independent long realizations of both sampling iterations, with seeds that bench.py
does not use:
- the paper's iteration (an HMC move and 20 external-coordinate moves at alpha < 0.01 per replica,
  then 25 exchange sweeps; "Sampling", "Equilibration and production");
- the same plus 4 learned moves per replica (an exact Metropolis-Hastings correction, so both
  iterations share their limit).
Each realization starts from its own seeded placements and warm-up, and its value is the mean
BPMF of the second half of its windows.  The reference is the mean over all realizations; the
spread (standard deviation) and standard error over realizations are stored beside it.  The FP64
oracle cannot run this workload; the GPU path's BPMF agrees with the oracle's within 0.05 kT on the
systems the oracle can run (tests/test_gpu_bpmf.py).

    python bpmf_reference.py [--paper-cycles 40000] [--learned-cycles 16000] [--realizations 2]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--paper-cycles", type=int, default=40000)
    p.add_argument("--learned-cycles", type=int, default=16000)
    p.add_argument("--realizations", type=int, default=2, help="per iteration")
    p.add_argument("--window", type=int, default=2000)
    p.add_argument("--out", default=os.path.join(ROOT, "bpmf_reference.json"))
    a = p.parse_args()
    import torch

    import bench
    from paper_1507_03703_gb300 import build as B
    B.build()
    from paper_1507_03703_gb300.algdock import Context
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    sys_ = bench.workload()
    T = np.concatenate([l.T for l in sys_.legs])
    alpha = np.concatenate([l.alpha for l in sys_.legs])
    dt = np.concatenate([l.dt_fs for l in sys_.legs])
    stream = torch.cuda.current_stream(dev)
    ctx = Context(0)
    ctx.set_stream(stream)
    nx, ny, nz = sys_.grid.n
    raw = [torch.empty((nz, ny, nx), dtype=torch.float32, device=dev) for _ in range(3)]
    ctx.grids_build(sys_.grid, sys_.receptor, *raw)
    ctx.grids_load(sys_.grid, *raw, ligand=sys_.ligand)
    ctx.ligand_load(sys_.ligand, sys_.site)
    ctx.states_set(T, alpha, dt)
    del raw
    runs = []
    t0 = time.time()
    for r in range(a.realizations):
        for method, n_cyc in (("paper", a.paper_cycles), ("learned", a.learned_cycles)):
            seed = 500 + 10 * r + (0 if method == "paper" else 5)
            pre, lp, _ = bench.bpmf_warm(ctx, sys_, seed)
            arm = bench.bpmf_arm(ctx, stream, dev, pre, lp if method == "learned" else None, n_cyc, a.window,
                                 seed + 1)
            w = [x["bpmf_kT"] for x in arm["windows"]]
            value = float(np.mean(w[len(w) // 2:]))
            runs.append({"method": method, "seed": seed, "cycles": n_cyc, "value_kT": value,
                         "windows_kT": w, "gpu_ms_per_cycle": arm["gpu_ms_per_cycle"]})
            print("%s seed %d: %.3f kT (windows %s)" % (method, seed, value, np.round(w, 2).tolist()), flush=True)
            del pre, lp
            torch.cuda.empty_cache()
    v = np.array([r["value_kT"] for r in runs])
    out = {"bpmf_kT": float(v.mean()), "spread_kT": float(v.std(ddof=1)), "sem_kT": float(v.std(ddof=1) / np.sqrt(v.size)),
           "realizations": len(runs), "runs": runs, "window_cycles": a.window,
           "source": "bpmf_reference.py --paper-cycles %d --learned-cycles %d --realizations %d"
                     % (a.paper_cycles, a.learned_cycles, a.realizations),
           "gpu": torch.cuda.get_device_name(0), "wall_s": time.time() - t0}
    with open(a.out, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: out[k] for k in ("bpmf_kT", "spread_kT", "sem_kT", "realizations")}))


if __name__ == "__main__":
    main()
