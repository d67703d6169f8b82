"""Writes bpmf_20atom_oracle.json: the FP64 oracle's BPMF of the twenty-atom test system, as
independent estimates from groups of chains ("Estimation": beta_T B = f_BC,L + f'_CD, MBAR over
each leg's replica-exchange samples).

Protocol of one group (the parity test repeats it on the GPU, group for group):
- the config-1 system (20-atom ligand, 1500 receptor atoms, 33^3 grids at 0.5 A), its 8 warming
  and 8 coupling states;
- 32 chains per leg, every group from the same starting configurations: the synthetic
  placements of seed 40 (warming leg) and 41 (coupling leg), 16 tries each, 256 per leg;
- 300 cycles of one 20-step HMC trial per replica and 25 exchange sweeps (separations 1..5),
  Philox seed 5000 + g, the first 50 cycles discarded; groups differ only in their seed, so each
  is an independent realization of the same process;
- MBAR per leg over the group's recorded samples; the group's BPMF is (f_C - f_B) + (f_D - f_C).

Only the oracle and the seeded input generators are used.  The file is rewritten after every
group, so an interrupted run keeps what it finished.

    python tests/golden/make_bpmf_20atom.py --groups 700 [--threads 0]
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from paper_1507_03703_gb300 import synthetic as S  # noqa: E402
from systems import oracle_system, raw_grids32  # noqa: E402

OUT = os.path.join(HERE, "bpmf_20atom_oracle.json")
PROTOCOL = {"system": "config_small(1)", "chains_per_group": 32, "cycles": 300, "vv_steps": 20, "burn_in": 50,
            "exchange_sweeps": 25, "max_sep": 5, "placement_seeds": "40, 41 (16 tries, 256 each)",
            "philox_seed": "5000 + g", "estimator": "MBAR per leg over the group's samples"}


def start_x0(system):
    """The starting configurations of every group: [warming leg C*K, coupling leg C*K]."""
    C, K = PROTOCOL["chains_per_group"], system.legs[0].K
    return [S.place_ligand(system.ligand, system.receptor, system.site, C * K, seed=40 + li,
                           n_tries=16).astype(np.float32) for li in range(2)]


def group_bpmf(system, g32, x0, g, n_threads=0):
    C = PROTOCOL["chains_per_group"]
    f = []
    for li, leg in enumerate(system.legs):
        osys = oracle_system(system, g32, leg.T, leg.alpha, leg.dt_fs)
        comps, st, _, _, _ = oracle.run_ladder(osys, x0[li], C, PROTOCOL["cycles"], PROTOCOL["vv_steps"],
                                               seed=5000 + g, n_sweeps=PROTOCOL["exchange_sweeps"],
                                               max_sep=PROTOCOL["max_sep"], burn_in=PROTOCOL["burn_in"],
                                               n_threads=n_threads)
        fk, _ = oracle.ladder_free_energies(leg.T, leg.alpha, comps, st)
        f.append(fk)
    return float(oracle.bpmf_kT(f[0], f[1]))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--groups", type=int, default=700)
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    system = S.config_small(1)
    g32 = raw_grids32(system)
    x0 = start_x0(system)
    done = {}
    if os.path.exists(OUT):
        prev = json.load(open(OUT))
        if prev.get("protocol") == PROTOCOL:
            done = {int(r["group"]): r["bpmf_kT"] for r in prev["groups"]}
    t0 = time.time()
    for g in range(args.groups):
        if g in done:
            continue
        done[g] = group_bpmf(system, g32, x0, g, args.threads)
        vals = np.array([done[k] for k in sorted(done)])
        rec = {"source": "tests/golden/make_bpmf_20atom.py (FP64 oracle)", "protocol": PROTOCOL,
               "n_groups": len(done), "mean_kT": float(vals.mean()),
               "standard_error_kT": float(vals.std(ddof=1) / np.sqrt(len(vals))) if len(vals) > 1 else None,
               "groups": [{"group": k, "bpmf_kT": done[k]} for k in sorted(done)]}
        tmp = OUT + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(rec, fh, indent=1)
        os.replace(tmp, OUT)
        print("group %d: %.4f kT; %d groups, mean %.4f +- %s (%.0f s)"
              % (g, done[g], len(done), rec["mean_kT"], rec["standard_error_kT"], time.time() - t0), flush=True)


if __name__ == "__main__":
    main()
