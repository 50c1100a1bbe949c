"""Writes tests/golden/longrun_ccp.json: the FP64 oracle's long-run
cycle-averaged profiles of the reduced argon CCP, one entry per seed.

The long-run statistical parity test compares the CUDA path's run of the same
seeds against these numbers.  The oracle takes tens of minutes per seed here,
too long to run beside the GPU test, so its results are stored; this script
calls only the oracle and the seeded input generators, and runs the seeds as
separate processes (one per host core).

    python tests/golden/make_longrun_ccp.py [--cycles N] [--seeds 1,2,3,4,5]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

# The reduced argon CCP of the long-run comparison (paper §1's scheme with the
# synthetic argon tables): 2.5 cm gap, 256 cells, 13.56 MHz, 30 mTorr, 300 K,
# 5e4 electrons and 5e4 ions loaded uniform at 2e14 m^-3 (Te = 2 eV).
SPEC = dict(n_cells=256, gap=0.025, n_per_species=50_000, mtorr=30.0, steps_per_cycle=400, diag_interval=8)


def case(seed: int, volts: float):
    from paper_2609_17151_b300 import workloads as W
    cfg, parts = W.ccp_case(seed=seed, n_cells=SPEC["n_cells"], gap=SPEC["gap"],
                            n_per_species=SPEC["n_per_species"], mtorr=SPEC["mtorr"], volts=volts,
                            steps_per_cycle=SPEC["steps_per_cycle"])
    cfg["diag_interval"] = SPEC["diag_interval"]
    return cfg, parts


def run_seed(seed: int, volts: float, cycles: int, avg_cycles: int) -> dict:
    import numpy as np

    import oracle
    from paper_2609_17151_b300 import workloads as W
    cfg, parts = case(seed, volts)
    c = oracle.Case(cfg)
    for s, p in enumerate(parts):
        c.load_particles(s, W.as_xi(p), p["vx"], p["vy"], p["vz"], p["id"])
    spc = SPEC["steps_per_cycle"]
    t0 = time.time()
    counts = []
    c.step(spc * (cycles - avg_cycles))
    c.reset_moments()
    for _ in range(avg_cycles):
        c.step(spc)
        counts.append([c.count(0), c.count(1)])
    m = c.moments()
    cnt = c.counters()
    n = cnt["n_steps"]
    return {"seed": seed, "seconds": time.time() - t0,
            "ne": (m["dens_sum"][0] / n).tolist(), "ni": (m["dens_sum"][1] / n).tolist(),
            "phi": (m["phi_sum"] / n).tolist(), "eepf": m["eepf"].tolist(), "n_diag": int(cnt["n_diag"]),
            "counts_per_cycle": counts, "final_counts": [c.count(0), c.count(1)],
            "mean_counts": np.mean(np.array(counts, dtype=float), axis=0).tolist()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cycles", type=int, default=300)
    ap.add_argument("--avg-cycles", type=int, default=100)
    ap.add_argument("--volts", type=float, default=200.0)
    ap.add_argument("--seeds", default="1,2,3,4,5")
    ap.add_argument("--out", default=os.path.join(HERE, "longrun_ccp.json"))
    a = ap.parse_args()
    seeds = [int(x) for x in a.seeds.split(",")]
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(seeds)) as pool:
        res = pool.starmap(run_seed, [(s, a.volts, a.cycles, a.avg_cycles) for s in seeds])
    out = {"what": "FP64 oracle, reduced argon CCP, profiles averaged over the last avg_cycles RF cycles",
           "spec": dict(SPEC, volts=a.volts, cycles=a.cycles, avg_cycles=a.avg_cycles),
           "made_by": "python tests/golden/make_longrun_ccp.py " + " ".join(sys.argv[1:]),
           "seeds": res}
    with open(a.out, "w") as f:
        json.dump(out, f)
    print(json.dumps({"seeds": seeds, "seconds": [r["seconds"] for r in res],
                      "final_counts": [r["final_counts"] for r in res]}))


if __name__ == "__main__":
    main()
