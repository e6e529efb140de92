"""Write the oracle's own reconstruction schedule for a benchmark workload
(TEST INFRASTRUCTURE: runs only the FP64 oracle on the seeded inputs).

For every FBS iteration of the multigrid schedule (Algorithm A1 under
Sec. II.C.3, with the benchmark's parameters) it records the ROF sub-solve's
accepted steps and step reductions, and the step tau of every level. The
benchmark's CPU baseline multiplies per-operation oracle timings by these
counts to estimate one full oracle reconstruction from a bounded sample.
The wall time of the full run is printed (it belongs to the machine that ran
it), not stored.

    python oracle/make_schedule.py paper      # about 25 min on 8 cores
    python oracle/make_schedule.py cube40
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

POWER_ITERS, POWER_ITERS_FINE = 20, 4   # the benchmark's step-size schedule


def schedule_path(name: str) -> str:
    return os.path.join(HERE, f"schedule_{name}.json")


def main(name: str) -> None:
    from oracle import oracle as orc
    from paper_1001_0599_gb300 import synthetic

    orc.build()
    wl = synthetic.workload(name)
    _, y = synthetic.make_problem(wl)
    g = orc.Geometry.from_workload(wl)
    t0 = time.perf_counter()
    res = orc.reconstruct(g, y, wl.lam, wl.iters, orc.TVParams(eps_tv=1e-5), power_iters=POWER_ITERS,
                          clamp=True, power_iters_fine=POWER_ITERS_FINE)
    wall = time.perf_counter() - t0
    levels = [{"fbs": []} for _ in wl.iters]
    for it in res.iters:
        levels[it.level]["fbs"].append({"n_inner": int(it.n_inner), "backtracks": int(sum(it.steps)),
                                        "flags": int(it.flags)})
    out = {"workload": name, "iters": list(wl.iters), "power_iters": POWER_ITERS,
           "power_iters_fine": POWER_ITERS_FINE, "taus": [float(t) for t in res.taus], "levels": levels,
           "_doc": "written by oracle/make_schedule.py from a full FP64 oracle reconstruction"}
    with open(schedule_path(name), "w") as fh:
        json.dump(out, fh, indent=1)
    cores = os.environ.get("OMP_NUM_THREADS") or os.cpu_count()
    print(json.dumps({"workload": name, "oracle_full_s": wall, "cores": int(cores)}))


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "paper")
