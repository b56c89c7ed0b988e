"""Runs the CPU oracle's restarted HPR (FP64, Eq. 9) to a KKT tolerance on a
synthetic SCUC preset and writes what it took: iterations, power-method
iterations, restarts, residuals, objective, wall time and the threads used.

TEST INFRASTRUCTURE ONLY.  It calls nothing but ``oracle`` and the seeded
input generator ``scuc_gen``.  The benchmark's CPU baseline reads the
oracle's own iteration count from the file this writes, so that count comes
from the oracle, never from the CUDA path.

    python oracle/solve_to_tolerance.py scuc13k [--tol 1e-4] [--threads 0] [--out FILE]
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("preset")
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--threads", type=int, default=0, help="OpenMP threads (0: all host cores; -1: single-threaded build)")
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    import oracle
    from scuc_gen import make_preset
    inst = make_preset(a.preset)
    lp = oracle.as_lp(inst)
    t0 = time.perf_counter()
    r = oracle.hpr_solve(lp, tol=a.tol, threads=None if a.threads < 0 else a.threads)
    el = time.perf_counter() - t0
    i = r["info"]
    rec = {"preset": a.preset, "m": inst.m, "n": inst.n, "nnz": inst.nnz, "tol": a.tol,
           "status": int(i["status"]), "iters": int(i["iters"]), "power_iters": int(i["power_iters"]),
           "restarts": int(i["restarts"]), "kkt": float(i["kkt"]), "rp": float(i["rp"]), "rd": float(i["rd"]),
           "gap": float(i["gap"]), "pobj": float(i["pobj"]), "dobj": float(i["dobj"]),
           "wall_s": el, "threads": int(i["threads"]), "host": platform.processor() or platform.machine(),
           "host_cores": os.cpu_count(),
           "command": "python oracle/solve_to_tolerance.py %s --tol %g --threads %d" % (a.preset, a.tol, a.threads)}
    out = a.out or os.path.join(ROOT, "profiles", "oracle_solve_%s.json" % a.preset)
    with open(out, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
