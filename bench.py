"""Benchmark: seconds to 1e-4 KKT on the 13,000-bus SCUC LP relaxation.

One step = one pass of the whole path over one LP: the warm-start network's
prediction for every generator-hour and the assembled starting point, then
Pock-Chambolle scaling, power method and restarted HPR iterations to
max(r_p, r_d, gap) <= 1e-4 (Sec. 3) from that point (with the cold-start
reference period and fallback), then Round + Algorithm 1 fixing and bound
propagation with the reduced-LP build (Sec. 4).  The LP, the features and
the network are on the device before timing (inputs resident in HBM); `e2e`
repeats the measurement through the C ABI from host buffers, host<->device
copies included.  Variants on the same GPU: plain FP64 from cold start, FP32
matvecs from cold start.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "s to 1e-4 KKT, 13k-bus SCUC LP: plain vs warm/batched/FP32; SpMV % HBM peak"
WORKLOAD = "scuc13k"
WORKLOAD_DESC = ("13,000 buses, 18,000 lines, 4,000 units, T=36, 200 N-1 lines; Eq. 1-7 LP relaxation, "
                 "PTDF network rows (Eq. 6), seed 20000")
WS_WEIGHTS = os.path.join(ROOT, "paper_2510_10891_b300", "weights", "ws_mlp.npz")
WS_FILL = 0   # u and p' from the network; v, w, segments and duals from the iteration


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def spmv_bytes(m, n, nnz_a, kind, prec, lay=None):
    """Algorithmic bytes of one fused SpMV launch (each matrix entry and each
    vector element touched once).  FP32 products read the matrix entries in
    the storage scuc_lp_layout reports (lay): 6 bytes (value + 16-bit
    offset) for entries of chunks and of a compressed sliced copy of A^T
    (with a 16-byte record per column), 8 bytes (value + 32-bit index) for
    the others; lay None: 8 bytes per entry and a 4-byte row pointer per
    row."""
    vb = 8 if prec == "fp64" else 4
    if kind == "dual":   # A x_t, then y/y0/lo/hi in, y out (+ FP32 shadow of y)
        mat = (vb + 4) * nnz_a + 4 * (m + 1)
        if vb == 4 and lay:
            mat -= 2 * lay["a_chunk16"]
        return mat + vb * n + 32 * m + 8 * m + (4 * m if vb == 4 else 0)
    # primal: A^T y, then x/x0/c/xl/xu in, x and x_t out
    mat = (vb + 4) * nnz_a + 4 * (n + 1)
    if vb == 4 and lay:
        if lay["t_sell_compressed"]:
            mat = 6 * nnz_a + 2 * lay["t_chunk32"] + 16 * n
        else:
            mat -= 2 * lay["t_chunk16"]
    return mat + vb * m + 40 * n + 8 * n + (8 * n if vb == 8 else 4 * n)


# sources the iteration SpMV kernels are built from (kernels and the
# partition planner): the stored DRAM traffic is valid while they are
SPMV_SOURCES = ("common.cuh", "spmv.cuh", "lp_kernels.cuh", "partition.cu")
TRAFFIC_FILE = "spmv_traffic_scuc6k.json"
# the launches of one half-step, timed together by the profiled solves
STEP_KERNELS = {
    "primal": "primal step: k_primal_sell (update fused) on plain iterations, + k_primal_epi on checks",
    "dual": "dual step: k_dual_fused + k_dual_long on plain iterations, k_chunks_iter + k_dual on checks",
}


def csrc_hash():
    h = hashlib.sha256()
    for name in SPMV_SOURCES:
        with open(os.path.join(ROOT, "paper_2510_10891_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1])); mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


ORACLE_RUN = os.path.join(ROOT, "profiles", "oracle_solve_scuc13k.json")
SMALL = "scuc2k"
SMALL_DESC = ("2,000 buses, 2,800 lines, 300 units, T=36, 50 N-1 lines; Eq. 1-7 LP relaxation, PTDF network "
              "rows (Eq. 6), seed 2")


def host_threads():
    """Host cores the oracle may use (the count nproc reports)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_to_tolerance(inst, threads):
    """The oracle (FP64, OpenMP build, loops as written) solving the LP to
    1e-4 KKT: wall seconds, iterations and what the solve returned."""
    import oracle
    lp = oracle.as_lp(inst)
    t0 = time.perf_counter()
    r = oracle.hpr_solve(lp, tol=1e-4, threads=threads)
    el = time.perf_counter() - t0
    i = r["info"]
    return {"s": el, "iters": int(i["iters"]), "power_iters": int(i["power_iters"]), "status": int(i["status"]),
            "kkt": float(i["kkt"]), "pobj": float(i["pobj"]), "threads": int(i["threads"])}


def oracle_13k_sample(inst, threads):
    """The oracle on all host cores over a bounded sample of the 13k-bus LP:
    set-up plus 8 and 24 iterations (lambda fixed, so no power method), the
    per-iteration time scaled to the oracle's own iteration count to 1e-4
    (HPR + power iterations, the latter as one iteration each) from its
    recorded run to tolerance (oracle/solve_to_tolerance.py)."""
    import oracle
    with open(ORACLE_RUN) as f:
        rec = json.load(f)
    lp = oracle.as_lp(inst)
    kw = dict(tol=0.0, lambda_in=1.0, check_every=8, threads=threads)
    t0 = time.perf_counter(); oracle.hpr_solve(lp, max_iter=8, **kw); t8 = time.perf_counter() - t0
    t0 = time.perf_counter(); r = oracle.hpr_solve(lp, max_iter=24, **kw); t24 = time.perf_counter() - t0
    per_iter = max((t24 - t8) / 16.0, 1e-9)
    setup = max(t8 - 8 * per_iter, 0.0)
    est = setup + (rec["iters"] + rec["power_iters"]) * per_iter
    return {"value": est, "unit": "s", "kind": "oracle, extrapolated from a bounded sample",
            "threads": int(r["info"]["threads"]), "s_per_iter": per_iter, "setup_s": setup,
            "sample_s": t8 + t24, "oracle_iters": rec["iters"], "oracle_power_iters": rec["power_iters"],
            "iterations_source": "profiles/oracle_solve_scuc13k.json (the oracle's own run to 1e-4: "
                                 + rec["command"] + ")"}


def cpu_baseline(inst, result=None):
    """The oracle as it stands on all host cores: a bounded sample of the
    13k-bus LP scaled to the oracle's own iteration count (value), the
    2,000-bus LP solved to 1e-4 (measured), and the oracle's FP64 KKT
    evaluation of the timed step's returned point on the unscaled LP (the
    error of the GPU result against the oracle)."""
    import oracle
    from scuc_gen import make_preset
    threads = host_threads()
    check = None
    if result is not None:
        k = oracle.kkt(oracle.as_lp(inst), *result)
        check = {k2: float(k[k2]) for k2 in ("kkt", "rp", "rd", "gap", "pobj", "dobj")}
    s13 = oracle_13k_sample(inst, threads)
    s13_1 = oracle_13k_sample(inst, None)   # the same sample, single-threaded build
    full = oracle_to_tolerance(make_preset(SMALL), threads)
    return {"value": s13["value"], "unit": "s", "cores": s13["threads"], "kind": "oracle",
            "sample": "oracle (FP64, OpenMP, %d threads) on the 13k-bus LP: set-up + 8 and + 24 iterations "
                      "(%.1f s of CPU work), %.3f s/iteration x (%d HPR + %d power iterations, the oracle's own "
                      "count to 1e-4) + %.2f s set-up" % (s13["threads"], s13["sample_s"], s13["s_per_iter"],
                                                          s13["oracle_iters"], s13["oracle_power_iters"],
                                                          s13["setup_s"]),
            "scuc13k_sample": s13, "scuc13k_sample_one_core": s13_1,
            "measured_to_tolerance": dict(full, workload=SMALL_DESC),
            "oracle_kkt_of_step_result": check}


def batched_variant(P, dist=None, pending=None):
    """The 64 uneven relaxations of the batch family (200-3,000 buses, 0.15
    units per bus, T in {24, 36}, seeds 1000-1063) to 1e-4 with FP32
    matvecs.  Under torchrun the family is sharded over the ranks by size
    (ranks.shard on buses x hours; no data-path collective): each rank
    solves its share, the job time is the slowest rank's.  On each rank:
    the share in one batched call (the first call tunes the SpMV partition
    shapes), the same call again (shapes reused: a later round of the same
    batch), and the share solved one by one on the same GPU; wall clock,
    set-up included on every side."""
    import multiprocessing as mp
    import torch
    from paper_2510_10891_b300.ranks import gather_on_rank0, max_over_ranks, shard
    from scuc_gen.scuc import batch_configs, make_scuc
    world = dist.get_world_size() if dist is not None and dist.is_initialized() else 1
    rank = dist.get_rank() if world > 1 else 0
    cfgs = batch_configs(64, 1000)
    mine = shard([c.buses * c.T for c in cfgs], rank, world)
    with mp.get_context("spawn").Pool(max(1, min(16, len(mine)))) as pool:
        insts = pool.map(make_scuc, [cfgs[i] for i in mine])
    lps = [P.LP(i) for i in insts]
    kw = dict(tol=1e-4, precision="mixed")
    P.solve_batch(lps[:2], **kw)                       # loads the kernels
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res, bi = P.solve_batch(lps, **kw)
    tb = time.perf_counter() - t0
    t0 = time.perf_counter()
    res2, bi2 = P.solve_batch(lps, **kw)
    tb2 = time.perf_counter() - t0
    t0 = time.perf_counter()
    solo = [lp.solve(want=("x",), **kw) for lp in lps]
    ts = time.perf_counter() - t0
    # the same LPs one by one again: each handle's first-solve set-up (its
    # sliced copies and chunk stream) already done, as for a later round
    t0 = time.perf_counter()
    for lp in lps:
        lp.solve(want=("x",), **kw)
    ts2 = time.perf_counter() - t0
    its = [r["info"]["iters"] for r in res]
    # each batched LP's answer against its solo solve, and (CPU leg) the
    # oracle's KKT evaluation of the batched point
    obj_diff = max(abs(r["info"]["pobj"] - q["info"]["pobj"]) / max(1.0, abs(q["info"]["pobj"]))
                   for r, q in zip(res, solo))
    kkt_refs = [{} for _ in res]
    if pending is not None:
        for i, r in enumerate(res):
            pending.append((kkt_refs[i], "kkt", insts[i], r["x"], r["y"], r["z"]))
    loc = {"rank": rank, "lps": len(lps), "nnz": int(sum(i.nnz for i in insts)), "batch_s": tb,
           "batch_again_s": tb2, "one_by_one_s": ts, "one_by_one_again_s": ts2,
           "all_optimal": all(r["info"]["status"] == 0 for r in res + res2),
           "iters_min": min(its), "iters_max": max(its), "max_rel_objective_diff_vs_solo": obj_diff,
           "first_call_ms": {"scaling_and_power": bi["scale_ms"], "setup": bi["setup_ms"], "tune": bi["tune_ms"],
                             "iterations": bi["solve_ms"], "total": bi["total_ms"]},
           "again_ms": {"scaling_and_power": bi2["scale_ms"], "setup": bi2["setup_ms"], "tune": bi2["tune_ms"],
                        "tune_cached": bi2["tune_cached"], "iterations": bi2["solve_ms"], "total": bi2["total_ms"]},
           "shape_A": [bi["ept_A"], bi["run_A"]], "shape_AT": [bi["ept_T"], bi["run_T"]],
           "launches": bi["launches"], "solo_iters_sum": int(sum(r["info"]["iters"] for r in solo))}
    for lp in lps:
        lp.close()
    job = {k: max_over_ranks(loc[k], dist, device="cuda")
           for k in ("batch_s", "batch_again_s", "one_by_one_s", "one_by_one_again_s")}
    per_rank = gather_on_rank0(loc, dist)
    out = {"ranks": world, "lps": 64, "job_batch_s": job["batch_s"], "job_batch_again_s": job["batch_again_s"],
           "job_one_by_one_s": job["one_by_one_s"], "job_one_by_one_again_s": job["one_by_one_again_s"],
           "speedup": job["one_by_one_s"] / job["batch_s"],
           "speedup_again": job["one_by_one_again_s"] / job["batch_again_s"],
           "sharding": "ranks.shard over buses x hours, no data-path collective"}
    if per_rank is not None:
        out["per_rank"] = per_rank
    out["_kkt_refs"] = kkt_refs
    return out


def build_instance():
    from scuc_gen import make_preset
    return make_preset(WORKLOAD)


def workload_config(m, n, nnz, world):
    """The workload both arms report (the reference arm prints the same
    dict): what is solved, not how or with what result."""
    return {"workload": WORKLOAD_DESC, "m": m, "n": n, "nnz": nnz, "tol": 1e-4,
            "parallelism": "replicas" if world > 1 else "1 GPU",
            "l2": "inputs larger than L2 (matrix %.2f GB per pass)" % (12 * nnz / 1e9)}


def run_reference(args):
    """CPU reference arm: the oracle (FP64, OpenMP build) on all host cores,
    on the GPU arm's workload (the 13k-bus LP) and config.  Every step is a
    bounded sample of that solve (set-up + 8 and set-up + 24 iterations), and
    its value is the sample's per-iteration time scaled to the oracle's own
    iteration count to 1e-4 plus its set-up time (oracle_13k_sample);
    ms_per_step is the wall time the sample took.  The 2,000-bus LP solved
    to 1e-4 in full (measured, not scaled) is reported beside it."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from scuc_gen import make_preset
    threads = host_threads()
    inst = build_instance()
    samples = [oracle_13k_sample(inst, threads) for _ in range(args.warmup + args.steps)]
    timed = samples[args.warmup:]
    v = float(np.mean([t["value"] for t in timed]))
    wall = float(np.mean([t["sample_s"] for t in timed]))
    last = timed[-1]
    full = oracle_to_tolerance(make_preset(SMALL), threads)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    sample = ("oracle (FP64, OpenMP, %d threads) on the 13k-bus LP: set-up + 8 and + 24 iterations per step "
              "(%.1f s of CPU work), %.4f s/iteration x (%d HPR + %d power iterations, the oracle's own count "
              "to 1e-4) + %.2f s set-up; mean of %d timed steps" %
              (last["threads"], wall, float(np.mean([t["s_per_iter"] for t in timed])), last["oracle_iters"],
               last["oracle_power_iters"], float(np.mean([t["setup_s"] for t in timed])), args.steps))
    line = {"metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": wall * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": workload_config(inst.m, inst.n, inst.nnz, world),
            "value_note": "seconds to 1e-4 scaled from each step's bounded sample; ms_per_step is the "
                          "sample's wall time",
            "cpu_baseline": {"value": v, "unit": "s", "cores": last["threads"], "kind": "oracle",
                             "sample": sample},
            "scuc13k_sample": last,
            "measured_to_tolerance": dict(full, workload=SMALL_DESC),
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def filtering_variant(P, inst, full_s):
    """Transmission filtering (Fig. 1) on the same LP: solve without the
    base-case line and N-1 rows, add the violated ones, re-solve warm, until
    none is violated (FP32 matvecs, tol 1e-4, violation tol 1e-4 relative).
    Wall clock of the whole loop (solves, violation checks, row appending)."""
    import torch
    from scuc_gen import split_network_rows
    base, pool, _ = split_network_rows(inst)
    gb, gp = P.LP(base), P.LP(pool)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f = P.transmission_filter(gb, gp, viol_tol=1e-4, tol=1e-4, precision="mixed", time_limit_s=120.0)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    res = {"s": el, "converged": bool(f["converged"]), "rounds": len(f["rounds"]),
           "pool_rows": pool["m"], "pool_nnz": int(len(pool["val"])), "rows_added": int(len(f["rows_added"])),
           "final_lp": [int(f["lp"].m), int(f["lp"].n), int(f["lp"].nnz)],
           "iters_per_round": [int(r["iters"]) for r in f["rounds"]], "pobj": f["result"]["info"]["pobj"],
           "full_lp_step_s": full_s}
    if f["lp"] is not gb:
        f["lp"].close()
    gb.close(); gp.close()
    return res


def row_box(inst):
    """Row bounds [lo, hi] of the instance's senses (G, L, E, R) as CUDA tensors."""
    import torch
    sense, rhs, rng = np.asarray(inst.sense), np.asarray(inst.rhs, float), np.asarray(inst.rng_, float)
    lo = np.where((sense == ord("G")) | (sense == ord("E")) | (sense == ord("R")), rhs, -np.inf)
    hi = np.where((sense == ord("L")) | (sense == ord("E")), rhs, np.where(sense == ord("R"), rhs + rng, np.inf))
    return torch.as_tensor(lo, device="cuda"), torch.as_tensor(hi, device="cuda")


def primal_violation(lp, x, lo, hi):
    """Absolute primal violation behind r_p at x: A x by the library's FP64
    product on the unscaled LP, its distance to [lo, hi] (l2 and largest
    entry) and l2 / (1 + ||b||), the normalised r_p."""
    import torch
    ax = lp.matvec(x, torch.empty(lp.m, dtype=torch.float64, device="cuda"))
    d = ax - torch.minimum(torch.maximum(ax, lo), hi)
    b = torch.where(torch.isfinite(lo), lo.abs(), torch.zeros_like(lo))
    b = torch.maximum(b, torch.where(torch.isfinite(hi), hi.abs(), torch.zeros_like(hi)))
    l2 = float(torch.linalg.vector_norm(d))
    return {"l2": l2, "max": float(d.abs().max()), "rows_violated_1e-6": int((d.abs() > 1e-6).sum()),
            "b_norm": float(torch.linalg.vector_norm(b)), "r_p": l2 / (1.0 + float(torch.linalg.vector_norm(b)))}


def fp64_kernel_profile(P, lp, m, n, nnz, peak, fp64_tflops):
    """Per-launch CUDA-event times of the two FP64 iteration steps (256
    iterations, host-launched periods): GB/s against the HBM peak and the
    FLOP rate of the products (2 per nonzero) against the measured FP64 FMA
    peak (the products are bound by both)."""
    r = P.LP.solve(lp, want=("x",), tol=0.0, max_iter=256, use_graph=0, profile=1, precision="fp64")
    i = r["info"]
    out = {}
    for kind, t, k in (("primal", i["ms_primal_spmv"], i["n_primal_spmv"]), ("dual", i["ms_dual_spmv"],
                                                                              i["n_dual_spmv"])):
        ms = t / max(k, 1)
        gbs = spmv_bytes(m, n, nnz, kind, "fp64") / (ms * 1e-3) / 1e9
        tf = 2.0 * nnz / (ms * 1e-3) / 1e12
        out["%s_fp64" % kind] = {"avg_ms": ms, "launches": k, "GBps": gbs, "frac_hbm": gbs / peak,
                                 "product_tflops": tf, "frac_fp64_fma_peak": tf / fp64_tflops}
    return out


def equal_answer_variant(P, WS, lp, inst, net, Xd, layout, stream, tol, pending, bounds, fix_tau=0.1):
    """Warm start + FP32 matvecs against plain FP64 from cold start, both to
    the same tolerance on the same GPU (CUDA events around each solve): times,
    iterations, relative objective difference, differing fix decisions on the
    two points; both points are queued for the oracle's FP64 KKT evaluation
    (the CPU leg).  ``bounds``: the model's column bounds, restored first
    (a fixing round changes them)."""
    import torch
    n, m = inst.n, inst.m
    xl0, xu0 = bounds
    res = {}
    pts = {}
    for name in ("plain_fp64", "warm_fp32_matvec"):
        lp.set_bounds(xl0, xu0)
        xo = torch.empty(n, dtype=torch.float64, device="cuda")
        yo = torch.empty(m, dtype=torch.float64, device="cuda")
        zo = torch.empty(n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if name == "plain_fp64":
            i = lp.solve_device(x_out=xo, y_out=yo, z_out=zo, tol=tol, precision="fp64", time_limit_s=300.0)
        else:
            pred = net.predict(Xd)
            x0, _ = WS.assemble(lp, layout, pred)
            i = lp.solve_warm(x0, x_out=xo, y_out=yo, z_out=zo, tol=tol, precision="mixed",
                              time_limit_s=300.0)["info"]
        e1.record(stream); e1.synchronize()
        res[name] = {"s": e0.elapsed_time(e1) / 1e3, "iters": i["iters"], "iters_fp32": i["iters_fp32"],
                     "status": i["status_name"], "kkt": i["kkt"], "pobj": i["pobj"], "dobj": i["dobj"]}
        pts[name] = (xo, yo, zo)
    fixes = {}
    for name, (xo, _, _) in pts.items():
        lp.set_bounds(xl0, xu0)
        fixes[name] = lp.fix_and_propagate(inst.G, inst.T, inst.u_idx, inst.v_idx, inst.w_idx, inst.u_init, xo,
                                           tau=fix_tau, is_int=inst.is_int, build_reduced=False)["fix"]
    lp.set_bounds(xl0, xu0)
    for name, (xo, yo, zo) in pts.items():
        pending.append((res[name], "oracle_kkt", inst, xo.cpu().numpy(), yo.cpu().numpy(), zo.cpu().numpy()))
    a, b = res["warm_fp32_matvec"], res["plain_fp64"]
    xw, x64 = pts["warm_fp32_matvec"][0], pts["plain_fp64"][0]
    res.update({"tol": tol, "speedup": b["s"] / a["s"],
                "rel_objective_diff": abs(a["pobj"] - b["pobj"]) / max(1.0, abs(b["pobj"])),
                "rel_x_distance": float(torch.linalg.vector_norm(xw - x64) / torch.linalg.vector_norm(x64)),
                "fix_decisions_differing": int(np.sum(fixes["warm_fp32_matvec"] != fixes["plain_fp64"])),
                "fix_decisions": int(fixes["plain_fp64"].size)})
    return res


def config2_variant(P):
    """The 2,000-bus LP (57 MB per iteration: L2-resident, so times, not an
    HBM fraction): microseconds per iteration step with FP64 and with FP32
    matvecs (per-launch CUDA events, 512 iterations), and seconds to 1e-4
    (one graph launch per solve, median of three)."""
    import torch
    from scuc_gen import make_preset
    inst = make_preset(SMALL)
    lp = P.LP(inst)
    out = {"workload": SMALL_DESC, "m": inst.m, "n": inst.n, "nnz": inst.nnz,
           "note": "working set fits in the 126 MB L2: times are L2-resident, not an HBM roofline"}
    for prec in ("fp64", "mixed"):
        r = lp.solve(want=("x",), tol=0.0, max_iter=512, use_graph=0, profile=1, precision=prec)
        i = r["info"]
        rec = {"primal_step_us": 1e3 * i["ms_primal_spmv"] / i["n_primal_spmv"],
               "dual_step_us": 1e3 * i["ms_dual_spmv"] / i["n_dual_spmv"]}
        ts = []
        for _ in range(3):
            torch.cuda.synchronize(); t0 = time.perf_counter()
            r = lp.solve(want=("x",), tol=1e-4, precision=prec)
            ts.append(time.perf_counter() - t0)
        rec.update({"s_to_1e-4": float(np.median(ts)), "iters": r["info"]["iters"], "pobj": r["info"]["pobj"],
                    "status": r["info"]["status_name"]})
        out["fp64" if prec == "fp64" else "fp32_matvec"] = rec
    out["fp64_over_fp32_matvec"] = out["fp64"]["s_to_1e-4"] / out["fp32_matvec"]["s_to_1e-4"]
    lp.close()
    return out


def config3_variant(P, pending):
    """Algorithm 2 on the 6,500-bus LP (Sec. 4.2): solve the relaxation (FP32
    matvecs, FP64 reductions, FP64 final phase below the precision floor),
    then per round fix with tau = 0.02, propagate, and solve the reduced LP
    from the previous point, until a round fixes no further binary.  Per
    round: fixed triples and columns, reduced-LP size, iterations, objective
    (with the fixed columns' constant) and the oracle's KKT evaluation of the
    round's point on its LP (queued for the CPU leg).  Wall clock of the
    whole loop."""
    import torch
    from scuc_gen import make_preset
    inst = make_preset("scuc6k")
    lp = P.LP(inst)
    m = inst.m
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = lp.solve(tol=1e-4, precision="mixed")
    i = r["info"]
    rounds = [{"lp": [inst.m, inst.n, inst.nnz], "iters": i["iters"], "iters_fp32": i["iters_fp32"],
               "status": i["status_name"], "pobj": i["pobj"]}]
    pts = [(inst, r["x"], r["y"], r["z"])]
    xs, ys = r["x"], r["y"]
    prev = None
    for _ in range(20):
        f = lp.fix_and_propagate(inst.G, inst.T, inst.u_idx, inst.v_idx, inst.w_idx, inst.u_init, xs, tau=0.02,
                                 is_int=inst.is_int)
        if f["reduced"] is None:
            rounds.append({"infeasible": bool(f["infeasible"])})
            break
        nfix = int(f["info"]["nfixed"])
        red = f["reduced"]
        if prev is not None and nfix == prev:
            red.close()
            rounds.append({"fixed_triples": nfix, "stop": "no further binary fixed"})
            break
        sr = red.solve(x0=xs[f["col_map"]], y0=ys[f["row_map"]], tol=1e-4, precision="mixed", time_limit_s=120.0)
        xl, _ = lp.get_bounds()
        pts.append((red.export(), sr["x"], sr["y"], sr["z"]))
        xs = xl.copy()
        xs[f["col_map"]] = sr["x"]
        ys = np.zeros(m)
        ys[f["row_map"]] = sr["y"]
        si = sr["info"]
        rounds.append({"fixed_triples": nfix, "fixed_cols": int(f["info"]["n_fixed_cols"]),
                       "lp": [int(red.m), int(red.n), int(red.nnz)], "iters": si["iters"],
                       "iters_fp32": si["iters_fp32"], "status": si["status_name"],
                       "pobj": si["pobj"] + f["info"]["obj_const"], "fix_ms": f["info"]["ms"]})
        red.close()
        prev = nfix
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    k = 0
    for rec in rounds:
        if "lp" in rec:
            pending.append((rec, "oracle_kkt", *pts[k]))
            k += 1
    lp.close()
    return {"workload": "6,500 buses, 9,000 lines, 1,000 units, T=36, 100 N-1 lines, seed 3", "tau": 0.02,
            "s": wall, "rounds": rounds}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--start", default="warm", choices=["warm", "cold"],
                    help="warm: learned warm start (weights in paper_2510_10891_b300/weights)")
    ap.add_argument("--ncu-case", default=None,
                    help="profiling target: 128 iterations (no graph; FP32 matvecs unless "
                         "--ncu-precision fp64) on this preset, no JSON line")
    ap.add_argument("--ncu-precision", default="mixed", choices=["mixed", "fp64"],
                    help="matvec precision of the --ncu-case iterations")
    ap.add_argument("--ncu-ws", type=int, default=0,
                    help="profiling target: the warm-start network's prediction for this many synthetic "
                         "generator-hours (twice), no JSON line")
    ap.add_argument("--ncu-fix", default=None,
                    help="profiling target: one fixing round (Round, Algorithm 1, propagation, reduced LP) "
                         "on this preset after a mixed-precision solve to 1e-4, no JSON line")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.ncu_case:
        import paper_2510_10891_b300 as P
        from scuc_gen import make_preset
        lp = P.LP(make_preset(args.ncu_case))
        r = lp.solve(want=("x",), tol=0.0, max_iter=128, use_graph=0, precision=args.ncu_precision,
                     polish_stall=10 ** 6, polish_factor=0.0)
        print("ncu case %s: %d iterations; layout %s" % (args.ncu_case, r["info"]["iters"], json.dumps(lp.layout())))
        return 0
    if args.ncu_ws:
        import torch
        from paper_2510_10891_b300 import warmstart as WS
        net = WS.WarmStartNet.load(WS_WEIGHTS)
        g = torch.Generator(device="cuda").manual_seed(0)
        X = torch.randn((args.ncu_ws, net.dims[0]), generator=g, device="cuda", dtype=torch.float32)
        for _ in range(2):
            p = net.predict(X)
        torch.cuda.synchronize()
        print("ncu ws: %d rows, mean prediction %s" % (args.ncu_ws, p.mean(0).tolist()))
        return 0
    if args.ncu_fix:
        import paper_2510_10891_b300 as P
        from scuc_gen import make_preset
        inst = make_preset(args.ncu_fix)
        lp = P.LP(inst)
        x = lp.solve(want=("x",), tol=1e-4, precision="mixed")["x"]
        f = lp.fix_and_propagate(inst.G, inst.T, inst.u_idx, inst.v_idx, inst.w_idx, inst.u_init, x, tau=0.1,
                                 is_int=inst.is_int)
        i = f["info"]
        print("ncu fix %s: %d fixed, %d passes, reduced LP %s, %.1f ms" %
              (args.ncu_fix, i["nfixed"], i["passes"], (i["m_red"], i["n_red"], i["nnz_red"]), i["ms"]))
        if f["reduced"] is not None:
            f["reduced"].close()
        return 0

    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_2510_10891_b300 as P
    from paper_2510_10891_b300 import warmstart as WS
    from scuc_gen.features import ws_features, ws_layout_arrays
    inst = build_instance()
    m, n, nnz = inst.m, inst.n, inst.nnz
    stream = torch.cuda.current_stream()
    lp = P.LP(inst, stream=stream.cuda_stream)
    xo = torch.empty(n, dtype=torch.float64, device="cuda")
    yo = torch.empty(m, dtype=torch.float64, device="cuda")
    zo = torch.empty(n, dtype=torch.float64, device="cuda")
    kw = dict(tol=1e-4, precision=args.precision, profile=1, time_limit_s=600.0)
    xl0, xu0 = lp.get_bounds()
    fix_ms = []
    warm = args.start == "warm"
    GT = inst.G * inst.T
    if warm:
        net = WS.WarmStartNet.load(WS_WEIGHTS, stream=stream.cuda_stream)
        lay_arrays = ws_layout_arrays(inst)
        layout = WS.Layout(lay_arrays, WS_FILL)
        feats = ws_features(inst)
        Xd = torch.as_tensor(feats, device="cuda")
        pred = torch.empty((GT, 3), dtype=torch.float32, device="cuda")
        x0 = torch.empty(n, dtype=torch.float64, device="cuda")

    def step():
        # W: predictions and starting point; A0-A7: solve the relaxation;
        # F1-F3: fix, propagate, build the reduced LP
        if warm:
            net.predict(Xd, out=pred)
            WS.assemble(lp, layout, pred, x0=x0)
            info = lp.solve_warm(x0, x_out=xo, y_out=yo, z_out=zo, **kw)["info"]
            info["launches"] += WS.launches_predict(net.dims) + WS.launches_assemble(layout)
        else:
            info = lp.solve_device(x_out=xo, y_out=yo, z_out=zo, **kw)
        r = lp.fix_and_propagate(inst.G, inst.T, inst.u_idx, inst.v_idx, inst.w_idx, inst.u_init, xo,
                                 tau=0.1, is_int=inst.is_int)
        if r["reduced"] is not None:
            info["reduced"] = (r["reduced"].m, r["reduced"].n, r["reduced"].nnz)
            r["reduced"].close()
        info["fix"] = r["info"]
        fix_ms.append(r["info"]["ms"])
        return info

    for _ in range(args.warmup):
        lp.set_bounds(xl0, xu0)
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    infos, times = [], []
    pending = []   # (dict, key, LP, x, y, z): points the CPU leg evaluates with the oracle
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        t_all0 = time.perf_counter()
        for _ in range(args.steps):
            lp.set_bounds(xl0, xu0)          # same model every step (not timed)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos.append(step())
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_all0
    # the last timed step's point, for the oracle's check in the CPU leg
    step_result = (xo.cpu().numpy(), yo.cpu().numpy(), zo.cpu().numpy()) if not args.no_cpu else None
    if dist:
        dist.barrier()
    from paper_2510_10891_b300.ranks import max_over_ranks
    per_step = max_over_ranks(float(np.mean(times)), dist, device="cuda")
    clocks = clk.summary()

    # roofline of the dominant SpMV (largest summed time), from the timed steps
    peak, peak_src = peaks()
    agg = {}
    for i in infos:
        for kind in ("dual", "primal"):
            t_all, n_all = i["ms_%s_spmv" % kind], i["n_%s_spmv" % kind]
            t32, n32 = i["ms_%s_spmv_f32" % kind], i["n_%s_spmv_f32" % kind]
            for prec, tt, nn in (("fp32", t32, n32), ("fp64", t_all - t32, n_all - n32)):
                a = agg.setdefault((kind, prec), [0.0, 0])
                a[0] += tt; a[1] += nn
    (dk, dp), (dms, dn) = max(agg.items(), key=lambda kv: kv[1][0])
    nnz_a = nnz
    lay = lp.layout()
    byts = spmv_bytes(m, n, nnz_a, dk, "fp64" if dp == "fp64" else "fp32", lay)
    avg_ms = dms / max(dn, 1)
    achieved = byts / (avg_ms * 1e-3) / 1e9
    traffic, traffic_note = None, None
    tf = os.path.join(ROOT, "profiles", TRAFFIC_FILE)
    if os.path.exists(tf):
        with open(tf) as f:
            t = json.load(f)
        key = "%s_%s" % (dk, dp)
        if t.get("csrc_sha") == csrc_hash() and key in t.get("dram_bytes_per_launch", {}):
            # captured on the 6.5k-bus LP (the capture size rule), scaled to
            # this launch by the ratio of algorithmic bytes
            scale = spmv_bytes(m, n, nnz, dk, dp, lay) / spmv_bytes(t["m"], t["n"], t["nnz"], dk, dp,
                                                                     t.get("layout"))
            traffic = t["dram_bytes_per_launch"][key] * scale
            traffic_note = "ncu DRAM bytes of the %s launch on the %s LP x %.3f (algorithmic-bytes ratio)" % (
                key, t["workload"], scale)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_source": traffic_note, "kernel": "%s (%s matvec)" % (STEP_KERNELS[dk], dp),
            "bytes_per_launch": byts, "avg_launch_ms": avg_ms, "launches": dn, "peak_source": peak_src,
            "all_kernels": {"%s_%s" % k: {"avg_ms": v[0] / max(v[1], 1), "launches": v[1],
                                          "GBps": spmv_bytes(m, n, nnz_a, k[0], "fp64" if k[1] == "fp64" else "fp32",
                                                             lay)
                                          / (v[0] / max(v[1], 1) * 1e-3) / 1e9 if v[1] else None}
                            for k, v in agg.items()}}

    last = infos[-1]
    out = {"metric": METRIC, "value": per_step, "unit": "s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 matvec + f64" if args.precision == "mixed" else "f64", "data": "synthetic",
           "config": workload_config(m, n, nnz, world),
           "result": {"precision": args.precision,
                      "iters": last["iters"], "iters_fp32": last["iters_fp32"],
                      "power_iters": last["power_iters"], "restarts": last["restarts"],
                      "kkt": last["kkt"], "status": last["status_name"],
                      "solve_s": float(np.mean([i["solve_ms"] + i["setup_ms"] for i in infos])) / 1e3,
                      "fix_propagate_reduce_s": float(np.mean(fix_ms[-args.steps:])) / 1e3,
                      "fixed_triples": last["fix"]["nfixed"], "propagation_passes": last["fix"]["passes"],
                      "fix_ms_parts": {k: float(np.mean([i["fix"][k] for i in infos]))
                                       for k in ("ms_propagate", "ms_reduce", "ms_setup")},
                      "reduced_lp": last.get("reduced")},
           "roofline": roof, "clocks": clocks,
           "gpu_launches": int(sum(i["launches"] for i in infos)),
           "wall_s_timed": wall}

    if warm:
        out["result"]["start"] = ("learned warm start: MLP %s (BF16 tensor cores) on %d generator-hours, "
                                  "u and p' assembled, cold-start reference period + fallback" %
                                  ("-".join(str(d) for d in net.dims), GT))
        out["result"]["warm"] = {"status": last["status_name"], "ref_iters": last["ref_iters"],
                                 "warm_iters_rejected": last["warm_iters"],
                                 "cold_first_kkt": last["cold_first_kkt"]}
    else:
        out["result"]["start"] = "cold"

    bv = None
    if not args.no_batch:
        bv = batched_variant(P, dist, pending if rank == 0 else None)   # every rank solves its share

    if rank == 0 and not args.no_plain:
        # the same LP from cold start on the same GPU: plain FP64 and FP32
        # matvecs (solve + fix, as in the step)
        def timed(prec, **extra):
            lp.set_bounds(xl0, xu0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pi = lp.solve_device(x_out=xo, y_out=yo, z_out=zo, tol=1e-4, precision=prec,
                                 **{"time_limit_s": 600.0, **extra})
            r = lp.fix_and_propagate(inst.G, inst.T, inst.u_idx, inst.v_idx, inst.w_idx, inst.u_init, xo,
                                     tau=0.1, is_int=inst.is_int)
            e1.record(stream); e1.synchronize()
            if r["reduced"] is not None:
                r["reduced"].close()
            return e0.elapsed_time(e1) / 1e3, pi, r["fix"]
        xw = xo.clone() if warm else None
        fix_w = None
        if warm:
            lp.set_bounds(xl0, xu0)
            fix_w = lp.fix_and_propagate(inst.G, inst.T, inst.u_idx, inst.v_idx, inst.w_idx, inst.u_init, xw,
                                         tau=0.1, is_int=inst.is_int, build_reduced=False)["fix"]
        t64, p64, fix64 = timed("fp64")
        x64 = xo.clone()
        tmx, pmx, _ = timed("mixed")
        # the second algorithm (restarted PDHG with ergodic averaging) and the
        # cost of infeasibility detection, same start and precision
        tpd, ppd, _ = timed("mixed", algo="pdhg_avg", time_limit_s=120.0)
        tdt, pdt, _ = timed("mixed", infeas_tol=1e-8)
        v = {"plain_fp64_s": t64, "plain_fp64_iters": p64["iters"], "plain_fp64_status": p64["status_name"],
             "cold_mixed_s": tmx, "cold_mixed_iters": pmx["iters"], "cold_mixed_pobj": pmx["pobj"],
             "speedup_vs_plain_fp64": t64 / per_step,
             "pdhg_avg_cold_mixed": {"s": tpd, "iters": ppd["iters"], "status": ppd["status_name"],
                                     "kkt": ppd["kkt"], "restarts": ppd["restarts"]},
             "cold_mixed_with_detection": {"s": tdt, "iters": pdt["iters"], "status": pdt["status_name"]}}
        if warm:
            v["warm_mixed_s"] = per_step
            v["warm_mixed_iters"] = last["iters"]
            v["warm_vs_plain_fp64"] = {
                "rel_objective_diff": abs(last["pobj"] - p64["pobj"]) / max(1.0, abs(p64["pobj"])),
                "kkt_warm": last["kkt"], "kkt_plain": p64["kkt"],
                "rel_x_distance": float(torch.linalg.vector_norm(xw - x64) / torch.linalg.vector_norm(x64)),
                "fix_decisions_differing": int(np.sum(fix_w != fix64))}
        if warm:
            # the absolute primal violation behind r_p <= 1e-4 of both points
            d0 = row_box(inst)
            v["primal_violation_at_1e-4"] = {"warm_fp32_matvec": primal_violation(lp, xw, *d0),
                                             "plain_fp64": primal_violation(lp, x64, *d0)}
            # equal answers: both solved to 1e-5, where their objectives agree
            v["equal_answer_1e-5"] = equal_answer_variant(P, WS, lp, inst, net, Xd, layout, stream, 1e-5,
                                                          pending, (xl0, xu0))
        fma64, _ = P.fma_peak(True)
        fma32, _ = P.fma_peak(False)
        v["fma_peak_tflops"] = {"fp64": fma64, "fp32": fma32,
                                "method": "scuc_probe_fma_peak: register-resident FMA chains, CUDA events"}
        lp.set_bounds(xl0, xu0)
        out["roofline"]["all_kernels"].update(
            {k: dict(vv, source="profiled FP64 solve, 256 iterations")
             for k, vv in fp64_kernel_profile(P, lp, m, n, nnz, peak, fma64).items()})
        out["variants"] = v

    if rank == 0 and not args.no_plain:
        # Algorithm 2 for two rounds: the relaxation (as in the step), then per
        # round fix + propagate on the model, solve the reduced LP from the
        # previous point restricted to its columns and rows, map back
        lp.set_bounds(xl0, xu0)
        torch.cuda.synchronize()
        ts = time.perf_counter()
        if warm:
            net.predict(Xd, out=pred)
            WS.assemble(lp, layout, pred, x0=x0)
            first = lp.solve_warm(x0, x_out=xo, y_out=yo, z_out=zo, **kw)["info"]
        else:
            first = lp.solve_device(x_out=xo, y_out=yo, z_out=zo, **kw)
        xs, ys = xo.cpu().numpy(), yo.cpu().numpy()
        rounds = [{"lp": [m, n, nnz], "iters": int(first["iters"]), "status": first["status_name"]}]
        for _ in range(2):
            r = lp.fix_and_propagate(inst.G, inst.T, inst.u_idx, inst.v_idx, inst.w_idx, inst.u_init, xs,
                                     tau=0.1, is_int=inst.is_int)
            red = r["reduced"]
            if red is None:
                rounds.append({"infeasible": bool(r["infeasible"])})
                break
            sr = red.solve(x0=xs[r["col_map"]], y0=ys[r["row_map"]], tol=1e-4, precision=args.precision,
                           time_limit_s=120.0)
            xl_r, _ = lp.get_bounds()
            xs = xl_r.copy()                       # fixed columns at their values
            xs[r["col_map"]] = sr["x"]
            ys = np.zeros(m)
            ys[r["row_map"]] = sr["y"]
            rounds.append({"fixed_triples": int(r["info"]["nfixed"]), "fixed_cols": int(r["info"]["n_fixed_cols"]),
                           "lp": [int(red.m), int(red.n), int(red.nnz)], "iters": int(sr["info"]["iters"]),
                           "status": sr["info"]["status_name"],
                           "pobj": sr["info"]["pobj"] + r["info"]["obj_const"]})
            red.close()
        torch.cuda.synchronize()
        out.setdefault("variants", {})["successive_fixing_2_rounds"] = {
            "s": time.perf_counter() - ts, "rounds": rounds,
            "note": "wall clock: relaxation, then two rounds of fixing + reduced-LP solve from the previous point"}

    if rank == 0 and not args.no_plain:
        out.setdefault("variants", {})["config2_scuc2k"] = config2_variant(P)
        out["variants"]["config3_scuc6k_successive_fixing"] = config3_variant(P, pending)


    if rank == 0 and bv is not None:
        out.setdefault("variants", {})["batched_64"] = bv

    if rank == 0 and not args.no_plain:
        tf = filtering_variant(P, inst, per_step)
        full_pobj = out["variants"].get("cold_mixed_pobj")
        if full_pobj is not None:
            tf["rel_objective_diff_vs_full"] = abs(tf["pobj"] - full_pobj) / max(1.0, abs(full_pobj))
        out["variants"]["transmission_filtering"] = tf

    if not args.no_e2e:
        # through the C ABI from host buffers: create (H2D + device setup), solve, copy back
        ets = []
        ws_h2d = 0
        for rep in range(4):             # one warm-up pass, then three timed ones
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lp2 = P.LP(inst)
            if warm:
                # this step's features and layout from host memory
                Xh = torch.as_tensor(feats).pin_memory().to("cuda", non_blocking=True)
                lay2 = WS.Layout(lay_arrays, WS_FILL)
                p2 = net.predict(Xh)
                x02, _ = WS.assemble(lp2, lay2, p2)
                xd = torch.empty(n, dtype=torch.float64, device="cuda")
                yd = torch.empty(m, dtype=torch.float64, device="cuda")
                zd = torch.empty(n, dtype=torch.float64, device="cuda")
                lp2.solve_warm(x02, x_out=xd, y_out=yd, z_out=zd, tol=1e-4, precision=args.precision,
                               time_limit_s=600.0)
                r = {"x": xd.cpu().numpy(), "y": yd.cpu().numpy(), "z": zd.cpu().numpy()}
                ws_h2d = feats.nbytes + sum(np.asarray(lay_arrays[k]).nbytes for k in
                                            ("u_col", "v_col", "w_col", "p_col", "seg_col", "p_cap", "seg_cap",
                                             "u_init", "unit_price_row", "price_row", "price_ptr",
                                             "price_member"))
            else:
                r = lp2.solve(tol=1e-4, precision=args.precision, time_limit_s=600.0)
            f = lp2.fix_and_propagate(inst.G, inst.T, inst.u_idx, inst.v_idx, inst.w_idx, inst.u_init,
                                      r["x"], tau=0.1, is_int=inst.is_int)
            fix_h = f["fix"]                 # decisions back on the host
            if f["reduced"] is not None:
                f["reduced"].close()
            lp2.close()
            if rep > 0:
                ets.append(time.perf_counter() - t0)
        h2d = 8 * (m + 1) + 12 * nnz + 24 * n + m + 16 * m + 8 * n + 12 * GT + inst.G + n + ws_h2d
        d2h = 16 * n + 8 * m + 3 * GT
        out["e2e"] = {"value": float(np.mean(ets)), "unit": "s", "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": d2h}

    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(inst, step_result)
        # the oracle's FP64 KKT evaluation of the points the variants returned
        import oracle
        for target, key, src, x, y, z in pending:
            k = oracle.kkt(oracle.as_lp(src), x, y, z)
            target[key] = {k2: float(k[k2]) for k2 in ("kkt", "rp", "rd", "gap", "pobj", "dobj")}
        b64 = out.get("variants", {}).get("batched_64")
        if b64 and b64.get("_kkt_refs") and all("kkt" in d for d in b64["_kkt_refs"]):
            b64["oracle_kkt_max"] = max(d["kkt"]["kkt"] for d in b64["_kkt_refs"])
            b64["oracle_kkt_note"] = "the oracle's KKT evaluation of every batched LP's point (rank 0's share)"
        c2 = out.get("variants", {}).get("config2_scuc2k")
        if c2:
            c2["oracle_to_1e-4_s"] = out["cpu_baseline"]["measured_to_tolerance"]["s"]
            c2["oracle_over_gpu_fp64"] = c2["oracle_to_1e-4_s"] / c2["fp64"]["s_to_1e-4"]
    out.pop("_fp64_iters", None); out.pop("_power_iters", None)
    if out.get("variants", {}).get("batched_64") is not None:
        out["variants"]["batched_64"].pop("_kkt_refs", None)
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
