"""CPU oracle (plain FP64) for the HPR LP solve, the fixing strategy and the
bound-propagation presolve.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check of
``__graft_entry__`` and by the CPU-baseline leg of ``bench.py``.  The CUDA
library never imports, links or calls anything here.  The arithmetic lives in
``hpr_oracle.c`` (scalar loops, in the order of the paper's formulas); this
module only compiles it and marshals numpy arrays.  ``tiny_lp`` holds the
exact small-LP solvers (dense simplex, vertex enumeration) that pin it.

Pins (tests/test_oracle_*.py): vertex enumeration and Bland simplex on tiny
LPs, HiGHS (scipy) on mid-size LPs, closed forms (bounds-only LP, fractional
knapsack, merit-order dispatch), eigvalsh for the power method, invariants of
an optimal pair (feasibility, complementary slackness, weak duality), the
O(1/k) envelope of Theorem 1, the scaling equivalence of Sec. 3.A, truth
tables for Round / Algorithm 1, and brute-force enumeration for propagation.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SO_OMP = os.path.join(_HERE, "liboracle_omp.so")
_SRC = os.path.join(_HERE, "hpr_oracle.c")
_lib = None
_lib_omp = None


def _compile(out, extra, force):
    if force or not os.path.exists(out) or os.path.getmtime(out) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "hpr_oracle.h"))):
        tmp = out + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math"] + extra + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no FMA
    contraction): the single-threaded library the tests use, and the same
    source with OpenMP for timing on all host cores."""
    _compile(_SO_OMP, ["-fopenmp"], force)
    return _compile(_SO, [], force)


class OrcLP(C.Structure):
    _fields_ = [("m", C.c_int32), ("n", C.c_int32), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("c", C.c_void_p), ("xl", C.c_void_p), ("xu", C.c_void_p),
                ("lo", C.c_void_p), ("hi", C.c_void_p)]


class OrcParams(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int64), ("check_every", C.c_int32),
                ("use_scaling", C.c_int32), ("sigma0", C.c_double), ("lambda_in", C.c_double),
                ("lambda_safety", C.c_double), ("power_max_iter", C.c_int32),
                ("power_tol", C.c_double), ("power_seed", C.c_uint64),
                ("restart_suff", C.c_double), ("restart_nec", C.c_double),
                ("restart_long", C.c_double), ("log_cap", C.c_int32),
                ("restart_ref", C.c_int32), ("restart_metric", C.c_int32),
                ("sigma_update", C.c_int32), ("algo", C.c_int32), ("infeas_tol", C.c_double)]


class OrcLog(C.Structure):
    _fields_ = [("iter", C.c_int64), ("restart", C.c_int32), ("first", C.c_int32),
                ("rp", C.c_double), ("rd", C.c_double), ("gap", C.c_double),
                ("pobj", C.c_double), ("dobj", C.c_double), ("rho", C.c_double),
                ("sigma", C.c_double), ("rmap", C.c_double)]


class OrcInfo(C.Structure):
    _fields_ = [("iters", C.c_int64), ("status", C.c_int32), ("restarts", C.c_int32),
                ("nlog", C.c_int32), ("power_iters", C.c_int32), ("kkt", C.c_double),
                ("rp", C.c_double), ("rd", C.c_double), ("gap", C.c_double),
                ("pobj", C.c_double), ("dobj", C.c_double), ("lambda_", C.c_double),
                ("sigma", C.c_double), ("beta", C.c_double), ("gamma", C.c_double)]


DEFAULTS = dict(tol=1e-4, max_iter=100000, check_every=64, use_scaling=1, sigma0=1.0,
                lambda_in=0.0, lambda_safety=1.01, power_max_iter=500, power_tol=1e-4,
                power_seed=0x5EED, restart_suff=0.2, restart_nec=0.8, restart_long=0.2,
                log_cap=100000, restart_ref=0, restart_metric=0,
                sigma_update=1, algo=0, infeas_tol=0.0)


def _load(path):
    L = C.CDLL(path)
    L.orc_power_lambda.restype = C.c_double
    L.orc_round.restype = C.c_int32
    L.orc_fix.restype = C.c_int64
    L.orc_propagate.restype = C.c_int32
    L.orc_reduce.restype = C.c_int
    L.orc_hpr_solve.restype = C.c_int
    L.orc_set_threads.restype = C.c_int32
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _load(_SO)
    return _lib


def lib_threads(threads):
    """The OpenMP build with ``threads`` threads (all host cores when 0);
    returns the library and the thread count its loops use."""
    global _lib_omp
    if _lib_omp is None:
        build()
        _lib_omp = _load(_SO_OMP)
    k = int(_lib_omp.orc_set_threads(C.c_int32(int(threads))))
    return _lib_omp, k


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def row_bounds(sense, rhs, rng):
    """Row box [lo, hi] of each sense: G [rhs, inf), L (-inf, rhs], E [rhs, rhs],
    R [rhs, rhs + range]."""
    sense = np.asarray(sense, dtype=np.uint8)
    m = len(sense)
    lo = np.full(m, -np.inf)
    hi = np.full(m, np.inf)
    g = sense == ord("G"); l = sense == ord("L"); e = sense == ord("E"); r = sense == ord("R")
    lo[g] = rhs[g]; hi[l] = rhs[l]; lo[e] = rhs[e]; hi[e] = rhs[e]
    lo[r] = rhs[r]; hi[r] = rhs[r] + rng[r]
    return lo, hi


def as_lp(src) -> dict:
    """Normalise an instance (SCUCInstance or dict with sense/rhs/rng_ or lo/hi)
    into a dict of contiguous arrays with lo/hi."""
    if not isinstance(src, dict):
        src = dict(m=src.m, n=src.n, row_ptr=src.row_ptr, col=src.col, val=src.val, c=src.c,
                   xl=src.xl, xu=src.xu, sense=src.sense, rhs=src.rhs, rng_=src.rng_)
    d = dict(m=int(src["m"]), n=int(src["n"]),
             row_ptr=np.ascontiguousarray(src["row_ptr"], dtype=np.int64),
             col=np.ascontiguousarray(src["col"], dtype=np.int32), val=_f64(src["val"]),
             c=_f64(src["c"]), xl=_f64(src["xl"]), xu=_f64(src["xu"]))
    if "lo" in src:
        d["lo"], d["hi"] = _f64(src["lo"]), _f64(src["hi"])
    else:
        d["lo"], d["hi"] = row_bounds(src["sense"], _f64(src["rhs"]), _f64(src["rng_"]))
    return d


def _struct(d):
    return OrcLP(d["m"], d["n"], _p(d["row_ptr"]), _p(d["col"]), _p(d["val"]), _p(d["c"]),
                 _p(d["xl"]), _p(d["xu"]), _p(d["lo"]), _p(d["hi"]))


def hpr_solve(src, x_init=None, y_init=None, threads=None, **params):
    """Restarted HPR (or PDHG with averaging) on the CPU.  ``threads``: None
    runs the single-threaded oracle; k >= 0 the OpenMP build on k threads
    (0: all host cores), whose norms and dot products add in another order."""
    d = as_lp(src)
    p = dict(DEFAULTS)
    p.update(params)
    L, nthr = (lib(), 1) if threads is None else lib_threads(threads)
    prm = OrcParams(**p)
    x = np.zeros(d["n"]); y = np.zeros(d["m"]); z = np.zeros(d["n"])
    info = OrcInfo()
    log = (OrcLog * max(1, p["log_cap"]))()
    xi = _f64(x_init) if x_init is not None else None
    yi = _f64(y_init) if y_init is not None else None
    L.orc_hpr_solve(C.byref(_struct(d)), C.byref(prm), _p(xi), _p(yi), _p(x), _p(y), _p(z),
                    C.byref(info), log)
    nlog = min(info.nlog, p["log_cap"])
    logs = [dict(iter=log[i].iter, restart=log[i].restart, first=log[i].first, rp=log[i].rp,
                 rd=log[i].rd, gap=log[i].gap, pobj=log[i].pobj, dobj=log[i].dobj,
                 rho=log[i].rho, sigma=log[i].sigma, rmap=log[i].rmap) for i in range(nlog)]
    inf = {f[0].rstrip("_"): getattr(info, f[0]) for f in OrcInfo._fields_}
    inf["threads"] = nthr
    return dict(x=x, y=y, z=z, info=inf, log=logs)


def kkt(src, x, y, z):
    d = as_lp(src)
    out = np.zeros(7)
    lib().orc_kkt(C.byref(_struct(d)), _p(_f64(x)), _p(_f64(y)), _p(_f64(z)), _p(out))
    return dict(rp=out[0], rd=out[1], gap=out[2], pobj=out[3], dobj=out[4], kkt=out[5],
                rmap=out[6])


def scale(src, use_scaling=1):
    d = as_lp(src)
    m, n = d["m"], d["n"]
    Dr, Dc = np.zeros(m), np.zeros(n)
    vs, cs = np.zeros(len(d["val"])), np.zeros(n)
    xls, xus, los, his = np.zeros(n), np.zeros(n), np.zeros(m), np.zeros(m)
    beta, gamma = C.c_double(), C.c_double()
    lib().orc_scale(C.byref(_struct(d)), C.c_int32(use_scaling), _p(Dr), _p(Dc), C.byref(beta),
                    C.byref(gamma), _p(vs), _p(cs), _p(xls), _p(xus), _p(los), _p(his))
    return dict(Dr=Dr, Dc=Dc, beta=beta.value, gamma=gamma.value, val=vs, c=cs, xl=xls, xu=xus,
                lo=los, hi=his)


def power_lambda(m, n, row_ptr, col, val, max_iter=500, tol=1e-4, seed=0x5EED):
    it = C.c_int32()
    lam = lib().orc_power_lambda(C.c_int32(m), C.c_int32(n),
                                 _p(np.ascontiguousarray(row_ptr, dtype=np.int64)),
                                 _p(np.ascontiguousarray(col, dtype=np.int32)), _p(_f64(val)),
                                 C.c_int32(max_iter), C.c_double(tol), C.c_uint64(seed),
                                 C.byref(it))
    return lam, it.value


def round_(s, tau):
    return int(lib().orc_round(C.c_double(s), C.c_double(tau)))


def fix(G, T, u, v, w, u_init, tau, t_first=1):
    out = np.full(3 * G * T, -1, dtype=np.int8)
    ui = np.ascontiguousarray(u_init, dtype=np.int8)
    nf = lib().orc_fix(C.c_int32(G), C.c_int32(T), _p(_f64(u)), _p(_f64(v)), _p(_f64(w)),
                       _p(ui), C.c_double(tau), C.c_int32(t_first), _p(out))
    return out, int(nf)


def propagate(src, xl, xu, is_int, max_passes=100):
    d = as_lp(src)
    xl = _f64(xl).copy(); xu = _f64(xu).copy()
    ii = np.ascontiguousarray(is_int, dtype=np.uint8)
    r = lib().orc_propagate(C.c_int32(d["m"]), C.c_int32(d["n"]), _p(d["row_ptr"]), _p(d["col"]),
                            _p(d["val"]), _p(d["lo"]), _p(d["hi"]), _p(xl), _p(xu), _p(ii),
                            C.c_int32(max_passes))
    return xl, xu, int(r)


def reduce(src, xl, xu):
    d = as_lp(src)
    m, n, nnz = d["m"], d["n"], len(d["val"])
    dims = np.zeros(3, dtype=np.int64)
    rp = np.zeros(m + 1, dtype=np.int64); col = np.zeros(max(nnz, 1), dtype=np.int32)
    val = np.zeros(max(nnz, 1)); c = np.zeros(n); lo = np.zeros(m); hi = np.zeros(m)
    xlr = np.zeros(n); xur = np.zeros(n)
    rmap = np.zeros(max(m, 1), dtype=np.int32); cmap = np.zeros(max(n, 1), dtype=np.int32)
    oc = C.c_double()
    bad = lib().orc_reduce(C.c_int32(m), C.c_int32(n), _p(d["row_ptr"]), _p(d["col"]),
                           _p(d["val"]), _p(d["c"]), _p(d["lo"]), _p(d["hi"]), _p(_f64(xl)),
                           _p(_f64(xu)), _p(dims), _p(rp), _p(col), _p(val), _p(c), _p(lo),
                           _p(hi), _p(xlr), _p(xur), _p(rmap), _p(cmap), C.byref(oc))
    mr, nr, kr = (int(v) for v in dims)
    red = dict(m=mr, n=nr, row_ptr=rp[:mr + 1].copy(), col=col[:kr].copy(), val=val[:kr].copy(),
               c=c[:nr].copy(), lo=lo[:mr].copy(), hi=hi[:mr].copy(), xl=xlr[:nr].copy(),
               xu=xur[:nr].copy())
    return red, rmap[:mr].copy(), cmap[:nr].copy(), oc.value, int(bad)


# ---------------------------------------------------------------------------
# Transmission filtering (Fig. 1): solve without the network security rows,
# add the violated ones, re-solve from the previous point, until none is
# violated.  Plain definitions on the unscaled LP.
# ---------------------------------------------------------------------------
def row_violations(pool, x, tol):
    """Rows i of ``pool`` violated at x: lo_i - a_i x > tol (1 + |lo_i|) or
    a_i x - hi_i > tol (1 + |hi_i|).  Returns the row indices (ascending) and
    the largest relative violation (0 when none)."""
    d = as_lp(pool)
    import scipy.sparse as sp
    A = sp.csr_matrix((d["val"], d["col"], d["row_ptr"]), shape=(d["m"], d["n"]))
    ax = A @ _f64(x)
    rows, worst = [], 0.0
    for i in range(d["m"]):
        lo, hi = d["lo"][i], d["hi"][i]
        v = 0.0
        if np.isfinite(lo) and lo - ax[i] > 0.0:
            v = (lo - ax[i]) / (1.0 + abs(lo))
        if np.isfinite(hi) and ax[i] - hi > 0.0:
            v = max(v, (ax[i] - hi) / (1.0 + abs(hi)))
        if v > tol:
            rows.append(i)
        worst = max(worst, v)
    return np.asarray(rows, dtype=np.int32), worst


def add_rows(base, pool, rows):
    """The LP with base's rows followed by pool rows ``rows`` (in that order);
    columns, costs and bounds are base's."""
    b, p = as_lp(base), as_lp(pool)
    rows = np.asarray(rows, dtype=np.int64)
    lens = p["row_ptr"][rows + 1] - p["row_ptr"][rows]
    rp = np.concatenate([b["row_ptr"], b["row_ptr"][-1] + np.cumsum(lens)]).astype(np.int64)
    col = np.concatenate([b["col"]] + [p["col"][p["row_ptr"][r]:p["row_ptr"][r + 1]] for r in rows])
    val = np.concatenate([b["val"]] + [p["val"][p["row_ptr"][r]:p["row_ptr"][r + 1]] for r in rows])
    return dict(m=b["m"] + len(rows), n=b["n"], row_ptr=rp, col=col.astype(np.int32), val=val,
                c=b["c"].copy(), xl=b["xl"].copy(), xu=b["xu"].copy(),
                lo=np.concatenate([b["lo"], p["lo"][rows]]), hi=np.concatenate([b["hi"], p["hi"][rows]]))


def transmission_filter(base, pool, viol_tol=1e-6, max_rounds=20, **params):
    """Solve base, then repeatedly add the pool rows violated by the solution
    (each at most once) and re-solve from the previous (x, y) with y = 0 on
    the new rows, until no violated pool row is outside the LP (Fig. 1).
    Returns the last LP, its solve and the rounds."""
    lp, x, y = as_lp(base), None, None
    added = np.zeros(as_lp(pool)["m"], dtype=bool)
    rounds, order = [], []
    for _ in range(max_rounds):
        r = hpr_solve(lp, x_init=x, y_init=y, **params)
        viol, worst = row_violations(pool, r["x"], viol_tol)
        new = viol[~added[viol]]
        rounds.append(dict(m=lp["m"], iters=r["info"]["iters"], status=r["info"]["status"], violated=len(viol),
                           added=len(new), max_violation=worst))
        if len(new) == 0:
            # every violated pool row is already in the LP, which holds it to
            # the solve's own tolerance: no round can add anything
            return dict(lp=lp, result=r, rounds=rounds, converged=True, violated_in_model=len(viol),
                        rows_added=np.asarray(order, dtype=np.int32))
        added[new] = True
        order.extend(new.tolist())
        lp = add_rows(lp, pool, new)
        x, y = r["x"], np.concatenate([r["y"], np.zeros(len(new))])
    return dict(lp=lp, result=r, rounds=rounds, converged=False, violated_in_model=int(np.sum(added[viol])),
                rows_added=np.asarray(order, dtype=np.int32))
