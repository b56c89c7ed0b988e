"""Python face of the C ABI (argument marshalling only; every step of the
solve runs in the CUDA library)."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def default_params(**kw) -> L.SolveParams:
    p = L.SolveParams()
    L.lib().scuc_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": L.FP64, "mixed": L.MIXED}[v]
        if k == "algo" and isinstance(v, str):
            v = L.ALGO[v]
        if not hasattr(p, k):
            raise TypeError("unknown solve parameter %r" % k)
        setattr(p, k, v)
    return p


def info_dict(info: L.SolveInfo) -> dict:
    d = {f[0].rstrip("_"): getattr(info, f[0]) for f in L.SolveInfo._fields_}
    d["status_name"] = L.STATUS.get(d["status"], "?")
    return d


class LP:
    """An LP  min c^T x, lo <= A x <= hi, xl <= x <= xu  resident on the GPU.

    ``src`` is a SCUCInstance or a dict with m, n, row_ptr, col, val, c, xl, xu
    and either (sense, rhs, rng_) or (lo, hi).  ``stream`` is a raw
    cudaStream_t value (e.g. ``torch.cuda.current_stream().cuda_stream``)."""

    def __init__(self, src, stream: int | None = None):
        if not isinstance(src, dict):
            src = dict(m=src.m, n=src.n, row_ptr=src.row_ptr, col=src.col, val=src.val, c=src.c,
                       xl=src.xl, xu=src.xu, sense=src.sense, rhs=src.rhs, rng_=src.rng_)
        self.m, self.n = int(src["m"]), int(src["n"])
        rp = np.ascontiguousarray(src["row_ptr"], dtype=np.int64)
        col = np.ascontiguousarray(src["col"], dtype=np.int32)
        val = _f64(src["val"])
        c, xl, xu = _f64(src["c"]), _f64(src["xl"]), _f64(src["xu"])
        self.nnz = int(rp[-1])
        h = C.c_void_p()
        st = C.c_void_p(stream) if stream else None
        if "lo" in src:
            lo, hi = _f64(src["lo"]), _f64(src["hi"])
            L.check(L.lib().scuc_lp_create_box(C.byref(h), self.m, self.n, self.nnz, _ptr(rp),
                                               _ptr(col), _ptr(val), _ptr(c), _ptr(xl), _ptr(xu),
                                               _ptr(lo), _ptr(hi), st))
        else:
            sense = np.ascontiguousarray(src["sense"], dtype=np.uint8)
            rhs, rng = _f64(src["rhs"]), _f64(src["rng_"])
            L.check(L.lib().scuc_lp_create(C.byref(h), self.m, self.n, self.nnz, _ptr(rp), _ptr(col),
                                           _ptr(val), _ptr(c), _ptr(xl), _ptr(xu), _ptr(sense),
                                           _ptr(rhs), _ptr(rng), st))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            L.lib().scuc_lp_destroy(self.h)
            self.h = None

    __del__ = close

    def solve(self, x0=None, y0=None, want=("x", "y", "z"), **params) -> dict:
        """Host-buffer solve: returns x, y, z (numpy), info and the check log."""
        p = default_params(**params)
        p.device_ptrs = 0
        out = {k: np.zeros(self.n if k in ("x", "z") else self.m) for k in want}
        info = L.SolveInfo()
        L.check(L.lib().scuc_lp_solve(self.h, C.byref(p),
                                      _ptr(_f64(x0)) if x0 is not None else None,
                                      _ptr(_f64(y0)) if y0 is not None else None,
                                      _ptr(out.get("x")), _ptr(out.get("y")), _ptr(out.get("z")),
                                      C.byref(info)))
        out["info"] = info_dict(info)
        out["log"] = self.log(info.nlog)
        return out

    def solve_device(self, x_out=None, y_out=None, z_out=None, x0=None, y0=None, **params) -> dict:
        """Device-buffer solve: arguments are torch CUDA float64 tensors (or None)."""
        p = default_params(**params)
        p.device_ptrs = 1
        dp = lambda t: None if t is None else C.c_void_p(t.data_ptr())
        info = L.SolveInfo()
        L.check(L.lib().scuc_lp_solve(self.h, C.byref(p), dp(x0), dp(y0), dp(x_out), dp(y_out),
                                      dp(z_out), C.byref(info)))
        return info_dict(info)

    def solve_warm(self, x0, y0=None, warm_max_iter=0, first_check=1, cold_first_kkt=0.0,
                   x_out=None, y_out=None, z_out=None, **params) -> dict:
        """Warm solve with cold start as the fallback (scuc_lp_solve_warm).
        x0/y0 and the outputs are torch CUDA float64 tensors (device) or numpy
        arrays (host; then the outputs are returned in the dict)."""
        p = default_params(**params)
        info = L.SolveInfo()
        wp = L.WarmParams()
        wp.warm_max_iter, wp.first_check, wp.cold_first_kkt = int(warm_max_iter), int(first_check), float(cold_first_kkt)
        if hasattr(x0, "data_ptr"):
            p.device_ptrs = 1
            dp = lambda t: None if t is None else C.c_void_p(t.data_ptr())
            L.check(L.lib().scuc_lp_solve_warm(self.h, C.byref(p), dp(x0), dp(y0), C.byref(wp),
                                               dp(x_out), dp(y_out), dp(z_out), C.byref(info)))
            return {"info": info_dict(info)}
        p.device_ptrs = 0
        out = {k: np.zeros(self.n if k in ("x", "z") else self.m) for k in ("x", "y", "z")}
        L.check(L.lib().scuc_lp_solve_warm(self.h, C.byref(p), _ptr(_f64(x0)),
                                           _ptr(_f64(y0)) if y0 is not None else None,
                                           C.byref(wp), _ptr(out["x"]), _ptr(out["y"]),
                                           _ptr(out["z"]), C.byref(info)))
        out["info"] = info_dict(info)
        return out

    def log(self, cap=None) -> list:
        cap = 4096 if cap is None else max(0, int(cap))
        buf = (L.CheckLog * max(cap, 1))()
        cnt = C.c_int32()
        L.check(L.lib().scuc_lp_get_log(self.h, buf, cap, C.byref(cnt)))
        return [{f[0]: getattr(buf[i], f[0]) for f in L.CheckLog._fields_ if f[0] != "pad"}
                for i in range(cnt.value)]

    def matvec(self, inp, out, transpose=False):
        """out = A inp (or A^T inp) on torch CUDA float64 tensors."""
        L.check(L.lib().scuc_lp_matvec(self.h, 1 if transpose else 0, C.c_void_p(inp.data_ptr()),
                                       C.c_void_p(out.data_ptr())))
        return out

    # ----- transmission filtering (Fig. 1) -----

    def row_violations(self, x, tol=1e-6, cap=None):
        """Rows of this LP (a pool of candidate rows) violated at x (numpy
        array, or torch CUDA float64 tensor): (row indices ascending, largest
        relative violation)."""
        cap = self.m if cap is None else int(cap)
        out = np.zeros(max(cap, 1), dtype=np.int32)
        cnt, worst = C.c_int32(), C.c_double()
        on_dev = not isinstance(x, np.ndarray)
        xp = C.c_void_p(x.data_ptr()) if on_dev else _ptr(_f64(x))
        L.check(L.lib().scuc_lp_row_violations(self.h, xp, 1 if on_dev else 0, float(tol),
                                               C.c_void_p(out.ctypes.data), cap, C.byref(cnt), C.byref(worst)))
        return out[:min(cnt.value, cap)].copy(), worst.value

    def add_rows(self, pool: "LP", rows) -> "LP":
        """A new LP: this LP's rows followed by the pool rows ``rows``."""
        r = np.ascontiguousarray(rows, dtype=np.int32)
        h = C.c_void_p()
        L.check(L.lib().scuc_lp_add_rows(self.h, pool.h, C.c_void_p(r.ctypes.data) if len(r) else None,
                                         len(r), C.byref(h)))
        return LP._adopt(h)

    # ----- fixing + presolve (Sec. 4.1-4.2) -----

    @classmethod
    def _adopt(cls, h):
        self = cls.__new__(cls)
        self.h = h
        m, n, nnz = C.c_int32(), C.c_int32(), C.c_int64()
        L.check(L.lib().scuc_lp_dims(h, C.byref(m), C.byref(n), C.byref(nnz)))
        self.m, self.n, self.nnz = m.value, n.value, nnz.value
        return self

    def set_index16(self, on):
        """scuc_lp_set_index16: 16-bit index offsets in FP32 products (before
        the first solve)."""
        L.check(L.lib().scuc_lp_set_index16(self.h, int(bool(on))))

    def layout(self):
        """Storage of the entries the FP32 iteration products read
        (scuc_lp_layout), valid after the first solve with FP32 products."""
        out = (C.c_int64 * 8)()
        L.check(L.lib().scuc_lp_layout(self.h, out))
        keys = ("a_chunk16", "a_chunk32", "a_sell", "t_sell", "t_sell_compressed", "t_sell_lanes",
                "t_chunk16", "t_chunk32")
        return {k: int(v) for k, v in zip(keys, out)}

    def fix_and_propagate(self, G, T, u_idx, v_idx, w_idx, u_init, x, tau=0.1, t_first=1,
                          max_passes=100, is_int=None, build_reduced=True):
        """One fixing round (Round + Algorithm 1, propagation, reduced LP).
        x: numpy array (host) or torch CUDA float64 tensor.  Updates this LP's
        bounds; returns fix (int8 [3*G*T]), the reduced LP (or None), maps and info."""
        keep = [np.ascontiguousarray(a, dtype=np.int32) for a in (u_idx, v_idx, w_idx)]
        ui = np.ascontiguousarray(u_init, dtype=np.int8)
        mp = L.ScucMap(int(G), int(T), keep[0].ctypes.data, keep[1].ctypes.data, keep[2].ctypes.data,
                       ui.ctypes.data)
        p = L.FixParams()
        L.lib().scuc_default_fix_params(C.byref(p))
        p.tau, p.t_first, p.max_passes = float(tau), int(t_first), int(max_passes)
        p.build_reduced = 1 if build_reduced else 0
        if isinstance(x, np.ndarray):
            xa = _f64(x)
            xp = C.c_void_p(xa.ctypes.data)
            p.x_on_device = 0
        else:
            xp = C.c_void_p(x.data_ptr())
            p.x_on_device = 1
        ii = None if is_int is None else np.ascontiguousarray(is_int, dtype=np.uint8)
        fix = np.full(3 * int(G) * int(T), -1, dtype=np.int8)
        cmap = np.zeros(max(self.n, 1), dtype=np.int32)
        rmap = np.zeros(max(self.m, 1), dtype=np.int32)
        red = C.c_void_p()
        info = L.FixInfo()
        rc = L.lib().scuc_fix_and_propagate(self.h, C.byref(mp), _ptr(ii), xp, C.byref(p),
                                            C.c_void_p(fix.ctypes.data),
                                            C.byref(red) if build_reduced else None,
                                            C.c_void_p(cmap.ctypes.data), C.c_void_p(rmap.ctypes.data),
                                            C.byref(info))
        d = {f[0]: getattr(info, f[0]) for f in L.FixInfo._fields_}
        if rc == L.SCUC_E_INFEASIBLE:
            return dict(fix=fix, reduced=None, col_map=None, row_map=None, info=d, infeasible=True)
        L.check(rc)
        out = dict(fix=fix, info=d, infeasible=False, col_map=cmap[:d["n_red"]].copy(),
                   row_map=rmap[:d["m_red"]].copy(), reduced=None)
        if build_reduced and red.value:
            out["reduced"] = LP._adopt(red)
        return out

    def get_bounds(self):
        xl, xu = np.zeros(self.n), np.zeros(self.n)
        L.check(L.lib().scuc_lp_get_bounds(self.h, C.c_void_p(xl.ctypes.data), C.c_void_p(xu.ctypes.data)))
        return xl, xu

    def set_bounds(self, xl, xu):
        xl, xu = _f64(xl), _f64(xu)
        L.check(L.lib().scuc_lp_set_bounds(self.h, C.c_void_p(xl.ctypes.data), C.c_void_p(xu.ctypes.data), 0))

    def export(self) -> dict:
        """The LP as host arrays (unscaled): row_ptr, col, val, c, xl, xu, lo, hi."""
        m, n, nnz = self.m, self.n, self.nnz
        d = dict(m=m, n=n, row_ptr=np.zeros(m + 1, np.int64), col=np.zeros(max(nnz, 1), np.int32),
                 val=np.zeros(max(nnz, 1)), c=np.zeros(max(n, 1)), xl=np.zeros(max(n, 1)),
                 xu=np.zeros(max(n, 1)), lo=np.zeros(max(m, 1)), hi=np.zeros(max(m, 1)))
        L.check(L.lib().scuc_lp_export(self.h, *[C.c_void_p(d[k].ctypes.data) for k in
                                                 ("row_ptr", "col", "val", "c", "xl", "xu", "lo", "hi")]))
        for k, ln in (("col", nnz), ("val", nnz), ("c", n), ("xl", n), ("xu", n), ("lo", m), ("hi", m)):
            d[k] = d[k][:ln]
        return d


def solve_batch(lps, outputs=None, autotune=True, **params):
    """Solve the LPs together (scuc_lp_solve_batch).

    ``outputs``: None (host solutions are returned), or a list with one
    (x, y, z) tuple of torch CUDA float64 tensors (entries may be None) per
    LP.  Returns (per-LP result dicts, batch info dict); with host outputs
    each result dict carries x, y and z."""
    p = default_params(**params)
    cnt = len(lps)
    hs = (C.c_void_p * max(cnt, 1))(*[lp.h for lp in lps])
    infos = (L.SolveInfo * max(cnt, 1))()
    bi = L.BatchInfo()
    bi.autotune = 1 if autotune else 0
    ptr3 = [(C.c_void_p * max(cnt, 1))() for _ in range(3)]
    host = None
    if outputs is None:
        p.device_ptrs = 0
        host = [(np.zeros(lp.n), np.zeros(lp.m), np.zeros(lp.n)) for lp in lps]
        for i, (x, y, z) in enumerate(host):
            ptr3[0][i], ptr3[1][i], ptr3[2][i] = x.ctypes.data, y.ctypes.data, z.ctypes.data
    else:
        p.device_ptrs = 1
        for i, trip in enumerate(outputs):
            for k, t in enumerate(trip):
                ptr3[k][i] = None if t is None else t.data_ptr()
    L.check(L.lib().scuc_lp_solve_batch(hs, cnt, C.byref(p), ptr3[0], ptr3[1], ptr3[2], infos, C.byref(bi)))
    res = []
    for i in range(cnt):
        d = {"info": info_dict(infos[i])}
        if host is not None:
            d["x"], d["y"], d["z"] = host[i]
        res.append(d)
    return res, {f[0]: getattr(bi, f[0]) for f in L.BatchInfo._fields_}


def fma_peak(fp64=True):
    """Measured FMA throughput of the current device in TFLOP/s
    (scuc_probe_fma_peak): FP64 (DFMA) or FP32.  Returns (tflops, ms)."""
    t, ms = C.c_double(), C.c_double()
    L.check(L.lib().scuc_probe_fma_peak(1 if fp64 else 0, C.byref(t), C.byref(ms)))
    return t.value, ms.value
