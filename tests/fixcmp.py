"""Comparison of propagated bounds and folded row bounds (the presolve of
Algorithm 2, Sec. 4.2) between the GPU and the oracle.

The oracle sums each row's terms in entry order; the GPU sums them in
another fixed order.  Two orders of the same FP64 sum of L terms t_k differ
by at most 2 gamma_L sum |t_k| with gamma_L = L u / (1 - L u), u = 2^-53
(each lies within gamma_L sum |t_k| of the exact sum).  Hence:

* a folded row bound lo_i - sum_{k fixed} a_ik x_k differs by at most
  2 gamma_L sum_{k fixed} |a_ik x_k| + 2 u |result|;
* a candidate bound (hi_i - rest) / a_ij, rest = an activity over the row's
  other columns, differs by at most (2 gamma_L S_i + 2 u |hi_i|) / |a_ij|
  + 2 u |candidate|, S_i = sum_k |a_ik| m_k with m_k the largest finite
  bound magnitude column k takes; the differences of one pass enter the
  next pass's activities, so the tolerance is taken per pass and summed
  over the passes.

Integer results are compared exactly: integer bounds, the fixed-column and
kept-row sets, and the reduced matrix structure.  A difference there needs a
rounding tie (a candidate within the tolerance above of an integer
threshold or of a row bound); the tests report the offending entries."""
from __future__ import annotations

import numpy as np

U = 2.0 ** -53


def _gamma(L):
    L = np.asarray(L, dtype=np.float64)
    return L * U / (1.0 - L * U)


def _finite_mag(*arrs):
    m = np.zeros_like(np.asarray(arrs[0], dtype=np.float64))
    for a in arrs:
        a = np.asarray(a, dtype=np.float64)
        m = np.maximum(m, np.where(np.isfinite(a), np.abs(a), 0.0))
    return m


def column_bound_tolerance(d, bound_sets, passes):
    """Per column: the largest candidate-bound difference the summation order
    can make over ``passes`` Jacobi passes (see the module docstring).
    ``bound_sets``: the bound arrays the columns took (initial and final)."""
    m, n = d["m"], d["n"]
    rp, col, val = d["row_ptr"], d["col"], d["val"]
    mk = _finite_mag(*bound_sets)
    lens = np.diff(rp)
    rows = np.repeat(np.arange(m), lens)
    S = np.zeros(m)
    np.add.at(S, rows, np.abs(val) * mk[col])
    rb = _finite_mag(d["lo"], d["hi"])
    per_row = 2.0 * _gamma(np.maximum(lens, 1)) * S + 2.0 * U * rb
    e = per_row[rows] / np.abs(val)
    tol = np.zeros(n)
    np.maximum.at(tol, col, e)
    return max(int(passes), 1) * tol


def assert_bounds_match(d, is_int, g_lo, g_hi, o_lo, o_hi, passes, initial):
    """GPU bounds (g_*) against the oracle's (o_*): integer columns and
    infinite bounds exactly, finite continuous bounds within the tolerance."""
    is_int = np.asarray(is_int).astype(bool)
    tol = column_bound_tolerance(d, [initial[0], initial[1], o_lo, o_hi], passes)
    for name, g, o in (("xl", g_lo, o_lo), ("xu", g_hi, o_hi)):
        g = np.asarray(g); o = np.asarray(o)
        bad = is_int & (g != o)
        assert not bad.any(), "%s: integer columns differ at %s" % (name, np.flatnonzero(bad)[:10])
        fin = np.isfinite(o)
        assert np.array_equal(np.isfinite(g), fin), "%s: infinite bounds differ" % name
        assert np.array_equal(np.sign(g[~fin]), np.sign(o[~fin]))
        err = np.abs(g[fin] - o[fin]) - (tol[fin] + 2.0 * U * np.abs(o[fin]))
        assert (err <= 0).all(), "%s: columns %s differ beyond the bound: gpu %s oracle %s tol %s" % (
            name, np.flatnonzero(fin)[err > 0][:5], g[fin][err > 0][:5], o[fin][err > 0][:5],
            tol[fin][err > 0][:5])
    # the fixed columns (equal bounds) are the same set
    gf = np.asarray(g_lo) == np.asarray(g_hi)
    of = np.asarray(o_lo) == np.asarray(o_hi)
    assert np.array_equal(gf, of), "fixed columns differ at %s" % np.flatnonzero(gf != of)[:10]


def folded_row_tolerance(d, row_map, xl_fixed, fixed):
    """Per kept row: the largest difference the order of the fixed-column
    shift can make in its folded bounds."""
    rp, col, val = d["row_ptr"], d["col"], d["val"]
    lens = np.diff(rp)
    rows = np.repeat(np.arange(d["m"]), lens)
    t = np.where(fixed[col], np.abs(val * xl_fixed[col]), 0.0)
    T = np.zeros(d["m"])
    np.add.at(T, rows, t)
    return (2.0 * _gamma(np.maximum(lens, 1)) * T)[row_map]


def assert_reduced_match(d, g, red, row_map, col_map, g_lo, g_hi, o_lo, o_hi):
    """Reduced LP from the GPU (exported dict g) against the oracle's reduce
    of its own bounds (red): structure, values and costs exactly; the column
    bounds are the GPU's propagated bounds of the kept columns (compared with
    the oracle's by assert_bounds_match); folded row bounds within the bound
    of the fixed-column shift's order."""
    for k in ("row_ptr", "col", "val", "c"):
        np.testing.assert_array_equal(g[k], red[k], err_msg=k)
    np.testing.assert_array_equal(g["xl"], np.asarray(g_lo)[col_map])
    np.testing.assert_array_equal(g["xu"], np.asarray(g_hi)[col_map])
    fixed = np.asarray(o_lo) == np.asarray(o_hi)
    tol = folded_row_tolerance(d, row_map, np.asarray(o_lo), fixed)
    for k in ("lo", "hi"):
        a, b = np.asarray(g[k]), np.asarray(red[k])
        fin = np.isfinite(b)
        assert np.array_equal(np.isfinite(a), fin), k
        assert np.array_equal(a[~fin], b[~fin]), k
        err = np.abs(a[fin] - b[fin]) - (tol[fin] + 2.0 * U * np.abs(b[fin]))
        assert (err <= 0).all(), "%s: rows %s differ beyond the bound" % (k, np.flatnonzero(fin)[err > 0][:5])


def propagation_case(seed, m=120, n=80):
    """A random LP around an integral point x* (integer columns integral,
    integer boxes; rows x* satisfies with small slack) with half its columns
    integer: propagation is feasible (it is sound and x* is feasible) and
    tightens bounds.  Returns the LP (lo/hi form) and the integer flags."""
    from scuc_gen import random_lp
    d = random_lp(m, n, density=0.05, seed=seed, long_rows=2)
    rng = np.random.default_rng(1000 + seed)
    is_int = rng.random(n) < 0.5
    xs = np.where(is_int, rng.integers(-3, 4, size=n), rng.uniform(-3, 3, size=n)).astype(np.float64)
    xl = xs - rng.uniform(0.5, 3.0, size=n)
    xu = xs + rng.uniform(0.5, 3.0, size=n)
    xl[is_int] = np.floor(xl[is_int]); xu[is_int] = np.ceil(xu[is_int])
    free = rng.random(n) < 0.1
    xl[free & ~is_int] = -np.inf
    rp, col, val = d["row_ptr"], d["col"], d["val"]
    ax = np.array([val[rp[i]:rp[i + 1]] @ xs[col[rp[i]:rp[i + 1]]] for i in range(m)])
    slack = rng.uniform(0.05, 1.0, size=(2, m))
    kind = rng.integers(0, 3, size=m)          # 0: >=, 1: <=, 2: both
    lo = np.where(kind != 1, ax - slack[0], -np.inf)
    hi = np.where(kind != 0, ax + slack[1], np.inf)
    out = dict(m=m, n=n, row_ptr=rp, col=col, val=val, c=d["c"], xl=xl, xu=xu, lo=lo, hi=hi)
    return out, is_int.astype(np.uint8)
