"""Exact solvers for tiny LPs that pin the HPR oracle (test infrastructure).

Both take the LP  min c^T x  s.t.  lo <= A x <= hi,  xl <= x <= xu  with
dense A and *finite* column bounds (so the feasible set is a polytope and
the optimum, if any, is attained at a vertex).

* ``vertex_enum``: brute force over every choice of n linearly independent
  active constraints; keeps the feasible basic solutions; returns the best.
* ``bland_simplex``: textbook two-phase tableau simplex with Bland's
  smallest-index rule (no cycling), on the standard form obtained by
  shifting x = xl + s, s + t = xu - xl, and one slack per finite row bound.
"""
from __future__ import annotations

import itertools

import numpy as np


def _constraints(A, lo, hi, xl, xu):
    """All finite inequalities as G x <= h."""
    m, n = A.shape
    G, h = [], []
    for i in range(m):
        if np.isfinite(hi[i]):
            G.append(A[i]); h.append(hi[i])
        if np.isfinite(lo[i]):
            G.append(-A[i]); h.append(-lo[i])
    for j in range(n):
        e = np.zeros(n); e[j] = 1.0
        G.append(e); h.append(xu[j])
        G.append(-e); h.append(-xl[j])
    return np.array(G), np.array(h)


def vertex_enum(A, lo, hi, c, xl, xu, tol=1e-9):
    A = np.atleast_2d(np.asarray(A, dtype=float))
    n = len(c)
    if A.size == 0:
        A = np.zeros((0, n))
    G, h = _constraints(A, lo, hi, xl, xu)
    best, bestx = np.inf, None
    for act in itertools.combinations(range(len(h)), n):
        M = G[list(act)]
        if abs(np.linalg.det(M)) < 1e-12:
            continue
        x = np.linalg.solve(M, h[list(act)])
        if np.all(G @ x <= h + tol * (1 + np.abs(h))):
            f = float(c @ x)
            if f < best - 1e-12:
                best, bestx = f, x
    return best, bestx


def bland_simplex(A, lo, hi, c, xl, xu, tol=1e-10, max_pivots=100000):
    """Returns (objective, x) or (None, None) when infeasible."""
    A = np.atleast_2d(np.asarray(A, dtype=float))
    n = len(c)
    if A.size == 0:
        A = np.zeros((0, n))
    m = A.shape[0]
    xl = np.asarray(xl, float); xu = np.asarray(xu, float)
    # variables: s (n, x = xl + s), t (n, s + t = xu - xl), slacks (one per finite row side)
    rows, rhs = [], []
    nslack = sum(int(np.isfinite(hi[i])) + int(np.isfinite(lo[i])) for i in range(m))
    nv = 2 * n + nslack
    k = 0
    for i in range(m):
        base = float(A[i] @ xl)
        if np.isfinite(hi[i]):  # A s + slack = hi - A xl
            r = np.zeros(nv); r[:n] = A[i]; r[2 * n + k] = 1.0; k += 1
            rows.append(r); rhs.append(hi[i] - base)
        if np.isfinite(lo[i]):  # A s - slack = lo - A xl
            r = np.zeros(nv); r[:n] = A[i]; r[2 * n + k] = -1.0; k += 1
            rows.append(r); rhs.append(lo[i] - base)
    for j in range(n):
        r = np.zeros(nv); r[j] = 1.0; r[n + j] = 1.0
        rows.append(r); rhs.append(xu[j] - xl[j])
    Aeq = np.array(rows); b = np.array(rhs)
    neg = b < 0
    Aeq[neg] *= -1.0; b[neg] *= -1.0
    me = Aeq.shape[0]
    cost = np.zeros(nv); cost[:n] = c

    # phase 1 with artificials
    T = np.zeros((me + 1, nv + me + 1))
    T[:me, :nv] = Aeq
    T[:me, nv:nv + me] = np.eye(me)
    T[:me, -1] = b
    basis = list(range(nv, nv + me))

    def pivot(r, q):
        T[r] /= T[r, q]
        for i in range(T.shape[0]):
            if i != r and T[i, q] != 0.0:
                T[i] -= T[i, q] * T[r]
        basis[r] = q

    def run(obj_row_cost, allowed):
        # reduced costs row = cost - c_B B^-1 A
        T[-1, :] = 0.0
        T[-1, :len(obj_row_cost)] = obj_row_cost
        for r, q in enumerate(basis):
            if T[-1, q] != 0.0:
                T[-1] -= T[-1, q] * T[r]
        for _ in range(max_pivots):
            q = next((j for j in allowed if T[-1, j] < -tol), None)   # Bland: smallest index
            if q is None:
                return True
            ratios = [(T[r, -1] / T[r, q], basis[r], r) for r in range(me) if T[r, q] > tol]
            if not ratios:
                return False  # unbounded (cannot happen with finite boxes)
            best = min(rt[0] for rt in ratios)
            r = min((rt for rt in ratios if rt[0] <= best + tol), key=lambda rt: rt[1])[2]
            pivot(r, q)
        raise RuntimeError("pivot limit")

    c1 = np.zeros(nv + me); c1[nv:] = 1.0
    run(c1, list(range(nv + me)))
    if -T[-1, -1] > 1e-7 * (1 + np.abs(b).sum()):
        return None, None
    # drive artificials out of the basis where possible
    for r in range(me):
        if basis[r] >= nv:
            q = next((j for j in range(nv) if abs(T[r, j]) > tol), None)
            if q is not None:
                pivot(r, q)
    c2 = np.zeros(nv + me); c2[:nv] = cost
    ok = run(c2, list(range(nv)))
    if not ok:
        return -np.inf, None
    sol = np.zeros(nv + me)
    for r, q in enumerate(basis):
        sol[q] = T[r, -1]
    x = xl + sol[:n]
    return float(c @ x), x
