"""Pins of the oracle's Round / Algorithm 1 (Sec. 4.1) and of the bound
propagation + reduction that stands in for MILP-/LP-Presolve (Sec. 4.2)."""
import itertools
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import linprog

import oracle
from scuc_gen import make_preset

GOLD = os.path.join(os.path.dirname(__file__), "golden", "round_alg1.txt")


def _golden():
    rounds, algs = [], []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        if f[0] == "round":
            rounds.append((float(f[1]), float(f[2]), int(f[3])))
        else:
            T, tau = int(f[1]), float(f[2])
            body, mask = line.split("->")
            parts = body.split()[3:]
            vals = [p for p in parts if p != "|"]
            u = np.array(vals[:T], float); v = np.array(vals[T:2 * T], float)
            w = np.array(vals[2 * T:3 * T], float)
            algs.append((T, tau, u, v, w, np.array(mask.split(), int)))
    return rounds, algs


def test_round_truth_table():
    rounds, _ = _golden()
    assert len(rounds) >= 10
    for s, tau, want in rounds:
        assert oracle.round_(s, tau) == want, (s, tau)


def test_alg1_cases():
    _, algs = _golden()
    assert len(algs) >= 8
    for T, tau, u, v, w, mask in algs:
        fix, nf = oracle.fix(1, T, u, v, w, np.array([1], np.int8), tau, t_first=1)
        fixed = (fix.reshape(T, 3)[:, 0] >= 0).astype(int)
        assert list(fixed) == list(mask), (u, v, w)
        assert nf == mask.sum()
        for t in np.flatnonzero(mask):
            assert list(fix.reshape(T, 3)[t]) == [oracle.round_(u[t], tau), oracle.round_(v[t], tau),
                                                  oracle.round_(w[t], tau)]


@pytest.mark.parametrize("seed", range(5))
def test_alg1_invariants(seed):
    """Fixed triples satisfy Eq. 1 with their predecessors; fixed hours form a
    prefix starting at hour 2; every fixed value is Round of its input."""
    rng = np.random.default_rng(seed)
    G, T, tau = 200, 24, 0.1
    # mostly near-integral schedules with noise
    u = (rng.random((G, T)) < 0.6).astype(float)
    u = np.clip(u + rng.normal(0, 0.07, (G, T)), 0, 1)
    du = np.diff(np.concatenate([np.ones((G, 1)), np.round(u)], 1), axis=1)
    v = np.clip(np.maximum(du, 0) + rng.normal(0, 0.05, (G, T)), 0, 1)
    w = np.clip(np.maximum(-du, 0) + rng.normal(0, 0.05, (G, T)), 0, 1)
    fix, nf = oracle.fix(G, T, u.ravel(), v.ravel(), w.ravel(), np.ones(G, np.int8), tau)
    F = fix.reshape(G, T, 3)
    assert nf == int((F[:, :, 0] >= 0).sum())
    for g in range(G):
        fixed = F[g, :, 0] >= 0
        assert not fixed[0]
        k = int(fixed.sum())
        assert fixed[1:1 + k].all()
        for t in range(1, 1 + k):
            ut, vt, wt = F[g, t]
            uprev = oracle.round_(u[g, t - 1], tau)
            assert ut - uprev == vt - wt and vt + wt <= 1
            assert (ut, vt, wt) == (oracle.round_(u[g, t], tau), oracle.round_(v[g, t], tau),
                                    oracle.round_(w[g, t], tau))


def _tiny_binary(seed):
    """Tiny pure-binary MILP rows with random small integer coefficients."""
    rng = np.random.default_rng(seed)
    n, m = int(rng.integers(3, 7)), int(rng.integers(2, 6))
    A = rng.integers(-3, 4, (m, n)).astype(float)
    A[rng.random((m, n)) < 0.3] = 0.0
    x0 = rng.integers(0, 2, n)
    ax = A @ x0
    lo = ax - rng.integers(0, 3, m)
    hi = ax + rng.integers(0, 3, m)
    lo[rng.random(m) < 0.3] = -np.inf
    hi[rng.random(m) < 0.3] = np.inf
    S = sp.csr_matrix(A)
    lp = dict(m=m, n=n, row_ptr=S.indptr, col=S.indices, val=S.data, c=np.zeros(n),
              xl=np.zeros(n), xu=np.ones(n), lo=lo, hi=hi)
    return A, lp


@pytest.mark.parametrize("seed", range(60))
def test_propagation_sound_monotone_idempotent(seed):
    A, lp = _tiny_binary(seed)
    n = lp["n"]
    # random partial fixing, then propagate
    rng = np.random.default_rng(100 + seed)
    xl, xu = lp["xl"].copy(), lp["xu"].copy()
    k = rng.integers(0, n)
    xl[k] = xu[k] = float(rng.integers(0, 2))
    pl, pu, r = oracle.propagate(lp, xl, xu, np.ones(n, np.uint8))
    feas = [np.array(p) for p in itertools.product([0, 1], repeat=n)
            if np.all(np.array(p) >= xl) and np.all(np.array(p) <= xu)
            and np.all(A @ np.array(p) >= lp["lo"]) and np.all(A @ np.array(p) <= lp["hi"])]
    if r < 0:
        assert len(feas) == 0, "propagation declared a feasible problem infeasible"
        return
    # monotone
    assert np.all(pl >= xl) and np.all(pu <= xu)
    # sound: every feasible integer point survives
    for p in feas:
        assert np.all(p >= pl) and np.all(p <= pu)
    # idempotent at the fixpoint
    ql, qu, r2 = oracle.propagate(lp, pl, pu, np.ones(n, np.uint8))
    np.testing.assert_array_equal(ql, pl)
    np.testing.assert_array_equal(qu, pu)


def test_propagation_continuous_single_row():
    """x1 + x2 <= 1 with x1 >= 0.7 forces x2 <= 0.3 (one Jacobi pass)."""
    S = sp.csr_matrix(np.array([[1.0, 1.0]]))
    lp = dict(m=1, n=2, row_ptr=S.indptr, col=S.indices, val=S.data, c=np.zeros(2),
              xl=np.array([0.7, 0.0]), xu=np.array([1.0, 5.0]), lo=np.array([-np.inf]),
              hi=np.array([1.0]))
    pl, pu, r = oracle.propagate(lp, lp["xl"], lp["xu"], np.zeros(2, np.uint8))
    assert pu[1] == pytest.approx(0.3, abs=1e-15) and pu[0] == 1.0 and r >= 1


def _highs_obj(lp):
    A = sp.csr_matrix((lp["val"], lp["col"], lp["row_ptr"]), shape=(lp["m"], lp["n"]))
    lo, hi = lp["lo"], lp["hi"]
    fh, fl = np.isfinite(hi), np.isfinite(lo)
    Aub = sp.vstack([A[fh], -A[fl]]).tocsr()
    bub = np.concatenate([hi[fh], -lo[fl]])
    bounds = np.c_[np.where(np.isfinite(lp["xl"]), lp["xl"], None),
                   np.where(np.isfinite(lp["xu"]), lp["xu"], None)]
    res = linprog(lp["c"], A_ub=Aub if Aub.shape[0] else None, b_ub=bub if Aub.shape[0] else None,
                  bounds=bounds, method="highs")
    return res


def test_reduce_preserves_lp_optimum():
    """Fixing + propagation + reduction: the reduced LP's optimum plus the
    folded constant equals the optimum of the full LP with the same bounds."""
    inst = make_preset("scuc14")
    lp = oracle.as_lp(inst)
    r = oracle.hpr_solve(lp, tol=1e-6, max_iter=400000)
    x = r["x"]
    fix, nf = oracle.fix(inst.G, inst.T, x[inst.u_idx], x[inst.v_idx], x[inst.w_idx],
                         inst.u_init, 0.1)
    assert nf > 0
    xl, xu = lp["xl"].copy(), lp["xu"].copy()
    F = fix.reshape(-1, 3)
    for slot, idx in enumerate((inst.u_idx, inst.v_idx, inst.w_idx)):
        sel = F[:, slot] >= 0
        xl[idx[sel]] = F[sel, slot]; xu[idx[sel]] = F[sel, slot]
    pl, pu, passes = oracle.propagate(lp, xl, xu, inst.is_int)
    assert passes >= 1
    red, rmap, cmap, oc, bad = oracle.reduce(lp, pl, pu)
    assert bad == 0 and red["n"] < lp["n"] and red["m"] < lp["m"]
    full = dict(lp); full["xl"], full["xu"] = pl, pu
    f_full = _highs_obj(full).fun
    f_red = _highs_obj(red).fun + oc
    assert f_red == pytest.approx(f_full, rel=1e-9)
