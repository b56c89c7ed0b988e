"""Oracle pins for the second algorithm (restarted PDHG with ergodic
averaging) and for infeasibility detection, against what the mathematics
fixes: the LP optimum (vertex enumeration / Bland simplex on tiny LPs, HiGHS
on mid-size ones, closed forms), HiGHS's feasibility verdicts, and the
defining inequalities of the returned certificates (Farkas ray, recession
direction), checked here directly from their definitions on the unscaled LP."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import linprog

import oracle
from oracle import tiny_lp
from scuc_gen import make_preset, random_lp

PRIMAL_INFEASIBLE, DUAL_INFEASIBLE = 5, 6


def _lp(A, lo, hi, c, xl, xu):
    S = sp.csr_matrix(np.atleast_2d(np.asarray(A, float)))
    return dict(m=S.shape[0], n=len(c), row_ptr=S.indptr, col=S.indices, val=S.data,
                c=np.asarray(c, float), xl=np.asarray(xl, float), xu=np.asarray(xu, float),
                lo=np.asarray(lo, float), hi=np.asarray(hi, float))


def _tiny(seed):
    rng = np.random.default_rng(100 + seed)
    m, n = int(rng.integers(1, 5)), int(rng.integers(1, 6))
    A = rng.uniform(-2, 2, (m, n))
    xl = rng.uniform(-3, 0, n)
    xu = xl + rng.uniform(0.5, 4, n)
    x0 = xl + rng.random(n) * (xu - xl)
    ax = A @ x0
    lo = ax - rng.uniform(0.05, 1, m)
    hi = ax + rng.uniform(0.05, 1, m)
    lo[rng.random(m) < 0.3] = -np.inf
    return A, lo, hi, rng.normal(size=n), xl, xu


def _highs_status(lp):
    """HiGHS verdict: 0 optimal, 2 infeasible, 3 unbounded."""
    A = sp.csr_matrix((lp["val"], lp["col"], lp["row_ptr"]), shape=(lp["m"], lp["n"]))
    fh, fl = np.isfinite(lp["hi"]), np.isfinite(lp["lo"])
    Aub = sp.vstack([A[fh], -A[fl]]).tocsr()
    bub = np.concatenate([lp["hi"][fh], -lp["lo"][fl]])
    bounds = np.c_[np.where(np.isfinite(lp["xl"]), lp["xl"], None),
                   np.where(np.isfinite(lp["xu"]), lp["xu"], None)]
    r = linprog(lp["c"], A_ub=Aub if Aub.shape[0] else None, b_ub=bub if Aub.shape[0] else None,
                bounds=bounds, method="highs")
    return r.status, r.fun


def _farkas(lp, u):
    """Homogeneous dual objective of the ray u (z = -A^T u) over the terms
    whose bounds are finite, and the size of the terms that would need an
    infinite bound."""
    A = sp.csr_matrix((lp["val"], lp["col"], lp["row_ptr"]), shape=(lp["m"], lp["n"]))
    z = -(A.T @ u)
    F, V = 0.0, 0.0
    for v, l, h in list(zip(u, lp["lo"], lp["hi"])) + list(zip(z, lp["xl"], lp["xu"])):
        b = l if v > 0 else h
        if v == 0:
            continue
        if np.isfinite(b):
            F += b * v
        else:
            V += v * v
    return F, np.sqrt(V)


def _recession(lp, d):
    """c^T d and the size of the violation of the recession cones of
    [lo, hi] (by A d) and [xl, xu] (by d)."""
    A = sp.csr_matrix((lp["val"], lp["col"], lp["row_ptr"]), shape=(lp["m"], lp["n"]))
    ad = A @ d
    viol = np.concatenate([np.where((d < 0) & np.isfinite(lp["xl"]), d, 0.0),
                           np.where((d > 0) & np.isfinite(lp["xu"]), d, 0.0),
                           np.where((ad < 0) & np.isfinite(lp["lo"]), ad, 0.0),
                           np.where((ad > 0) & np.isfinite(lp["hi"]), ad, 0.0)])
    return float(lp["c"] @ d), float(np.linalg.norm(viol))


@pytest.mark.parametrize("seed", range(20))
def test_pdhg_tiny_lp_optimum(seed):
    """PDHG_AVG objective == vertex enumeration == Bland simplex."""
    A, lo, hi, c, xl, xu = _tiny(seed)
    f_v, _ = tiny_lp.vertex_enum(A, lo, hi, c, xl, xu)
    f_s, _ = tiny_lp.bland_simplex(A, lo, hi, c, xl, xu)
    assert f_v == pytest.approx(f_s, rel=1e-9, abs=1e-9)
    r = oracle.hpr_solve(_lp(A, lo, hi, c, xl, xu), tol=1e-10, max_iter=400000, algo=1)
    assert r["info"]["status"] == 0
    assert r["info"]["pobj"] == pytest.approx(f_v, rel=1e-7, abs=1e-7)


def test_pdhg_bounds_only_closed_form():
    rng = np.random.default_rng(8)
    n = 40
    c = rng.normal(size=n)
    xl = rng.uniform(-4, 0, n)
    xu = xl + rng.uniform(0.1, 3, n)
    lp = _lp(np.zeros((0, n)), np.zeros(0), np.zeros(0), c, xl, xu)
    r = oracle.hpr_solve(lp, tol=1e-12, max_iter=10000, algo=1)
    np.testing.assert_allclose(r["x"], np.where(c > 0, xl, xu), rtol=0, atol=1e-9)


def test_pdhg_fractional_knapsack_closed_form():
    rng = np.random.default_rng(12)
    k = 10
    v, w = rng.uniform(1, 10, k), rng.uniform(1, 5, k)
    cap = 0.35 * w.sum()
    x, left = np.zeros(k), cap
    for j in np.argsort(-v / w):
        x[j] = min(1.0, left / w[j])
        left -= x[j] * w[j]
        if left <= 0:
            break
    r = oracle.hpr_solve(_lp(w[None, :], [-np.inf], [cap], -v, np.zeros(k), np.ones(k)),
                         tol=1e-10, max_iter=400000, algo=1)
    assert -r["info"]["pobj"] == pytest.approx(float(v @ x), rel=1e-8)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_pdhg_random_lp_vs_highs(seed):
    lp = oracle.as_lp(random_lp(60, 40, density=0.1, seed=seed))
    st, f = _highs_status(lp)
    assert st == 0
    r = oracle.hpr_solve(lp, tol=1e-8, max_iter=400000, algo=1)
    assert r["info"]["status"] == 0
    assert r["info"]["pobj"] == pytest.approx(f, rel=1e-6, abs=1e-6)


def test_pdhg_scuc14_vs_highs():
    lp = oracle.as_lp(make_preset("scuc14"))
    st, f = _highs_status(lp)
    r = oracle.hpr_solve(lp, tol=1e-7, max_iter=400000, algo=1)
    assert st == 0 and r["info"]["status"] == 0
    assert r["info"]["pobj"] == pytest.approx(f, rel=1e-5)


def _infeasible_box(seed):
    """Rows that no point of a finite box satisfies (primal infeasible; the
    box keeps the dual feasible)."""
    rng = np.random.default_rng(seed)
    m, n = int(rng.integers(2, 6)), int(rng.integers(2, 6))
    A = rng.uniform(-2, 2, (m, n))
    xl, xu = rng.uniform(-2, 0, n), rng.uniform(0.5, 2, n)
    hi = np.full(m, np.inf)
    # row 0 asks for more than its maximum over the box
    amax = np.sum(np.where(A[0] > 0, A[0] * xu, A[0] * xl))
    lo = np.full(m, -np.inf)
    lo[0] = amax + rng.uniform(0.1, 1.0)
    return _lp(A, lo, hi, rng.normal(size=n), xl, xu)


def _unbounded(seed):
    """A feasible LP plus a column with negative cost and no upper bound whose
    entries only loosen rows with lower bounds (primal unbounded)."""
    rng = np.random.default_rng(seed)
    m, n = int(rng.integers(2, 6)), int(rng.integers(2, 5))
    A = rng.uniform(-2, 2, (m, n))
    xl, xu = rng.uniform(-2, 0, n), rng.uniform(0.5, 2, n)
    x0 = (xl + xu) / 2
    lo = A @ x0 - rng.uniform(0.1, 1, m)
    hi = np.full(m, np.inf)
    A = np.c_[A, rng.uniform(0.2, 1.0, m)]
    return _lp(A, lo, hi, np.r_[rng.normal(size=n), -1.0], np.r_[xl, 0.0], np.r_[xu, np.inf])


@pytest.mark.parametrize("algo", [0, 1])
@pytest.mark.parametrize("seed", range(6))
def test_detection_primal_infeasible(algo, seed):
    lp = _infeasible_box(seed)
    assert _highs_status(lp)[0] == 2
    r = oracle.hpr_solve(lp, tol=1e-8, max_iter=100000, algo=algo, infeas_tol=1e-8)
    assert r["info"]["status"] == PRIMAL_INFEASIBLE
    F, V = _farkas(lp, r["y"])
    assert F > 0 and V <= 1e-6 * F, (F, V)


@pytest.mark.parametrize("algo", [0, 1])
@pytest.mark.parametrize("seed", range(6))
def test_detection_unbounded(algo, seed):
    lp = _unbounded(seed)
    assert _highs_status(lp)[0] == 3
    r = oracle.hpr_solve(lp, tol=1e-8, max_iter=100000, algo=algo, infeas_tol=1e-8)
    assert r["info"]["status"] == DUAL_INFEASIBLE
    cd, V = _recession(lp, r["x"])
    assert cd < 0 and V <= 1e-6 * -cd, (cd, V)


@pytest.mark.parametrize("algo", [0, 1])
def test_detection_silent_on_feasible_lps(algo):
    """Detection never fires on feasible bounded LPs and does not change the
    iteration (same checks, same result as without it)."""
    for lp in [oracle.as_lp(random_lp(60, 40, density=0.1, seed=s)) for s in (1, 2)] + \
              [oracle.as_lp(make_preset("scuc14"))]:
        kw = dict(tol=1e-6, max_iter=200000, algo=algo)
        a = oracle.hpr_solve(lp, infeas_tol=1e-8, **kw)
        b = oracle.hpr_solve(lp, **kw)
        assert a["info"]["status"] == 0
        assert a["info"]["iters"] == b["info"]["iters"]
        np.testing.assert_array_equal(a["x"], b["x"])


def test_pdhg_average_is_the_mean_of_projected_gradient_steps():
    """No rows: PDHG is projected gradient descent on the box, x^{k+1} =
    clamp(x^k - sigma c), and the point a check returns is the plain mean of
    the iterates since the last restart (no scaling, restarts off)."""
    sigma = 0.3
    c = np.array([1.0, -2.0, 0.5, -0.25])
    xl = np.array([-1.0, -1.0, -0.2, -5.0])
    xu = np.array([1.0, 0.9, 1.0, 5.0])
    lp = _lp(np.zeros((0, 4)), np.zeros(0), np.zeros(0), c, xl, xu)
    steps, x = [], np.zeros(4)
    for _ in range(5):
        x = np.clip(x - sigma * c, xl, xu)
        steps.append(x)
    for k in range(1, 6):
        r = oracle.hpr_solve(lp, tol=0.0, max_iter=k, check_every=k, use_scaling=0, sigma0=sigma,
                             lambda_in=1.0, restart_suff=0.0, restart_nec=0.0, restart_long=2.0,
                             algo=1)
        np.testing.assert_allclose(r["x"], np.mean(steps[:k], axis=0), rtol=0, atol=1e-15)
