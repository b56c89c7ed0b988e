"""Oracle pins for the second algorithm (restarted PDHG with ergodic
averaging) and for infeasibility detection, against what the mathematics
fixes: the LP optimum (vertex enumeration / Bland simplex on tiny LPs, HiGHS
on mid-size ones, closed forms), HiGHS's feasibility verdicts, and the
defining inequalities of the returned certificates (Farkas ray, recession
direction), checked here directly from their definitions on the unscaled LP."""
import numpy as np
import pytest

import oracle
from lp_cases import (DUAL_INFEASIBLE, PRIMAL_INFEASIBLE, farkas, highs_status, infeasible_box, dense_lp,
                      recession, unbounded)
from oracle import tiny_lp
from scuc_gen import make_preset, random_lp


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


@pytest.mark.parametrize("seed", range(20))
def test_pdhg_tiny_lp_optimum(seed):
    """PDHG_AVG objective == vertex enumeration == Bland simplex."""
    A, lo, hi, c, xl, xu = _tiny(seed)
    f_v, _ = tiny_lp.vertex_enum(A, lo, hi, c, xl, xu)
    f_s, _ = tiny_lp.bland_simplex(A, lo, hi, c, xl, xu)
    assert f_v == pytest.approx(f_s, rel=1e-9, abs=1e-9)
    r = oracle.hpr_solve(dense_lp(A, lo, hi, c, xl, xu), tol=1e-10, max_iter=400000, algo=1)
    assert r["info"]["status"] == 0
    assert r["info"]["pobj"] == pytest.approx(f_v, rel=1e-7, abs=1e-7)


def test_pdhg_bounds_only_closed_form():
    rng = np.random.default_rng(8)
    n = 40
    c = rng.normal(size=n)
    xl = rng.uniform(-4, 0, n)
    xu = xl + rng.uniform(0.1, 3, n)
    lp = dense_lp(np.zeros((0, n)), np.zeros(0), np.zeros(0), c, xl, xu)
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
    r = oracle.hpr_solve(dense_lp(w[None, :], [-np.inf], [cap], -v, np.zeros(k), np.ones(k)),
                         tol=1e-10, max_iter=400000, algo=1)
    assert -r["info"]["pobj"] == pytest.approx(float(v @ x), rel=1e-8)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_pdhg_random_lp_vs_highs(seed):
    lp = oracle.as_lp(random_lp(60, 40, density=0.1, seed=seed))
    st, f = highs_status(lp)
    assert st == 0
    r = oracle.hpr_solve(lp, tol=1e-8, max_iter=400000, algo=1)
    assert r["info"]["status"] == 0
    assert r["info"]["pobj"] == pytest.approx(f, rel=1e-6, abs=1e-6)


def test_pdhg_scuc14_vs_highs():
    lp = oracle.as_lp(make_preset("scuc14"))
    st, f = highs_status(lp)
    r = oracle.hpr_solve(lp, tol=1e-7, max_iter=400000, algo=1)
    assert st == 0 and r["info"]["status"] == 0
    assert r["info"]["pobj"] == pytest.approx(f, rel=1e-5)


@pytest.mark.parametrize("algo", [0, 1])
@pytest.mark.parametrize("seed", range(6))
def test_detection_primal_infeasible(algo, seed):
    lp = infeasible_box(seed)
    assert highs_status(lp)[0] == 2
    r = oracle.hpr_solve(lp, tol=1e-8, max_iter=100000, algo=algo, infeas_tol=1e-8)
    assert r["info"]["status"] == PRIMAL_INFEASIBLE
    F, V = farkas(lp, r["y"])
    assert F > 0 and V <= 1e-6 * F, (F, V)


@pytest.mark.parametrize("algo", [0, 1])
@pytest.mark.parametrize("seed", range(6))
def test_detectionunbounded(algo, seed):
    lp = unbounded(seed)
    assert highs_status(lp)[0] == 3
    r = oracle.hpr_solve(lp, tol=1e-8, max_iter=100000, algo=algo, infeas_tol=1e-8)
    assert r["info"]["status"] == DUAL_INFEASIBLE
    cd, V = recession(lp, r["x"])
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
    lp = dense_lp(np.zeros((0, 4)), np.zeros(0), np.zeros(0), c, xl, xu)
    steps, x = [], np.zeros(4)
    for _ in range(5):
        x = np.clip(x - sigma * c, xl, xu)
        steps.append(x)
    for k in range(1, 6):
        r = oracle.hpr_solve(lp, tol=0.0, max_iter=k, check_every=k, use_scaling=0, sigma0=sigma,
                             lambda_in=1.0, restart_suff=0.0, restart_nec=0.0, restart_long=2.0,
                             algo=1)
        np.testing.assert_allclose(r["x"], np.mean(steps[:k], axis=0), rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", range(5))
def test_pdhg_averaged_point_invariants(seed):
    """The checked point of PDHG is an average of projected points, so it
    stays in K, its y has the sign each row's bounds allow, and z vanishes
    where the bound it would price is infinite (at every iteration limit)."""
    lp = oracle.as_lp(random_lp(50, 35, density=0.15, seed=seed, senses="GLER"))
    for k in (64, 256, 1024):
        r = oracle.hpr_solve(lp, tol=0.0, max_iter=k, algo=1)
        x, y, z = r["x"], r["y"], r["z"]
        assert np.all(x >= lp["xl"] - 1e-12) and np.all(x <= lp["xu"] + 1e-12)
        assert np.all(y[~np.isfinite(lp["lo"])] <= 0.0) and np.all(y[~np.isfinite(lp["hi"])] >= 0.0)
        assert np.all(z[~np.isfinite(lp["xl"])] <= 0.0) and np.all(z[~np.isfinite(lp["xu"])] >= 0.0)


@pytest.mark.parametrize("algo", [0, 1])
def test_detection_silent_on_feasible_tiny_lps(algo):
    """Ten feasible tiny LPs (HiGHS optimal): detection never declares them
    infeasible and both algorithms reach HiGHS's optimum."""
    for seed in range(10):
        A, lo, hi, c, xl, xu = _tiny(50 + seed)
        lp = dense_lp(A, lo, hi, c, xl, xu)
        st, f = highs_status(lp)
        assert st == 0
        r = oracle.hpr_solve(lp, tol=1e-9, max_iter=400000, algo=algo, infeas_tol=1e-8)
        assert r["info"]["status"] == 0
        assert r["info"]["pobj"] == pytest.approx(f, rel=1e-6, abs=1e-6)
