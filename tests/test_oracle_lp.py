"""Pins of the CPU oracle's LP solve (restarted HPR, Eq. 9) against things other
than itself: exact tiny-LP solvers, closed forms, HiGHS, eigvalsh, the
invariants of an optimal primal-dual pair, and the O(1/k) bound of Theorem 1.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import linprog

import oracle
from oracle import tiny_lp
from scuc_gen import make_preset, random_lp


def _dense_lp(A, lo, hi, c, xl, xu):
    S = sp.csr_matrix(np.atleast_2d(A)) if np.size(A) else sp.csr_matrix((0, len(c)))
    return dict(m=S.shape[0], n=len(c), row_ptr=S.indptr, col=S.indices, val=S.data,
                c=np.asarray(c, float), xl=np.asarray(xl, float), xu=np.asarray(xu, float),
                lo=np.asarray(lo, float), hi=np.asarray(hi, float))


def _tiny(seed):
    rng = np.random.default_rng(seed)
    m, n = int(rng.integers(1, 5)), int(rng.integers(1, 6))
    A = rng.uniform(-2, 2, (m, n))
    A[rng.random((m, n)) < 0.25] = 0.0
    xl = rng.uniform(-3, 0, n)
    xu = xl + rng.uniform(0.5, 4, n)
    x0 = xl + rng.random(n) * (xu - xl)
    ax = A @ x0
    lo = ax - rng.uniform(0.05, 1, m)
    hi = ax + rng.uniform(0.05, 1, m)
    kind = rng.integers(0, 4, m)
    lo[kind == 1] = -np.inf
    hi[kind == 2] = np.inf
    hi[kind == 3] = lo[kind == 3]          # equality rows
    if np.any(kind == 3):                   # keep equality rows satisfiable
        lo[kind == 3] = ax[kind == 3]; hi[kind == 3] = ax[kind == 3]
    c = rng.normal(size=n)
    return A, lo, hi, c, xl, xu


@pytest.mark.parametrize("seed", range(40))
def test_tiny_lp_three_way(seed):
    """Vertex enumeration == Bland simplex == HPR oracle objective."""
    A, lo, hi, c, xl, xu = _tiny(seed)
    f_v, _ = tiny_lp.vertex_enum(A, lo, hi, c, xl, xu)
    f_s, _ = tiny_lp.bland_simplex(A, lo, hi, c, xl, xu)
    assert f_v == pytest.approx(f_s, rel=1e-9, abs=1e-9)
    r = oracle.hpr_solve(_dense_lp(A, lo, hi, c, xl, xu), tol=1e-10, max_iter=400000)
    assert r["info"]["status"] == 0
    assert r["info"]["pobj"] == pytest.approx(f_v, rel=1e-7, abs=1e-7)
    # the solution itself is feasible
    x = r["x"]
    assert np.all(x >= xl - 1e-8) and np.all(x <= xu + 1e-8)
    ax = A @ x
    assert np.all(ax >= lo - 1e-6) and np.all(ax <= hi + 1e-6)


def test_bounds_only_lp_closed_form():
    """No rows: x_j = xl_j if c_j > 0 else xu_j (c_j < 0)."""
    rng = np.random.default_rng(3)
    n = 50
    c = rng.normal(size=n)
    xl = rng.uniform(-4, 0, n)
    xu = xl + rng.uniform(0.1, 3, n)
    lp = _dense_lp(np.zeros((0, n)), np.zeros(0), np.zeros(0), c, xl, xu)
    r = oracle.hpr_solve(lp, tol=1e-12, max_iter=10000)
    want = np.where(c > 0, xl, xu)
    np.testing.assert_allclose(r["x"], want, rtol=0, atol=1e-9)
    assert r["info"]["pobj"] == pytest.approx(float(c @ want), rel=1e-10)


def test_fractional_knapsack_closed_form():
    """max v^T x, w^T x <= W, 0 <= x <= 1: greedy by v/w ratio."""
    rng = np.random.default_rng(11)
    k = 12
    v = rng.uniform(1, 10, k)
    w = rng.uniform(1, 5, k)
    Wcap = 0.4 * w.sum()
    order = np.argsort(-v / w)
    x = np.zeros(k)
    left = Wcap
    for j in order:
        take = min(1.0, left / w[j])
        x[j] = take
        left -= take * w[j]
        if left <= 0:
            break
    best = float(v @ x)
    lp = _dense_lp(w[None, :], np.array([-np.inf]), np.array([Wcap]), -v, np.zeros(k), np.ones(k))
    r = oracle.hpr_solve(lp, tol=1e-10, max_iter=400000)
    assert -r["info"]["pobj"] == pytest.approx(best, rel=1e-8)
    np.testing.assert_allclose(r["x"], x, atol=1e-6)


def test_economic_dispatch_merit_order():
    """Single bus, one hour, all units committed: fill Pmin, then the
    cheapest segments first (merit order); unserved load at the penalty."""
    rng = np.random.default_rng(5)
    G = 6
    pmax = rng.uniform(50, 200, G)
    pmin = 0.3 * pmax
    segw = np.repeat(((pmax - pmin) / 3)[:, None], 3, axis=1)
    segc = np.sort(rng.uniform(10, 80, (G, 3)), axis=1)
    D = pmin.sum() + 0.55 * segw.sum()
    pen = 1000.0
    # variables: p_{g,h} (3G), d
    n = 3 * G + 1
    A = np.ones((1, n))
    lo = hi = np.array([D - pmin.sum()])
    c = np.concatenate([segc.ravel(), [pen]])
    xl = np.zeros(n)
    xu = np.concatenate([segw.ravel(), [D]])
    lp = _dense_lp(A, lo, hi, c, xl, xu)
    r = oracle.hpr_solve(lp, tol=1e-10, max_iter=400000)
    # closed form
    need = D - pmin.sum()
    cost = 0.0
    for j in np.argsort(c[:-1], kind="stable"):
        take = min(need, xu[j])
        cost += take * c[j]
        need -= take
    assert need == pytest.approx(0.0, abs=1e-12)
    assert r["info"]["pobj"] == pytest.approx(cost, rel=1e-8)


def _highs(lp):
    A = sp.csr_matrix((lp["val"], lp["col"], lp["row_ptr"]), shape=(lp["m"], lp["n"]))
    lo, hi = lp["lo"], lp["hi"]
    eq = lo == hi
    fh = np.isfinite(hi) & ~eq
    fl = np.isfinite(lo) & ~eq
    Aub = sp.vstack([A[fh], -A[fl]]).tocsr()
    bub = np.concatenate([hi[fh], -lo[fl]])
    bounds = np.c_[np.where(np.isfinite(lp["xl"]), lp["xl"], None),
                   np.where(np.isfinite(lp["xu"]), lp["xu"], None)]
    res = linprog(lp["c"], A_ub=Aub if Aub.shape[0] else None, b_ub=bub if Aub.shape[0] else None,
                  A_eq=A[eq] if eq.any() else None, b_eq=lo[eq] if eq.any() else None,
                  bounds=bounds, method="highs")
    assert res.status == 0
    return res


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_lp_vs_highs(seed):
    lp = oracle.as_lp(random_lp(60, 40, density=0.15, seed=seed, long_rows=2, long_cols=2))
    res = _highs(lp)
    r = oracle.hpr_solve(lp, tol=1e-8, max_iter=400000)
    assert r["info"]["status"] == 0
    assert r["info"]["pobj"] == pytest.approx(res.fun, rel=1e-6, abs=1e-6)


@pytest.fixture(scope="module")
def scuc14():
    return make_preset("scuc14")


def test_scuc14_vs_highs(scuc14):
    lp = oracle.as_lp(scuc14)
    res = _highs(lp)
    r = oracle.hpr_solve(lp, tol=1e-8, max_iter=400000)
    assert r["info"]["status"] == 0
    assert r["info"]["pobj"] == pytest.approx(res.fun, rel=1e-7)


def test_optimality_invariants(scuc14):
    """At a tight solution: primal feasibility, dual sign feasibility,
    complementary slackness and weak duality, all measured on the unscaled LP."""
    lp = oracle.as_lp(scuc14)
    r = oracle.hpr_solve(lp, tol=1e-9, max_iter=400000)
    x, y, z = r["x"], r["y"], r["z"]
    A = sp.csr_matrix((lp["val"], lp["col"], lp["row_ptr"]), shape=(lp["m"], lp["n"]))
    ax = A @ x
    scale = 1 + np.abs(np.where(np.isfinite(lp["lo"]), lp["lo"], 0)).max()
    assert np.all(ax >= lp["lo"] - 1e-6 * scale) and np.all(ax <= lp["hi"] + 1e-6 * scale)
    assert np.all(x >= lp["xl"] - 1e-9) and np.all(x <= lp["xu"] + 1e-9)
    # dual sign: y_i > 0 only where lo finite, y_i < 0 only where hi finite
    assert np.all(y[~np.isfinite(lp["lo"])] <= 1e-12)
    assert np.all(y[~np.isfinite(lp["hi"])] >= -1e-12)
    # complementary slackness (row side the multiplier prices is active)
    ysc = np.abs(y).max() + 1
    slack_lo = np.where(np.isfinite(lp["lo"]), ax - lp["lo"], np.inf)
    slack_hi = np.where(np.isfinite(lp["hi"]), lp["hi"] - ax, np.inf)
    cs = np.where(y > 0, y * slack_lo, np.where(y < 0, -y * slack_hi, 0.0))
    assert np.max(np.abs(cs)) <= 1e-5 * ysc * scale
    # weak duality for this (primal feasible, dual feasible) pair
    k = oracle.kkt(lp, x, y, z)
    assert k["dobj"] <= k["pobj"] + 1e-7 * (1 + abs(k["pobj"]))
    assert k["gap"] <= 1e-9 and k["rp"] <= 1e-9 and k["rd"] <= 1e-9


def test_power_method_vs_eigvalsh():
    for seed in range(4):
        lp = random_lp(40, 30, density=0.2, seed=seed)
        A = sp.csr_matrix((lp["val"], lp["col"], lp["row_ptr"]), shape=(lp["m"], lp["n"])).toarray()
        true = np.linalg.eigvalsh(A @ A.T).max()
        lam, it = oracle.power_lambda(lp["m"], lp["n"], lp["row_ptr"], lp["col"], lp["val"],
                                      max_iter=20000, tol=1e-13)
        assert lam == pytest.approx(true, rel=1e-8)
        lam_d, _ = oracle.power_lambda(lp["m"], lp["n"], lp["row_ptr"], lp["col"], lp["val"])
        assert 1.01 * lam_d >= true * (1 - 1e-6)   # the safety factor covers the default stop


def test_theorem1_envelope():
    """Theorem 1: ||R(w_bar^{k+1})|| <= C/(k+1) without restarts.  With the
    Halpern anchor the late-window maximum of ||R||*(k+1) must not grow; a
    wrong anchor weight (plain reflected iteration) grows like sqrt(k)."""
    A, lo, hi, c, xl, xu = _tiny(7)
    rng = np.random.default_rng(0)
    lp = oracle.as_lp(random_lp(30, 20, density=0.3, seed=4, senses="G", free_frac=0.0))
    r = oracle.hpr_solve(lp, tol=0.0, max_iter=4096, check_every=1, use_scaling=0,
                         restart_suff=0.0, restart_nec=0.0, restart_long=1e9, log_cap=4096)
    it = np.array([e["iter"] for e in r["log"]], dtype=float)
    R = np.array([e["rmap"] for e in r["log"]])
    prod = R * it
    early = prod[(it >= 64) & (it < 512)].max()
    late = prod[(it >= 2048)].max()
    assert late <= 1.05 * early
    assert np.all(np.isfinite(R))


def test_pock_chambolle_scaling_equivalence(scuc14):
    """Sec. 3.A: the diagonal scaling is a change of variables; the unscaled
    objective is the same with and without it."""
    lp = oracle.as_lp(scuc14)
    a = oracle.hpr_solve(lp, tol=1e-7, max_iter=400000, use_scaling=1)
    b = oracle.hpr_solve(lp, tol=1e-7, max_iter=2000000, use_scaling=0)
    c = oracle.hpr_solve(lp, tol=1e-7, max_iter=400000, use_scaling=2)   # Ruiz + PC
    assert a["info"]["status"] == 0 and b["info"]["status"] == 0 and c["info"]["status"] == 0
    assert a["info"]["pobj"] == pytest.approx(b["info"]["pobj"], rel=2e-6)
    assert c["info"]["pobj"] == pytest.approx(b["info"]["pobj"], rel=2e-6)


def test_scale_function_definition():
    """D_r = 1/sqrt(row abs sums), D_c = 1/sqrt(col abs sums) (alpha = 1),
    then bounds / (1+||b||), cost / (1+||c||); x = beta D_c x_hat."""
    lp = oracle.as_lp(random_lp(25, 15, density=0.3, seed=9))
    s = oracle.scale(lp)
    A = sp.csr_matrix((lp["val"], lp["col"], lp["row_ptr"]), shape=(lp["m"], lp["n"])).toarray()
    Dr = 1 / np.sqrt(np.abs(A).sum(1))
    Dc = 1 / np.sqrt(np.abs(A).sum(0))
    np.testing.assert_allclose(s["Dr"], Dr, rtol=1e-14)
    np.testing.assert_allclose(s["Dc"], Dc, rtol=1e-14)
    Ah = sp.csr_matrix((s["val"], lp["col"], lp["row_ptr"]), shape=A.shape).toarray()
    np.testing.assert_allclose(Ah, Dr[:, None] * A * Dc[None, :], rtol=1e-14)
    lo_s, hi_s = Dr * lp["lo"], Dr * lp["hi"]
    bmag = np.maximum(np.where(np.isfinite(lo_s), np.abs(lo_s), 0), np.where(np.isfinite(hi_s), np.abs(hi_s), 0))
    beta = 1 + np.linalg.norm(bmag)
    assert s["beta"] == pytest.approx(beta, rel=1e-14)
    gamma = 1 + np.linalg.norm(Dc * lp["c"])
    assert s["gamma"] == pytest.approx(gamma, rel=1e-14)


def test_ruiz_definition():
    """use_scaling = 2: ten passes dividing rows and columns by sqrt of their
    largest magnitude, then one Pock-Chambolle pass, all on the current matrix."""
    lp = oracle.as_lp(random_lp(25, 15, density=0.3, seed=9))
    s = oracle.scale(lp, use_scaling=2)
    A = sp.csr_matrix((lp["val"], lp["col"], lp["row_ptr"]), shape=(lp["m"], lp["n"])).toarray()
    Dr, Dc = np.ones(lp["m"]), np.ones(lp["n"])
    for _ in range(10):
        B = np.abs(Dr[:, None] * A * Dc[None, :])
        Dr, Dc = Dr / np.sqrt(B.max(1)), Dc / np.sqrt(B.max(0))
    B = np.abs(Dr[:, None] * A * Dc[None, :])
    Dr, Dc = Dr / np.sqrt(B.sum(1)), Dc / np.sqrt(B.sum(0))
    np.testing.assert_allclose(s["Dr"], Dr, rtol=1e-12)
    np.testing.assert_allclose(s["Dc"], Dc, rtol=1e-12)
    # after Ruiz the largest magnitude in every row/column is close to 1
    Bh = np.abs(sp.csr_matrix((s["val"], lp["col"], lp["row_ptr"]), shape=A.shape).toarray())
    assert Bh.max() <= 1.0 + 1e-12


def test_eta_scaling_equivalence():
    """Sec. 3.A instance-aware scaling: the eta-scaled and unscaled models have
    the same optimum once the objective is multiplied by eta^C (and powers by
    eta^P); checked with HiGHS and with the oracle."""
    a = make_preset("scuc14", eta_scaling=True)
    b = make_preset("scuc14", eta_scaling=False)
    fa = _highs(oracle.as_lp(a)).fun * a.objective_scale
    fb = _highs(oracle.as_lp(b)).fun * b.objective_scale
    assert fa == pytest.approx(fb, rel=1e-9)
    ra = oracle.hpr_solve(a, tol=1e-7, max_iter=400000)
    assert ra["info"]["pobj"] * a.objective_scale == pytest.approx(fb, rel=2e-6)


def _golden_kkt_points():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "kkt_2x3.txt")
    pts = []
    with open(path) as f:
        for line in f:
            if line.startswith("point "):
                a, b = line[len("point "):].split("|")
                v = [float(t) for t in a.split()]
                pts.append((v[0:3], v[3:5], v[5:8], [float(t) for t in b.split()]))
    return pts


def test_kkt_hand_worked_golden():
    """orc_kkt against residuals, objectives and Theorem 1's map worked by hand
    on a 2x3 LP at two non-optimal points (tests/golden/kkt_2x3.txt): both
    signs of y and z, terms left out at infinite bounds, the bound norm of a
    ranged row taken from its larger finite bound."""
    inf = np.inf
    lp = dict(m=2, n=3, row_ptr=np.array([0, 2, 4]), col=np.array([0, 1, 1, 2]),
              val=np.array([1.0, 2.0, 1.0, -1.0]), c=np.array([2.0, -1.0, 2.0]),
              xl=np.array([0.0, -inf, 0.0]), xu=np.array([4.0, 5.0, inf]),
              lo=np.array([3.0, -4.0]), hi=np.array([inf, 2.0]))
    pts = _golden_kkt_points()
    assert len(pts) == 2
    for x, y, z, want in pts:
        k = oracle.kkt(lp, np.array(x), np.array(y), np.array(z))
        got = [k[key] for key in ("rp", "rd", "gap", "pobj", "dobj", "kkt", "rmap")]
        np.testing.assert_allclose(got, want, rtol=1e-14, atol=0)
