"""Oracle pins for the transmission-filtering loop (Fig. 1: solve without
the network security rows, add the violated ones, re-solve from the
previous point): the violation test on a hand-worked case, row appending
against scipy's vstack, and the loop's optimum against HiGHS on the full LP
(when the loop stops with no violated row, its LP's optimum is optimal for
the full LP)."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from lp_cases import dense_lp
from scuc_gen import make_preset, random_lp, split_network_rows


def _highs_obj(d):
    from scipy.optimize import linprog
    A = sp.csr_matrix((d["val"], d["col"], d["row_ptr"]), shape=(d["m"], d["n"]))
    fh, fl = np.isfinite(d["hi"]), np.isfinite(d["lo"])
    r = linprog(d["c"], A_ub=sp.vstack([A[fh], -A[fl]]).tocsr(), b_ub=np.r_[d["hi"][fh], -d["lo"][fl]],
                bounds=np.c_[np.where(np.isfinite(d["xl"]), d["xl"], None),
                             np.where(np.isfinite(d["xu"]), d["xu"], None)], method="highs")
    assert r.status == 0
    return r.fun


def test_row_violations_hand_worked():
    # rows: x0 + x1 in [1, 2];  x0 - x1 <= 0;  2 x1 >= -1;  x0 = 3 (equality)
    pool = dense_lp([[1, 1], [1, -1], [0, 2], [1, 0]], [1, -np.inf, -1, 3], [2, 0, np.inf, 3], [0, 0],
                    [-10, -10], [10, 10])
    x = np.array([2.5, 0.5])
    # a x = [3, 2, 1, 2.5]: row 0 above 2 by 1 -> 1/3; row 1 above 0 by 2 -> 2/1;
    # row 2 fine; row 3 below 3 by 0.5 -> 0.5/4
    rows, worst = oracle.row_violations(pool, x, 0.2)
    np.testing.assert_array_equal(rows, [0, 1])
    assert worst == pytest.approx(2.0, rel=1e-15)
    rows, _ = oracle.row_violations(pool, x, 0.1)
    np.testing.assert_array_equal(rows, [0, 1, 3])
    rows, worst = oracle.row_violations(pool, np.array([1.0, 1.0]), 0.0)   # a x = [2, 0, 2, 1]: only row 3
    np.testing.assert_array_equal(rows, [3])
    assert worst == pytest.approx(0.5, rel=1e-15)


def test_add_rows_is_vstack():
    base = oracle.as_lp(random_lp(30, 20, density=0.2, seed=4))
    pool = oracle.as_lp(random_lp(25, 20, density=0.3, seed=5))
    rows = np.array([7, 2, 19, 3])
    out = oracle.add_rows(base, pool, rows)
    Ab = sp.csr_matrix((base["val"], base["col"], base["row_ptr"]), shape=(30, 20))
    Ap = sp.csr_matrix((pool["val"], pool["col"], pool["row_ptr"]), shape=(25, 20))
    want = sp.vstack([Ab, Ap[rows]]).tocsr()
    np.testing.assert_array_equal(out["row_ptr"], want.indptr)
    np.testing.assert_array_equal(out["col"], want.indices)
    np.testing.assert_array_equal(out["val"], want.data)
    np.testing.assert_array_equal(out["lo"], np.r_[base["lo"], pool["lo"][rows]])
    np.testing.assert_array_equal(out["hi"], np.r_[base["hi"], pool["hi"][rows]])


def test_filtering_scuc14_reaches_the_full_optimum():
    inst = make_preset("scuc14")
    base, pool, _ = split_network_rows(inst)
    f = oracle.transmission_filter(base, pool, viol_tol=1e-6, tol=1e-8, max_iter=400000)
    assert f["converged"] and len(f["rounds"]) >= 2            # some line rows had to be added
    assert f["rounds"][0]["added"] > 0
    assert all(r["status"] == 0 for r in f["rounds"])
    assert f["result"]["info"]["pobj"] == pytest.approx(_highs_obj(oracle.as_lp(inst)), rel=1e-6)
    rows, worst = oracle.row_violations(pool, f["result"]["x"], 1e-6)
    assert len(rows) == 0 and worst <= 1e-6


def test_filtering_random_lp_reaches_the_full_optimum():
    full = oracle.as_lp(random_lp(80, 50, density=0.15, seed=9))
    A = sp.csr_matrix((full["val"], full["col"], full["row_ptr"]), shape=(80, 50))
    rng = np.random.default_rng(9)
    in_pool = rng.random(80) < 0.5

    def part(sel):
        S = A[sel].tocsr()
        return dict(m=S.shape[0], n=50, row_ptr=S.indptr, col=S.indices, val=S.data, c=full["c"],
                    xl=full["xl"], xu=full["xu"], lo=full["lo"][sel], hi=full["hi"][sel])

    base, pool = part(~in_pool), part(in_pool)
    f = oracle.transmission_filter(base, pool, viol_tol=1e-7, tol=1e-9, max_iter=400000)
    assert f["converged"]
    assert f["result"]["info"]["pobj"] == pytest.approx(_highs_obj(full), rel=1e-6, abs=1e-7)
