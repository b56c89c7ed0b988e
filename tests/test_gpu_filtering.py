"""GPU parity of the transmission-filtering steps (Fig. 1) with the oracle,
through the C ABI: the violated pool rows at a point (same rows as the
oracle's definition, except rows within rounding of the threshold), the LP
with rows appended (bit for bit), and the loop, whose last solution is a
KKT point of the full LP (oracle evaluator) with the full LP's objective."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from scuc_gen import make_preset, split_network_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2510_10891_b300 as P
    return P


@pytest.fixture(scope="module")
def split2k():
    inst = make_preset("scuc2k")
    base, pool, pool_rows = split_network_rows(inst)
    return inst, base, pool, pool_rows


def _rel_violation(pool, x):
    A = sp.csr_matrix((pool["val"], pool["col"], pool["row_ptr"]), shape=(pool["m"], pool["n"]))
    ax = A @ x
    lo, hi = pool["lo"], pool["hi"]
    with np.errstate(invalid="ignore"):
        vl = np.where(np.isfinite(lo) & (lo - ax > 0), (lo - ax) / (1 + np.abs(lo)), 0.0)
        vh = np.where(np.isfinite(hi) & (ax - hi > 0), (ax - hi) / (1 + np.abs(hi)), 0.0)
    return np.maximum(vl, vh)


def test_row_violations_parity(P, split2k):
    import torch
    inst, base, pool, _ = split2k
    x = P.LP(base).solve(tol=1e-4, precision="mixed")["x"]     # the base solution violates line rows
    gp = P.LP(pool)
    rel = _rel_violation(pool, x)
    for tol in (1e-6, 1e-3, 1e-1):
        rows, worst = gp.row_violations(x, tol)
        orows, oworst = oracle.row_violations(pool, x, tol)
        assert worst == pytest.approx(oworst, rel=1e-12)
        clear = np.abs(rel - tol) > 1e-12 * max(1.0, tol)         # not within rounding of the threshold
        np.testing.assert_array_equal(np.intersect1d(rows, np.flatnonzero(clear)),
                                      np.intersect1d(orows, np.flatnonzero(clear)))
        assert np.all(np.diff(rows) > 0)
        drows, dworst = gp.row_violations(torch.as_tensor(x, device="cuda"), tol)   # x on the device
        np.testing.assert_array_equal(drows, rows)
        assert dworst == worst
    assert len(gp.row_violations(x, 1e-6)[0]) > 0
    rows, worst = gp.row_violations(x, 1e30)
    assert len(rows) == 0 and worst == pytest.approx(float(rel.max()), rel=1e-12)
    few, _ = gp.row_violations(x, 1e-6, cap=3)                    # capacity: the first rows only
    np.testing.assert_array_equal(few, gp.row_violations(x, 1e-6)[0][:3])


def test_add_rows_bit_identical(P, split2k):
    inst, base, pool, _ = split2k
    gb, gp = P.LP(base), P.LP(pool)
    rows = np.array([5, 0, 1799, 5, pool["m"] - 1], dtype=np.int32)   # any order, repeats allowed
    out = gb.add_rows(gp, rows)
    want = oracle.add_rows(gb.export(), gp.export(), rows)
    got = out.export()
    for k in ("row_ptr", "col", "val", "c", "xl", "xu", "lo", "hi"):
        np.testing.assert_array_equal(got[k], want[k], err_msg=k)
    assert (out.m, out.n) == (base["m"] + len(rows), base["n"])
    same = gb.add_rows(gp, [])
    assert same.m == base["m"]
    with pytest.raises(P._lib.ScucError) as e:
        gb.add_rows(gp, [pool["m"]])
    assert e.value.code == P._lib.SCUC_E_INVALID


def test_filtering_loop_scuc14_reaches_the_full_optimum(P):
    inst = make_preset("scuc14")
    base, pool, _ = split_network_rows(inst)
    f = P.transmission_filter(P.LP(base), P.LP(pool), viol_tol=1e-6, tol=1e-8, max_iter=400000)
    o = oracle.transmission_filter(base, pool, viol_tol=1e-6, tol=1e-8, max_iter=400000)
    assert f["converged"] and o["converged"]
    assert len(f["rounds"]) == len(o["rounds"])
    assert [r["added"] for r in f["rounds"]] == [r["added"] for r in o["rounds"]]
    full = oracle.hpr_solve(inst, tol=1e-9, max_iter=800000)
    assert f["result"]["info"]["pobj"] == pytest.approx(full["info"]["pobj"], rel=1e-6)


def test_filtering_loop_scuc2k_is_a_kkt_point_of_the_full_lp(P, split2k):
    inst, base, pool, pool_rows = split2k
    gp = P.LP(pool)
    f = P.transmission_filter(P.LP(base), gp, viol_tol=1e-5, tol=1e-5, precision="mixed")
    assert f["converged"] and len(f["rounds"]) >= 2
    assert all(r["status"] == 0 for r in f["rounds"])
    assert f["rounds"][-1]["m"] < base["m"] + pool["m"]          # fewer rows than the full LP
    x = f["result"]["x"]
    viol = oracle.row_violations(pool, x, 1e-5)[0]
    assert np.all(np.isin(viol, f["rows_added"]))               # none outside the LP
    assert len(oracle.row_violations(pool, x, 1e-4)[0]) == 0    # inside: within the solve's accuracy
    # the multipliers of the full LP: the filtered LP's, 0 on pool rows never added
    y = f["result"]["y"]
    y_full = np.zeros(inst.m)
    y_full[np.setdiff1d(np.arange(inst.m), pool_rows)] = y[:base["m"]]
    y_full[pool_rows[f["rows_added"]]] = y[base["m"]:]
    k = oracle.kkt(inst, x, y_full, f["result"]["z"])
    assert k["kkt"] <= 1e-4, k
    full = P.LP(inst).solve(tol=1e-6, precision="mixed")
    assert f["result"]["info"]["pobj"] == pytest.approx(full["info"]["pobj"], rel=1e-4)
    f["lp"].close()

