"""GPU parity of the restarted HPR solve (Eq. 9) against the CPU oracle,
through the C ABI.  FP64 runs take the same restart decisions as the oracle
at every check; iterates agree to rounding (relative 1e-9 on the KKT values,
1e-8 on the returned point); the final objective agrees to 1e-9 relative."""
import numpy as np
import pytest

import oracle
from scuc_gen import make_preset, random_lp, seeded_vector

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.fixture(scope="module")
def P(torch_cuda):
    import paper_2510_10891_b300 as P
    return P


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


def _compare_logs(glog, olog, rtol=1e-7, sigma_rtol=1e-9):
    assert len(glog) == len(olog), (len(glog), len(olog))
    for g, o in zip(glog, olog):
        assert g["iter"] == o["iter"]
        assert g["restart"] == o["restart"], (g, o)
        assert g["first"] == o["first"]
        for k in ("rp", "rd"):
            assert g[k] == pytest.approx(o[k], rel=rtol, abs=1e-13), (k, g, o)
        # the gap is a normalised difference of two O(1) objectives: its
        # rounding error is absolute (~1e-13 after 1e4 iterations), not
        # relative to the gap
        assert g["gap"] == pytest.approx(o["gap"], rel=rtol, abs=1e-11), ("gap", g, o)
        assert g["pobj"] == pytest.approx(o["pobj"], rel=1e-9, abs=1e-9)
        assert g["sigma"] == pytest.approx(o["sigma"], rel=sigma_rtol)


LP_CASES = [
    # (m, n, density, seed, long_rows, long_cols, senses)
    (40, 30, 0.2, 0, 0, 0, "GLER"),
    (300, 200, 0.02, 1, 3, 2, "GLER"),      # long rows (> 256 nnz) and long columns
    (1000, 700, 0.004, 2, 0, 4, "GE"),
    (513, 1025, 0.01, 3, 2, 0, "LR"),       # ragged sizes
]


@pytest.mark.parametrize("case", LP_CASES)
def test_matvec_parity(P, torch_cuda, case):
    torch = torch_cuda
    m, n, dens, seed, lr, lc, sen = case
    d = random_lp(m, n, density=dens, seed=seed, long_rows=lr, long_cols=lc, senses=sen)
    lp = P.LP(d)
    import scipy.sparse as sp
    A = sp.csr_matrix((d["val"], d["col"], d["row_ptr"]), shape=(m, n))
    x = seeded_vector(n, 10 + seed)
    y = seeded_vector(m, 20 + seed)
    ax = lp.matvec(torch.tensor(x, device="cuda"), torch.zeros(m, dtype=torch.float64, device="cuda"))
    aty = lp.matvec(torch.tensor(y, device="cuda"), torch.zeros(n, dtype=torch.float64, device="cuda"),
                    transpose=True)
    np.testing.assert_allclose(ax.cpu().numpy(), A @ x, rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(aty.cpu().numpy(), A.T @ y, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("case", LP_CASES)
def test_solve_parity_random(P, case):
    m, n, dens, seed, lr, lc, sen = case
    d = random_lp(m, n, density=dens, seed=seed, long_rows=lr, long_cols=lc, senses=sen)
    kw = dict(tol=1e-6, max_iter=20480, check_every=64)
    o = oracle.hpr_solve(d, **kw)
    g = P.LP(d).solve(**kw)
    gi, oi = g["info"], o["info"]
    assert gi["lambda"] == pytest.approx(oi["lambda"], rel=1e-12)
    assert gi["power_iters"] == oi["power_iters"]
    assert gi["status"] == oi["status"] and gi["iters"] == oi["iters"]
    _compare_logs(g["log"], o["log"])
    assert gi["pobj"] == pytest.approx(oi["pobj"], rel=1e-9, abs=1e-9)
    assert _rel(g["x"], o["x"]) < 1e-8
    assert _rel(g["y"], o["y"]) < 1e-8
    assert _rel(g["z"], o["z"]) < 1e-8
    # the returned point is what the oracle's KKT evaluator says it is
    k = oracle.kkt(d, g["x"], g["y"], g["z"])
    assert k["kkt"] == pytest.approx(gi["kkt"], rel=1e-9, abs=1e-14)


@pytest.mark.parametrize("case", LP_CASES + [(5000, 40, 0.002, 4, 0, 1, "GL")])
def test_spmv_layouts_agree(P, case):
    """The primal step's A^T y on the sliced ELL copy of A^T (the default)
    and on the CSR partition (spmv_layout = 1): FP64 solves take the same
    restart decisions at every check with iterates equal to rounding, and
    mixed solves reach the tolerance under the oracle's KKT evaluation.
    Covers ragged slices, empty columns, columns of more than 512 entries
    (chunked, their chunk sums added by the sliced kernel) and a column of
    5,000 entries."""
    m, n, dens, seed, lr, lc, sen = case
    d = random_lp(m, n, density=dens, seed=seed, long_rows=lr, long_cols=lc, senses=sen)
    lp = P.LP(d)
    kw = dict(tol=1e-6, max_iter=20480, check_every=64)
    a, b = lp.solve(spmv_layout=0, **kw), lp.solve(spmv_layout=1, **kw)
    assert a["info"]["status"] == b["info"]["status"] and a["info"]["iters"] == b["info"]["iters"]
    # sigma is the square root of a ratio of norms of displacements over a
    # restart cycle: its rounding is amplified like the residuals'
    _compare_logs(a["log"], b["log"], sigma_rtol=1e-7)
    assert _rel(a["x"], b["x"]) < 1e-8 and _rel(a["y"], b["y"]) < 1e-8
    for layout in (0, 1):
        r = lp.solve(spmv_layout=layout, tol=1e-4, precision="mixed", max_iter=20480)
        assert r["info"]["status"] == 0
        assert oracle.kkt(d, r["x"], r["y"], r["z"])["kkt"] <= 1e-4 * 1.0001


def _same_log(la, lb):
    """Check logs equal entry by entry, bit for bit (NaN equal to NaN)."""
    assert len(la) == len(lb)
    for ea, eb in zip(la, lb):
        assert ea.keys() == eb.keys()
        for k in ea:
            assert np.array_equal(np.float64(ea[k]), np.float64(eb[k]), equal_nan=True), (k, ea, eb)


FUSE_CASES = [
    (300, 200, 0.02, 1, 3, 2, "GLER"),       # sliced ELL primal step, no chunked rows
    (513, 1025, 0.01, 3, 2, 0, "LR"),        # rows of 1,025 entries: 3 chunks each
    (5000, 40, 0.002, 4, 0, 1, "GL"),        # a column of 5,000 entries (chunked primal)
    (2000, 3000, 0.003, 7, 20, 3, "GLER"),   # 20 rows of 6 chunks, 3 columns of 4 chunks
]


@pytest.mark.parametrize("case", FUSE_CASES)
@pytest.mark.parametrize("algo", ["hpr", "pdhg_avg"])
def test_fused_steps_agree(P, case, algo):
    """Plain iterations with the updates fused into the products' launches
    (the default) against separate launches on the CSR partition
    (split_steps = 1), through the solve graph and period by period.  With
    no row of A above 512 entries only the primal update moves (same sums):
    bit-identical iterates, logs and outputs.  Otherwise the dual step sums
    A's short rows on its sliced ELL copy, in row order: FP64 solves take
    the same restart decisions at every check with iterates equal to
    rounding, and FP32-matvec solves reach the tolerance under the oracle's
    KKT evaluation."""
    m, n, dens, seed, lr, lc, sen = case
    d = random_lp(m, n, density=dens, seed=seed, long_rows=lr, long_cols=lc, senses=sen)
    lp = P.LP(d)
    chunked_rows = max(np.diff(d["row_ptr"])) > 512
    for graph in (1, 0):
        kw = dict(tol=1e-7, max_iter=4096, check_every=64, algo=algo, precision="fp64", use_graph=graph)
        a, b = lp.solve(split_steps=0, **kw), lp.solve(split_steps=1, **kw)
        assert a["info"]["iters"] == b["info"]["iters"] and a["info"]["status"] == b["info"]["status"]
        if not chunked_rows:
            _same_log(a["log"], b["log"])
            for k in ("x", "y", "z"):
                assert np.array_equal(a[k], b[k]), (graph, k)
        else:
            _compare_logs(a["log"], b["log"], sigma_rtol=1e-7)
            assert _rel(a["x"], b["x"]) < 1e-8 and _rel(a["y"], b["y"]) < 1e-8
        kw.update(precision="mixed", tol=1e-4, max_iter=20480)
        a, b = lp.solve(split_steps=0, **kw), lp.solve(split_steps=1, **kw)
        if not chunked_rows:
            _same_log(a["log"], b["log"])
            assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["y"], b["y"])
        for r in (a, b):
            assert r["info"]["status"] == 0
            assert oracle.kkt(d, r["x"], r["y"], r["z"])["kkt"] <= 1e-4 * 1.0001


def test_fused_steps_scuc2k(P):
    """The same on the 2,000-bus relaxation (dense PTDF and N-1 rows chunked,
    sliced ELL copies of A and A^T), mixed precision to 1e-4 as the
    benchmark runs it: both points certified by the oracle, objectives
    within the tolerance's reach of each other."""
    inst = make_preset("scuc2k")
    lp = P.LP(inst)
    a = lp.solve(tol=1e-4, precision="mixed")
    b = lp.solve(tol=1e-4, precision="mixed", split_steps=1)
    for r in (a, b):
        assert r["info"]["status"] == 0
        assert oracle.kkt(inst, r["x"], r["y"], r["z"])["kkt"] <= 1e-4 * 1.0001
    assert abs(a["info"]["pobj"] - b["info"]["pobj"]) <= 1e-3 * abs(b["info"]["pobj"])


def test_solve_parity_scuc14(P):
    inst = make_preset("scuc14")
    kw = dict(tol=1e-4, max_iter=100000)
    o = oracle.hpr_solve(inst, **kw)
    g = P.LP(inst).solve(**kw)
    assert g["info"]["status"] == 0 and o["info"]["status"] == 0
    assert g["info"]["iters"] == o["info"]["iters"]
    _compare_logs(g["log"], o["log"])
    assert g["info"]["pobj"] == pytest.approx(o["info"]["pobj"], rel=1e-9)
    assert _rel(g["x"], o["x"]) < 1e-8
    k = oracle.kkt(inst, g["x"], g["y"], g["z"])
    assert k["kkt"] <= 1e-4


def test_solve_tight_objective_scuc14(P):
    """Both sides to 1e-7: relative objective difference <= 1e-5 (and far less)."""
    inst = make_preset("scuc14")
    o = oracle.hpr_solve(inst, tol=1e-7, max_iter=400000)
    for prec in ("fp64", "mixed"):
        g = P.LP(inst).solve(tol=1e-7, max_iter=400000, precision=prec)
        assert g["info"]["status"] == 0
        assert abs(g["info"]["pobj"] - o["info"]["pobj"]) <= 1e-5 * abs(o["info"]["pobj"])
        assert oracle.kkt(inst, g["x"], g["y"], g["z"])["kkt"] <= 1e-7 * 1.0001


def test_mixed_precision_kkt(P):
    inst = make_preset("scuc14")
    g = P.LP(inst).solve(tol=1e-4, precision="mixed")
    assert g["info"]["status"] == 0
    assert g["info"]["iters_fp32"] > 0
    k = oracle.kkt(inst, g["x"], g["y"], g["z"])
    assert k["kkt"] <= 1e-4
    o = oracle.hpr_solve(inst, tol=1e-4)
    # both within the 1e-4 gap of the same optimum
    assert abs(g["info"]["pobj"] - o["info"]["pobj"]) <= 4e-4 * abs(o["info"]["pobj"])


def test_warm_start_parity(P):
    d = random_lp(200, 150, density=0.03, seed=7, long_rows=1)
    x0 = seeded_vector(150, 1, -2, 2)
    y0 = seeded_vector(200, 2, -1, 1)
    kw = dict(tol=1e-6, max_iter=20480)
    o = oracle.hpr_solve(d, x_init=x0, y_init=y0, **kw)
    g = P.LP(d).solve(x0=x0, y0=y0, **kw)
    _compare_logs(g["log"], o["log"])
    assert _rel(g["x"], o["x"]) < 1e-8


def test_fixed_lambda_no_scaling_parity(P):
    d = random_lp(120, 90, density=0.05, seed=8, long_cols=1)
    lam = 1.5 * oracle.hpr_solve(d, use_scaling=0, max_iter=64)["info"]["lambda"]
    kw = dict(tol=1e-6, max_iter=20480, use_scaling=0, lambda_in=lam, sigma0=0.3, check_every=32)
    o = oracle.hpr_solve(d, **kw)
    g = P.LP(d).solve(**kw)
    _compare_logs(g["log"], o["log"])
    assert g["info"]["lambda"] == lam


@pytest.mark.parametrize("opts", [dict(use_scaling=2), dict(sigma_update=0, sigma0=0.5),
                                  dict(restart_ref=1, restart_metric=1),
                                  dict(restart_ref=1, restart_metric=2)])
def test_option_parity(P, opts):
    """Scaling, sigma and restart options take the same decisions on both sides."""
    d = random_lp(300, 200, density=0.02, seed=1, long_rows=3, long_cols=2)
    kw = dict(tol=1e-6, max_iter=20480, **opts)
    o = oracle.hpr_solve(d, **kw)
    g = P.LP(d).solve(**kw)
    _compare_logs(g["log"], o["log"])
    assert _rel(g["x"], o["x"]) < 1e-8


def test_bounds_only_and_empty_rows(P):
    rng = np.random.default_rng(0)
    n = 37
    c = rng.normal(size=n)
    xl = rng.uniform(-2, 0, n)
    xu = xl + 1
    d = dict(m=0, n=n, row_ptr=np.zeros(1, np.int64), col=np.zeros(0, np.int32), val=np.zeros(0),
             c=c, xl=xl, xu=xu, lo=np.zeros(0), hi=np.zeros(0))
    g = P.LP(d).solve(tol=1e-9)
    np.testing.assert_allclose(g["x"], np.where(c > 0, xl, xu), atol=1e-9)
    # a row with no entries (0 in [lo, hi]) and a column in no row
    d2 = dict(m=2, n=2, row_ptr=np.array([0, 1, 1], np.int64), col=np.array([0], np.int32),
              val=np.array([1.0]), c=np.array([1.0, -1.0]), xl=np.array([0.0, 0.0]),
              xu=np.array([5.0, 3.0]), lo=np.array([2.0, -1.0]), hi=np.array([np.inf, 1.0]))
    g2 = P.LP(d2).solve(tol=1e-9, max_iter=200000)
    assert g2["info"]["status"] == 0
    np.testing.assert_allclose(g2["x"], [2.0, 3.0], atol=1e-7)


def test_iteration_limit_and_graph_modes(P):
    inst = make_preset("scuc14")
    a = P.LP(inst).solve(tol=1e-12, max_iter=640, use_graph=1)
    b = P.LP(inst).solve(tol=1e-12, max_iter=640, use_graph=0, profile=1)
    assert a["info"]["status"] == 1 and a["info"]["iters"] == 640
    assert b["info"]["iters"] == 640 and b["info"]["n_dual_spmv"] == 640
    assert b["info"]["ms_dual_spmv"] > 0
    _compare_logs(a["log"], b["log"], rtol=0)
    np.testing.assert_array_equal(a["x"], b["x"])      # deterministic


def test_scuc2k_full_size(P):
    """2,000-bus instance (220k columns, N-1 rows): the first 256 iterations
    match the oracle check by check, and the 1e-4 solve is certified by the
    oracle's KKT evaluator."""
    inst = make_preset("scuc2k")
    kw = dict(tol=0.0, max_iter=256)
    o = oracle.hpr_solve(inst, **kw)
    lp = P.LP(inst)
    g = lp.solve(**kw)
    _compare_logs(g["log"], o["log"], rtol=1e-6)
    assert _rel(g["x"], o["x"]) < 1e-7
    for prec in ("fp64", "mixed"):
        s = lp.solve(tol=1e-4, precision=prec)
        assert s["info"]["status"] == 0, s["info"]
        assert oracle.kkt(inst, s["x"], s["y"], s["z"])["kkt"] <= 1e-4 * 1.0001


def test_scuc13k_full_size(P):
    """The 13,000-bus relaxation the benchmark solves (1.6M rows, 1.5M
    columns, 113M nonzeros), in the benchmark's launch configuration: the
    first 128 FP64 iterations (two check periods) match the oracle (OpenMP
    build on all host cores) check by check, and a solve to 1e-4 with FP32
    matvecs from cold start (the sliced copies on 16-bit offsets and the
    chunk stream) returns a point the oracle certifies."""
    inst = make_preset("scuc13k")
    kw = dict(tol=0.0, max_iter=128)
    o = oracle.hpr_solve(inst, threads=0, **kw)
    lp = P.LP(inst)
    g = lp.solve(**kw)
    _compare_logs(g["log"], o["log"], rtol=1e-6)
    assert _rel(g["x"], o["x"]) < 1e-7
    s = lp.solve(tol=1e-4, precision="mixed")
    assert s["info"]["status"] == 0 and s["info"]["iters_fp32"] == s["info"]["iters"], s["info"]
    k = oracle.kkt(inst, s["x"], s["y"], s["z"])
    assert k["kkt"] <= 1e-4 * 1.0001, k
    assert k["pobj"] == pytest.approx(s["info"]["pobj"], rel=1e-9)
    lay = lp.layout()
    assert lay["t_sell_compressed"] == 1 and lay["a_chunk32"] == 0 and lay["a_chunk16"] > 0.9 * inst.nnz
    lp.close()


def test_invalid_inputs_rejected_before_any_kernel(P):
    """Malformed inputs give SCUC_E_INVALID with the first failing row or
    column named (the entries are checked by several host threads while
    they are copied; the first failure in row order is reported)."""
    import scipy.sparse as sp
    good = random_lp(40, 30, density=0.2, seed=3)
    d0 = dict(m=good["m"], n=good["n"], row_ptr=good["row_ptr"].copy(), col=good["col"].copy(),
              val=good["val"].copy(), c=good["c"].copy(), xl=good["xl"].copy(), xu=good["xu"].copy(),
              sense=good["sense"].copy(), rhs=good["rhs"].copy(), rng_=good["rng_"].copy())
    P.LP(d0).close()

    def expect(d, text):
        with pytest.raises(P._lib.ScucError) as e:
            P.LP(d)
        assert e.value.code == P._lib.SCUC_E_INVALID
        assert text in str(e.value), str(e.value)

    r = int(np.argmax(np.diff(d0["row_ptr"]) >= 2))      # a row with two entries
    a = int(d0["row_ptr"][r])
    d = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in d0.items()}
    d["col"][a], d["col"][a + 1] = d["col"][a + 1], d["col"][a]
    expect(d, "not increasing in row %d" % r)
    d = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in d0.items()}
    d["col"][a] = d0["n"]
    expect(d, "out of range")
    d = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in d0.items()}
    d["val"][a] = np.nan
    expect(d, "non-finite matrix value in row %d" % r)
    d = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in d0.items()}
    d["xl"][5], d["xu"][5] = 1.0, 0.0
    expect(d, "invalid cost or bounds at column 5")
    d = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in d0.items()}
    d["row_ptr"][3] = d["row_ptr"][4] + 1
    expect(d, "row_ptr decreases")
    # a large LP (several host threads): errors in two chunks, the first row is reported
    big = sp.random(20000, 3000, density=0.02, random_state=np.random.default_rng(1), format="csr")
    big.sort_indices()
    db = dict(m=20000, n=3000, row_ptr=big.indptr.astype(np.int64), col=big.indices.astype(np.int32),
              val=big.data.copy(), c=np.ones(3000), xl=np.zeros(3000), xu=np.ones(3000),
              lo=np.full(20000, -np.inf), hi=np.full(20000, 10.0))
    P.LP(db).close()
    db["val"][big.indptr[17000]] = np.inf
    db["val"][big.indptr[1234] + 1] = np.nan
    expect(db, "non-finite matrix value in row 1234")


def test_create_page_locks_large_arrays_and_releases_them(P, torch_cuda):
    """scuc_lp_create page-locks matrix arrays of >= 64 MiB for the copy and
    releases them: the caller can register the same memory afterwards; an
    array the caller has already pinned is copied as it is (registration
    fails, plain copy); both give the same LP bit for bit."""
    import scipy.sparse as sp
    torch = torch_cuda
    m, n = 20000, 9000
    A = sp.random(m, n, density=0.05, random_state=np.random.default_rng(5), format="csr")   # 9M entries
    A.sort_indices()
    assert A.nnz * 8 >= 64 << 20
    d = dict(m=m, n=n, row_ptr=A.indptr.astype(np.int64), col=A.indices.astype(np.int32), val=A.data.copy(),
             c=np.ones(n), xl=np.zeros(n), xu=np.ones(n), lo=np.full(m, -np.inf), hi=np.full(m, 1.0))
    a = P.LP(d)
    cudart = torch.cuda.cudart()
    rc = cudart.cudaHostRegister(d["val"].ctypes.data, d["val"].nbytes, 0)
    assert int(rc) == 0, rc                        # released by create
    cudart.cudaHostUnregister(d["val"].ctypes.data)
    pinned = torch.from_numpy(d["val"]).pin_memory()            # caller-pinned copy of the values
    d2 = dict(d, val=pinned.numpy())
    b = P.LP(d2)
    ea, eb = a.export(), b.export()
    for k in ("row_ptr", "col", "val", "lo", "hi"):
        np.testing.assert_array_equal(ea[k], eb[k], err_msg=k)
    np.testing.assert_array_equal(eb["val"], d["val"])
    a.close()
    b.close()
