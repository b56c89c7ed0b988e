"""GPU parity of the second algorithm (restarted PDHG with ergodic averaging)
and of infeasibility detection with the CPU oracle, through the C ABI.  FP64
PDHG runs take the oracle's restart decisions at every check (same iteration
counts, KKT values to 1e-7 relative); detection gives the oracle's verdict
at the same check, and the returned rays satisfy the certificates' defining
inequalities on the unscaled LP."""
import numpy as np
import pytest

import oracle
from lp_cases import (DUAL_INFEASIBLE, PRIMAL_INFEASIBLE, farkas, highs_status, infeasible_box, recession,
                      unbounded)
from scuc_gen import make_preset, random_lp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2510_10891_b300 as P
    return P


def _compare_logs(glog, olog, rtol=1e-7):
    assert len(glog) == len(olog), (len(glog), len(olog))
    for g, o in zip(glog, olog):
        assert g["iter"] == o["iter"]
        assert g["restart"] == o["restart"], (g, o)
        for k in ("rp", "rd"):
            assert g[k] == pytest.approx(o[k], rel=rtol, abs=1e-13), (k, g, o)
        assert g["gap"] == pytest.approx(o["gap"], rel=rtol, abs=1e-11), ("gap", g, o)
        # sigma is a ratio of the norms of (average - previous restart point):
        # a difference of averaged iterates, so the rounding differences of
        # the iterates reach it amplified like the residuals above
        assert g["sigma"] == pytest.approx(o["sigma"], rel=rtol)


CASES = [(40, 30, 0.2, 0, 0, 0, "GLER"), (300, 200, 0.02, 1, 3, 2, "GLER"), (513, 1025, 0.01, 3, 2, 0, "LR")]


@pytest.mark.parametrize("case", CASES)
def test_pdhg_solve_parity_random(P, case):
    m, n, dens, seed, lr, lc, sen = case
    d = random_lp(m, n, density=dens, seed=seed, long_rows=lr, long_cols=lc, senses=sen)
    kw = dict(tol=1e-6, max_iter=20480, algo=1)
    g = P.LP(d).solve(**kw)
    o = oracle.hpr_solve(d, **kw)
    assert g["info"]["status"] == o["info"]["status"]
    assert g["info"]["iters"] == o["info"]["iters"]
    assert g["info"]["restarts"] == o["info"]["restarts"]
    _compare_logs(g["log"], o["log"])
    for k in ("x", "y", "z"):
        scale = max(1.0, float(np.max(np.abs(o[k]))))
        assert float(np.max(np.abs(g[k] - o[k]))) <= 1e-8 * scale, k


def test_pdhg_parity_scuc14_and_graph_modes(P):
    inst = make_preset("scuc14")
    kw = dict(tol=1e-6, max_iter=40960, algo="pdhg_avg")
    lp = P.LP(inst)
    g = lp.solve(**kw)
    o = oracle.hpr_solve(inst, **{**kw, "algo": 1})
    assert g["info"]["status"] == 0 and o["info"]["status"] == 0
    assert g["info"]["iters"] == o["info"]["iters"]
    _compare_logs(g["log"], o["log"])
    assert g["info"]["pobj"] == pytest.approx(o["info"]["pobj"], rel=1e-9)
    # one graph launch and period-by-period launches give the same result
    h = lp.solve(use_graph=0, **kw)
    np.testing.assert_array_equal(g["x"], h["x"])
    assert g["info"]["iters"] == h["info"]["iters"]


def test_pdhg_mixed_precision_scuc2k_certified(P):
    inst = make_preset("scuc2k")
    r = P.LP(inst).solve(tol=1e-4, precision="mixed", algo="pdhg_avg")
    assert r["info"]["status"] == 0
    assert r["info"]["iters_fp32"] > 0
    k = oracle.kkt(inst, r["x"], r["y"], r["z"])
    assert k["kkt"] <= 1e-4 * 1.0001, k


@pytest.mark.parametrize("algo", [0, 1])
@pytest.mark.parametrize("seed", range(4))
def test_detection_verdicts_and_certificates(P, algo, seed):
    for lp, verdict in ((infeasible_box(seed), PRIMAL_INFEASIBLE), (unbounded(seed), DUAL_INFEASIBLE)):
        assert highs_status(lp)[0] == (2 if verdict == PRIMAL_INFEASIBLE else 3)
        kw = dict(tol=1e-8, max_iter=100000, algo=algo, infeas_tol=1e-8)
        g = P.LP(lp).solve(**kw)
        o = oracle.hpr_solve(lp, **kw)
        assert o["info"]["status"] == verdict
        assert g["info"]["status"] == verdict, g["info"]["status_name"]
        assert g["info"]["iters"] == o["info"]["iters"]     # found at the same check
        if verdict == PRIMAL_INFEASIBLE:
            F, V = farkas(lp, g["y"])
            assert F > 0 and V <= 1e-6 * F, (F, V)
        else:
            cd, V = recession(lp, g["x"])
            assert cd < 0 and V <= 1e-6 * -cd, (cd, V)


@pytest.mark.parametrize("algo", [0, 1])
def test_detection_silent_on_feasible_lps(P, algo):
    """Detection never fires on feasible bounded LPs and does not change the
    iteration: the same result bit for bit as without it."""
    for src in [random_lp(300, 200, density=0.02, seed=1, long_rows=3, long_cols=2), make_preset("scuc14")]:
        lp = P.LP(src)
        kw = dict(tol=1e-6, max_iter=40960, algo=algo)
        a = lp.solve(infeas_tol=1e-8, **kw)
        b = lp.solve(**kw)
        assert a["info"]["status"] == 0
        assert a["info"]["iters"] == b["info"]["iters"]
        np.testing.assert_array_equal(a["x"], b["x"])
        assert a["info"]["launches"] > b["info"]["launches"]    # the certificate products ran


def test_batch_rejects_pdhg_and_detection(P):
    hs = [P.LP(random_lp(40, 30, density=0.2, seed=s)) for s in (1, 2)]
    for kw in (dict(algo=1), dict(infeas_tol=1e-8)):
        with pytest.raises(P._lib.ScucError) as e:
            P.solve_batch(hs, **kw)
        assert e.value.code == P._lib.SCUC_E_INVALID


def test_invalid_algo_rejected(P):
    lp = P.LP(random_lp(40, 30, density=0.2, seed=1))
    for kw in (dict(algo=2), dict(infeas_tol=-1.0)):
        with pytest.raises(P._lib.ScucError):
            lp.solve(**kw)
