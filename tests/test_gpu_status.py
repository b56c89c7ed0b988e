"""GPU tests of the solve's stopping outcomes and of the precision switch
(Sec. 3.B: FP32 for the core steps, FP64 for the final phase), through the
C ABI: the switch to FP64 matvecs near the tolerance and on a stall, the
time limit, and the numerical stop (a NaN or infinite residual)."""
import numpy as np
import pytest

import oracle
from scuc_gen import make_preset

pytestmark = pytest.mark.gpu

ST = {"optimal": 0, "iter_limit": 1, "time_limit": 2, "numerical": 3}


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    import paper_2510_10891_b300 as P
    return P


@pytest.fixture(scope="module")
def scuc2k():
    return make_preset("scuc2k")


def _switch_check(log):
    """Index of the check after which the matvecs ran in FP64 (the log's fp64
    flag records the phase of the period that ended at the check)."""
    flags = [e["fp64"] for e in log]
    assert flags[0] == 0
    first = flags.index(1)
    assert all(flags[first:]), "the FP64 phase, once entered, is kept"
    return first - 1


def test_polish_switch_near_tolerance(P, scuc2k):
    """polish_factor = 10: the first check with KKT <= 10 tol moves the solve
    to FP64 matvecs; the FP32 iteration count ends there; the returned point
    meets the tolerance under the oracle's FP64 KKT evaluation."""
    tol = 1e-4
    r = P.LP(scuc2k).solve(tol=tol, precision="mixed", polish_factor=10.0, polish_stall=10 ** 6)
    i, log = r["info"], r["log"]
    assert i["status"] == ST["optimal"]
    assert 0 < i["iters_fp32"] < i["iters"]
    c = _switch_check(log)
    kkt = [max(e["rp"], e["rd"], e["gap"]) for e in log]
    assert kkt[c] <= 10.0 * tol and all(k > 10.0 * tol for k in kkt[:c])
    assert i["iters_fp32"] == log[c]["iter"]
    assert oracle.kkt(scuc2k, r["x"], r["y"], r["z"])["kkt"] <= tol * 1.0001


def test_polish_switch_at_floor(P, scuc2k):
    """polish_floor: below the tolerance trigger, the first check with KKT <=
    polish_floor moves the solve to FP64 matvecs (a tolerance below the
    accuracy FP32 matvecs reach gets an FP64 final phase)."""
    tol, floor = 1e-5, 1e-4
    r = P.LP(scuc2k).solve(tol=tol, precision="mixed", polish_floor=floor, polish_stall=10 ** 6)
    i, log = r["info"], r["log"]
    assert i["status"] == ST["optimal"]
    assert 0 < i["iters_fp32"] < i["iters"]
    c = _switch_check(log)
    kkt = [max(e["rp"], e["rd"], e["gap"]) for e in log]
    assert kkt[c] <= floor and all(k > floor for k in kkt[:c])
    assert i["iters_fp32"] == log[c]["iter"]
    assert oracle.kkt(scuc2k, r["x"], r["y"], r["z"])["kkt"] <= tol * 1.0001
    # with the default floor (1e-6) the same solve keeps FP32 matvecs throughout
    d = P.LP(scuc2k).solve(tol=tol, precision="mixed", want=("x",))["info"]
    assert d["status"] == ST["optimal"] and d["iters_fp32"] == d["iters"]


def test_polish_switch_on_stall(P, scuc2k):
    """polish_stall = 2 (and no tolerance trigger): the switch follows the
    stall rule replayed on the logged KKT values (a check that does not cut
    the best KKT so far by 10% counts as a stall; two in a row switch)."""
    tol = 1e-4
    r = P.LP(scuc2k).solve(tol=tol, precision="mixed", polish_factor=0.0, polish_stall=2)
    i, log = r["info"], r["log"]
    assert i["status"] == ST["optimal"]
    assert 0 < i["iters_fp32"] < i["iters"]
    best, stall, want = np.inf, 0, None
    for j, e in enumerate(log):
        k = max(e["rp"], e["rd"], e["gap"])
        if k < 0.9 * best:
            best, stall = k, 0
        else:
            stall += 1
        if stall >= 2:
            want = j
            break
    assert want is not None
    assert _switch_check(log) == want
    assert i["iters_fp32"] == log[want]["iter"]
    assert oracle.kkt(scuc2k, r["x"], r["y"], r["z"])["kkt"] <= tol * 1.0001


@pytest.mark.parametrize("use_graph", [1, 0])
def test_time_limit(P, use_graph):
    """A time limit shorter than one period stops the solve at its first
    check with SCUC_ST_TIME_LIMIT; the returned point is that check's, whose
    residuals the oracle reproduces."""
    inst = make_preset("scuc14")
    r = P.LP(inst).solve(tol=1e-12, time_limit_s=1e-9, use_graph=use_graph)
    i = r["info"]
    assert i["status"] == ST["time_limit"], i["status_name"]
    assert i["iters"] == 64 and len(r["log"]) == 1
    k = oracle.kkt(inst, r["x"], r["y"], r["z"])
    assert k["kkt"] == pytest.approx(i["kkt"], rel=1e-7)
    # the same solve without a limit goes on past that check
    assert P.LP(inst).solve(tol=1e-12, max_iter=256, use_graph=use_graph)["info"]["iters"] == 256


@pytest.mark.parametrize("use_scaling", [0, 1])
def test_numerical_stop(P, use_scaling):
    """Finite data whose iterates overflow (cost -1e300, a 1e10 coefficient):
    a residual becomes NaN at the first check and the solve stops there with
    SCUC_ST_NUMERICAL, as the oracle does, instead of taking the NaN for a
    small error."""
    inf = np.inf
    lp = dict(m=1, n=1, row_ptr=np.array([0, 1]), col=np.array([0]), val=np.array([1e10]),
              c=np.array([-1e300]), xl=np.array([0.0]), xu=np.array([inf]), lo=np.array([0.0]),
              hi=np.array([inf]))
    o = oracle.hpr_solve(lp, tol=1e-6, use_scaling=use_scaling, max_iter=640)
    assert o["info"]["status"] == ST["numerical"] and o["info"]["iters"] == 64
    for graph in (1, 0):
        r = P.LP(lp).solve(tol=1e-6, use_scaling=use_scaling, max_iter=640, use_graph=graph)
        assert r["info"]["status"] == ST["numerical"], r["info"]["status_name"]
        assert r["info"]["iters"] == 64
        assert not np.isfinite(r["info"]["kkt"])
