"""GPU parity of the fixing round (Round + Algorithm 1, Sec. 4.1) and of the
presolve of Algorithm 2 (bound propagation + reduced LP, Sec. 4.2) with the
CPU oracle, through the C ABI.  Integer and index results are compared
bit for bit (fix decisions, pass counts, integer bounds, fixed columns, maps,
reduced structure); continuous bounds and folded row bounds, which the two
sides sum in different orders, within the error bound of that order
(tests/fixcmp.py)."""
import numpy as np
import pytest

import fixcmp
import oracle
from scuc_gen import make_preset, random_lp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    import paper_2510_10891_b300 as P
    return P


def _oracle_round(inst, lp_d, x, tau, t_first=1):
    fix, nf = oracle.fix(inst.G, inst.T, x[inst.u_idx], x[inst.v_idx], x[inst.w_idx], inst.u_init, tau,
                         t_first)
    xl, xu = lp_d["xl"].copy(), lp_d["xu"].copy()
    F = fix.reshape(-1, 3)
    for slot, idx in enumerate((inst.u_idx, inst.v_idx, inst.w_idx)):
        sel = F[:, slot] >= 0
        xl[idx[sel]] = F[sel, slot]
        xu[idx[sel]] = F[sel, slot]
    pl, pu, passes = oracle.propagate(lp_d, xl, xu, inst.is_int)
    return fix, nf, pl, pu, passes, (xl, xu)


def _same_transpose(P, reduced, exported):
    """The reduced LP's A^T, compacted on the device from the parent's, is the
    one a new handle builds from the exported LP (sorted by row within each
    column): A^T y and A x agree bit for bit."""
    import torch
    fresh = P.LP(exported)
    g = torch.Generator().manual_seed(7)
    y = torch.randn(reduced.m, generator=g, dtype=torch.float64).cuda()
    x = torch.randn(reduced.n, generator=g, dtype=torch.float64).cuda()
    outs = {}
    for name, h in (("reduced", reduced), ("fresh", fresh)):
        outs[name] = (h.matvec(y, torch.empty(reduced.n, dtype=torch.float64, device="cuda"), transpose=True),
                      h.matvec(x, torch.empty(reduced.m, dtype=torch.float64, device="cuda")))
    for a, b in zip(outs["reduced"], outs["fresh"]):
        assert torch.equal(a, b)
    fresh.close()


@pytest.mark.parametrize("name,tau,t_first", [("scuc14", 0.1, 1), ("scuc14", 0.3, 0),
                                              ("scuc2k", 0.1, 1), ("scuc2k", 0.02, 1)])
def test_fix_propagate_reduce_parity(P, name, tau, t_first):
    inst = make_preset(name)
    lp_d = oracle.as_lp(inst)
    x = oracle.hpr_solve(inst, tol=1e-4, max_iter=200000)["x"] if name == "scuc14" else \
        P.LP(inst).solve(tol=1e-4)["x"]
    fix, nf, pl, pu, passes, init = _oracle_round(inst, lp_d, x, tau, t_first)
    lp = P.LP(inst)
    r = lp.fix_and_propagate(inst.G, inst.T, inst.u_idx, inst.v_idx, inst.w_idx, inst.u_init, x, tau=tau,
                             t_first=t_first, is_int=inst.is_int)
    np.testing.assert_array_equal(r["fix"], fix)
    assert r["info"]["nfixed"] == nf and nf > 0
    assert r["infeasible"] == (passes < 0)      # both sides agree on infeasibility
    if passes < 0:
        assert r["info"]["passes"] == -passes
        return
    assert r["info"]["passes"] == passes
    gxl, gxu = lp.get_bounds()
    fixcmp.assert_bounds_match(lp_d, inst.is_int, gxl, gxu, pl, pu, passes, init)
    red, rmap, cmap, oc, bad = oracle.reduce(lp_d, pl, pu)
    assert bad == 0
    gi = r["info"]
    assert (gi["m_red"], gi["n_red"], gi["nnz_red"]) == (red["m"], red["n"], len(red["val"]))
    np.testing.assert_array_equal(r["row_map"], rmap)
    np.testing.assert_array_equal(r["col_map"], cmap)
    assert gi["obj_const"] == pytest.approx(oc, rel=1e-12, abs=1e-12)
    g = r["reduced"].export()
    fixcmp.assert_reduced_match(lp_d, g, red, rmap, cmap, gxl, gxu, pl, pu)
    _same_transpose(P, r["reduced"], g)
    # the reduced LP solves; small case: to the oracle's optimum, large case:
    # certified by the oracle's KKT evaluator on the reduced LP
    if name == "scuc14":
        s = r["reduced"].solve(tol=1e-6, max_iter=200000)
        o = oracle.hpr_solve(red, tol=1e-6, max_iter=200000)
        assert s["info"]["status"] == 0 and o["info"]["status"] == 0
        assert s["info"]["pobj"] == pytest.approx(o["info"]["pobj"], rel=1e-6)
    else:
        s = r["reduced"].solve(tol=1e-4)
        assert s["info"]["status"] == 0
        assert oracle.kkt(red, s["x"], s["y"], s["z"])["kkt"] <= 1e-4 * 1.0001


def test_propagation_random_binary_parity(P):
    """Random LPs around an integral point, half the columns integer: the
    propagation is feasible and tightens bounds; pass counts and integer
    bounds equal the oracle's, continuous bounds within the order bound, and
    the reduced LP matches."""
    for seed in range(8):
        d, is_int = fixcmp.propagation_case(seed)
        d = oracle.as_lp(d)
        pl, pu, passes = oracle.propagate(d, d["xl"], d["xu"], is_int)
        assert passes > 1
        lp = P.LP(d)
        # empty map: propagation only
        r = lp.fix_and_propagate(0, 1, np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(d["n"]),
                                 is_int=is_int)
        assert not r["infeasible"]
        assert r["info"]["passes"] == passes
        gxl, gxu = lp.get_bounds()
        fixcmp.assert_bounds_match(d, is_int, gxl, gxu, pl, pu, passes, (d["xl"], d["xu"]))
        red, rmap, cmap, oc, bad = oracle.reduce(d, pl, pu)
        np.testing.assert_array_equal(r["row_map"], rmap)
        np.testing.assert_array_equal(r["col_map"], cmap)
        fixcmp.assert_reduced_match(d, r["reduced"].export(), red, rmap, cmap, gxl, gxu, pl, pu)
        r["reduced"].close()


def test_propagation_random_infeasible_verdicts(P):
    """Random LPs whose integer columns have boxes without enough integers:
    the GPU declares infeasibility in the same pass as the oracle."""
    for seed in range(5):
        d = random_lp(120, 80, density=0.05, seed=seed, long_rows=2)
        d = oracle.as_lp(d)
        rng = np.random.default_rng(seed)
        is_int = (rng.random(80) < 0.5).astype(np.uint8)
        pl, pu, passes = oracle.propagate(d, d["xl"], d["xu"], is_int)
        assert passes < 0
        lp = P.LP(d)
        r = lp.fix_and_propagate(0, 1, np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(80),
                                 is_int=is_int, build_reduced=False)
        assert r["infeasible"]
        assert r["info"]["passes"] == -passes


def test_successive_rounds(P):
    """Algorithm 2 loop on the 2,000-bus LP: solve, fix, propagate, re-solve the
    reduced LP, map back; the fixed set only grows and every reduced LP solves."""
    inst = make_preset("scuc2k")
    lp = P.LP(inst)
    x = lp.solve(tol=1e-4)["x"]
    prev = 0
    for rnd in range(3):
        r = lp.fix_and_propagate(inst.G, inst.T, inst.u_idx, inst.v_idx, inst.w_idx, inst.u_init, x, tau=0.1)
        assert not r["infeasible"]
        xl, xu = lp.get_bounds()
        nfixed = int(np.sum(xl == xu))
        assert nfixed >= prev
        prev = nfixed
        red = r["reduced"]
        s = red.solve(tol=1e-4)
        assert s["info"]["status"] == 0
        x = xl.copy()                       # fixed columns at their values
        x[r["col_map"]] = s["x"]            # free columns from the reduced solve


def test_fix_propagate_full_size_13k(P):
    """The 13,000-bus LP (the benchmarked workload, same launch path as
    bench.py): fixing decisions, propagated bounds and reduced-LP sizes and
    maps equal the oracle's on the same solution."""
    inst = make_preset("scuc13k")
    d = oracle.as_lp(inst)
    lp = P.LP(inst)
    x = lp.solve(tol=1e-4, precision="mixed")["x"]
    fix, nf, pl, pu, passes, init = _oracle_round(inst, d, x, 0.1)
    r = lp.fix_and_propagate(inst.G, inst.T, inst.u_idx, inst.v_idx, inst.w_idx, inst.u_init, x, tau=0.1,
                             is_int=inst.is_int)
    np.testing.assert_array_equal(r["fix"], fix)
    assert r["infeasible"] == (passes < 0)
    if passes < 0:
        return
    assert r["info"]["passes"] == passes
    gxl, gxu = lp.get_bounds()
    fixcmp.assert_bounds_match(d, inst.is_int, gxl, gxu, pl, pu, passes, init)
    red, rmap, cmap, oc, bad = oracle.reduce(d, pl, pu)
    gi = r["info"]
    assert (gi["m_red"], gi["n_red"], gi["nnz_red"]) == (red["m"], red["n"], len(red["val"]))
    np.testing.assert_array_equal(r["row_map"], rmap)
    np.testing.assert_array_equal(r["col_map"], cmap)
    g = r["reduced"].export()
    fixcmp.assert_reduced_match(d, g, red, rmap, cmap, gxl, gxu, pl, pu)
    _same_transpose(P, r["reduced"], g)
