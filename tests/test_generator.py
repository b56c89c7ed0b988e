"""The synthetic SCUC generator builds the rows of Sec. 2 (Eqs. 1-7): checked
by evaluating a hand-built schedule (all units on at the proportional
dispatch, DC power-flow angles) against every row and against Eq. 7."""
import numpy as np
import pytest

import oracle
from scuc_gen import make_preset
from scuc_gen.scuc import NVU, P, S1, U, V, W


@pytest.mark.parametrize("name", ["scuc14"])
def test_sizes_and_layout(name):
    inst = make_preset(name)
    G, T, B = inst.G, inst.T, inst.cfg.buses
    assert inst.n == 7 * G * T + 2 * B * T
    assert inst.m == 11 * G * T + B * T + inst.cfg.lines * T + T + inst.cfg.contingencies * T
    assert np.all(np.diff(inst.row_ptr) > 0)
    assert inst.is_int.sum() == 3 * G * T
    assert np.all(inst.xl[inst.u_idx] == 0) and np.all(inst.xu[inst.u_idx] == 1)


def _schedule(inst):
    """All units on, proportional dispatch, segments filled in order, angles
    from the DC power flow of the resulting injections, no unserved load."""
    p = inst.params
    G, T, B = inst.G, inst.T, inst.cfg.buses
    etaP = inst.power_scale
    share = p["pmax"] / p["pmax"].sum()
    x = np.zeros(inst.n)
    nU = 7 * G * T
    for t in range(T):
        for g in range(G):
            base = (t * G + g) * NVU
            tot = share[g] * p["Dt"][t]
            x[base + U] = 1.0
            above = (tot - p["pmin"][g]) / etaP
            x[base + P] = above
            left = above
            for h in range(3):
                take = min(left, p["segw"][g, h] / etaP)
                x[base + S1 + h] = take
                left -= take
    if inst.cfg.network == "ptdf":
        return x
    # angles: solve the nodal balance for theta (reference bus 0)
    from scuc_gen.scuc import _DCGrid
    dc = _DCGrid(B, p["fr"], p["to"], p["x"])
    gen = np.zeros((B, T))
    np.add.at(gen, p["bus_g"], share[:, None] * p["Dt"][None, :])
    th = dc.angles((gen - p["Dbt"]) / 100.0)
    for t in range(T):
        x[nU + (t * B + np.arange(B)) * 2] = th[:, t]
    return x


def test_rows_hold_for_a_feasible_schedule():
    inst = make_preset("scuc14")
    lp = oracle.as_lp(inst)
    x = _schedule(inst)
    import scipy.sparse as sp
    ax = inst.csr() @ x
    tol = 1e-9
    blocks = inst.params["row_blocks"]
    lo, hi = lp["lo"], lp["hi"]
    bad = np.flatnonzero((ax < lo - tol) | (ax > hi + tol))
    # the schedule violates at most ramp rows at hour changes larger than the ramp
    # limit (none for this load profile) and nothing else
    assert bad.size == 0, [(int(i), ax[i], lo[i], hi[i]) for i in bad[:5]]
    # nodal balance is tight (Eq. 6 with B-theta)
    b0, b1 = blocks["bus"]
    np.testing.assert_allclose(ax[b0:b1], lo[b0:b1], rtol=0, atol=1e-9)
    # Eq. 7 objective in model units
    p = inst.params
    share = p["pmax"] / p["pmax"].sum()
    cost = 0.0
    for t in range(inst.T):
        for g in range(inst.G):
            tot = share[g] * p["Dt"][t]
            left = tot - p["pmin"][g]
            c = p["pmin"][g] * p["segc"][g, 0]
            for h in range(3):
                take = min(left, p["segw"][g, h])
                c += take * p["segc"][g, h]
                left -= take
            cost += c
    assert float(inst.c @ x) * inst.objective_scale == pytest.approx(cost, rel=1e-12)


def test_dense_rows_present():
    inst = make_preset("scuc14", contingencies=3)
    b0, b1 = inst.params["row_blocks"]["ctg"]
    assert b1 - b0 == 3 * inst.T
    lens = np.diff(inst.row_ptr)[b0:b1]
    assert lens.min() > 4


def test_ptdf_network_rows():
    """Eq. 6 as written (network="ptdf"): one balance row per hour, tight at
    the proportional dispatch; base-case PTDF rows of the monitored lines hold
    with the 1.5x margin the limits were sized with; no angle columns."""
    from scuc_gen import SCUCConfig, make_scuc
    inst = make_scuc(SCUCConfig(buses=60, lines=84, units=12, T=8, contingencies=4, seed=5,
                                network="ptdf"))
    G, T, B = inst.G, inst.T, inst.cfg.buses
    assert inst.n == 7 * G * T + B * T
    assert np.all(np.isfinite(inst.xl)) and np.all(np.isfinite(inst.xu))
    lp = oracle.as_lp(inst)
    x = _schedule(inst)
    ax = inst.csr() @ x
    blocks = inst.params["row_blocks"]
    b0, b1 = blocks["bus"]
    assert b1 - b0 == T
    np.testing.assert_allclose(ax[b0:b1], lp["lo"][b0:b1], rtol=1e-12)
    l0, l1 = blocks["line"]
    assert l1 - l0 == 4 * T
    w = (lp["hi"][l0:l1] - lp["lo"][l0:l1]) / 2
    mid = (lp["hi"][l0:l1] + lp["lo"][l0:l1]) / 2
    assert np.all(np.abs(ax[l0:l1] - mid) <= w / 1.5 + 2e-3 * np.abs(mid).max() + 1e-9)
    u0, u1 = blocks["unit"]
    assert np.all(ax[u0:u1] >= lp["lo"][u0:u1] - 1e-9) and np.all(ax[u0:u1] <= lp["hi"][u0:u1] + 1e-9)


def test_split_network_rows_partitions_the_rows():
    """Transmission-filtering split: the pool is exactly the base-case line
    and N-1 row blocks, the base is every other row, and together they are
    the full instance's rows (same columns, values and row bounds)."""
    import numpy as np
    import scipy.sparse as sp
    from scuc_gen import make_preset, split_network_rows
    inst = make_preset("scuc14")
    base, pool, pool_rows = split_network_rows(inst)
    blocks = inst.params["row_blocks"]
    want = np.concatenate([np.arange(*blocks["line"]), np.arange(*blocks["ctg"])])
    np.testing.assert_array_equal(pool_rows, want)
    assert base["m"] + pool["m"] == inst.m and base["n"] == pool["n"] == inst.n
    A = inst.csr()
    lo, hi = inst.row_bounds()
    base_rows = np.setdiff1d(np.arange(inst.m), pool_rows)
    for part, rows in ((base, base_rows), (pool, pool_rows)):
        P = sp.csr_matrix((part["val"], part["col"], part["row_ptr"]), shape=(part["m"], part["n"]))
        assert (P != A[rows]).nnz == 0
        np.testing.assert_array_equal(part["lo"], lo[rows])
        np.testing.assert_array_equal(part["hi"], hi[rows])
        np.testing.assert_array_equal(part["c"], inst.c)
