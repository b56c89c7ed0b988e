"""Per generator-hour inputs of the learned warm start.

Like the rest of ``scuc_gen`` this only builds *inputs* from an instance's
data (units, load, grid); it holds none of the solver's or the network's
arithmetic.  Rows are unit-hours k = g*T + t (g-major, the order of
``SCUCInstance.u_idx``).

Features (all ratios, so that instances of different sizes share one scale):
  0-2  segment costs c_{g,h} / eta^C (Eq. 7; eta^C = the largest cost)
  3    P^U_g / mean P^U     4  P^L_g / mean P^U     5  ramp RU_g / mean P^U
  6    system load D_t / sum P^U (Eq. 6)
  7    load of the unit's bus and its neighbours, per bus, / (D_t / buses)
  8    merit position: share of sum P^U held by units with a lower average
       cost at full output
  9    D_{t+1}/sum P^U - feature 6 (0 in the last hour)
  10   D_{t-1}/sum P^U - feature 6 (0 in the first hour)
  11   feature 8 - feature 6
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

NFEAT = 12


def ws_features(inst) -> np.ndarray:
    p = inst.params
    G, T = inst.G, inst.T
    pmax, pmin, ru, segc, segw = p["pmax"], p["pmin"], p["ru"], p["segc"], p["segw"]
    Dt, Dbt, fr, to, bus = p["Dt"], p["Dbt"], p["fr"], p["to"], p["bus_g"]
    B = Dbt.shape[0]
    etaC = float(segc.max())
    mp = float(pmax.mean())
    cap = float(pmax.sum())
    avgc = (pmin * segc[:, 0] + (segw * segc).sum(axis=1)) / pmax
    order = np.argsort(avgc, kind="stable")
    below = np.zeros(G)
    below[order] = np.cumsum(pmax[order]) - pmax[order]
    merit = below / cap
    adj = sp.coo_matrix((np.ones(2 * len(fr)), (np.r_[fr, to], np.r_[to, fr])), shape=(B, B)).tocsr()
    deg = np.asarray(adj.sum(axis=1)).ravel()
    local = (Dbt + adj @ Dbt) / (1.0 + deg)[:, None] / (Dt / B)[None, :]     # [B, T]
    lr = Dt / cap
    X = np.zeros((G, T, NFEAT), np.float64)
    X[:, :, 0:3] = (segc / etaC)[:, None, :]
    X[:, :, 3] = (pmax / mp)[:, None]
    X[:, :, 4] = (pmin / mp)[:, None]
    X[:, :, 5] = (ru / mp)[:, None]
    X[:, :, 6] = lr[None, :]
    X[:, :, 7] = local[bus, :]
    X[:, :, 8] = merit[:, None]
    X[:, :, 9] = (np.r_[lr[1:], lr[-1:]] - lr)[None, :]
    X[:, :, 10] = (np.r_[lr[:1], lr[:-1]] - lr)[None, :]
    X[:, :, 11] = merit[:, None] - lr[None, :]
    return X.reshape(G * T, NFEAT).astype(np.float32)


def ws_layout_arrays(inst) -> dict:
    """Index and capacity arrays of the warm-start layout (host numpy).

    Unit-hour k = g*T + t: columns of u, v, w, p' and the cost segments
    (Eq. 1, 3, 5), the capacities P^U - P^L and the segment widths in LP units
    (the column upper bounds of the unfixed model), the commitment before
    the first hour, and the row whose dual is the unit-hour's price: the
    system balance row of hour t (Eq. 6, PTDF network) or the nodal balance
    row of the unit's bus (B-theta network).  The dual of a balance row is
    price_scale times the price in units of eta^C per MWh (Sec. 3.A scaling:
    costs times eta^P/eta^C, powers over eta^P)."""
    G, T = inst.G, inst.T
    k = np.arange(G * T)
    g, t = k // T, k % T
    u = inst.u_idx.astype(np.int32)
    p_col = (u + 3).astype(np.int32)
    seg_col = np.stack([u + 4, u + 5, u + 6], axis=1).astype(np.int32)
    rb0 = inst.params["row_blocks"]["bus"][0]
    if inst.params["network"] == "ptdf":
        unit_row = (rb0 + t).astype(np.int32)
    else:
        B = inst.cfg.buses
        unit_row = (rb0 + t * B + inst.params["bus_g"][g]).astype(np.int32)
    # price rows and their members (unit-hours), members in increasing k
    order = np.argsort(unit_row, kind="stable")
    rows, first = np.unique(unit_row[order], return_index=True)
    ptr = np.r_[first, len(order)].astype(np.int32)
    return dict(G=G, T=T, u_col=u, v_col=(u + 1).astype(np.int32), w_col=(u + 2).astype(np.int32),
                p_col=p_col, seg_col=seg_col, p_cap=inst.xu[p_col].astype(np.float64),
                seg_cap=inst.xu[seg_col].astype(np.float64), u_init=inst.u_init.astype(np.float64),
                unit_price_row=unit_row, price_row=rows.astype(np.int32), price_ptr=ptr,
                price_member=order.astype(np.int32), price_scale=float(inst.power_scale))
