"""Seeded synthetic SCUC instances and the LP relaxation of their 3-binary model.

This module only builds *inputs*: the grid, the units, the load, and the
constraint matrix of the SCUC model of Sec. 2 (Eqs. 1-7) with the binaries
relaxed to [0, 1].  It holds none of the solver's arithmetic (no scaling of
the matrix, no iteration, no fixing); both the CPU oracle and the CUDA
library receive exactly the arrays produced here.

Layout: unit columns and unit rows are hour-major ((t*G + g)*7 + slot and
(t*G + g)*11 + row), bus columns are hour-major ((t*B + b)*2 + slot), and the
buses are numbered in Morton order of their positions, so the dense N-1 rows
of one hour and the rows of one unit gather from a few contiguous blocks.

Model (Sec. 2), per unit g and hour t (0-based t here, hour t+1 in the paper):
    variables  u, v, w (commitment/start/stop, relaxed to [0,1]),
               p' (output above P^L), p_1..p_3 (piecewise segments);
per bus b and hour t:
    theta (bus angle, free; reference bus fixed to 0), d^pen (unserved load).
Rows per (g,t): Eq. 1 (logic, v+w<=1), Eq. 2 (min up / min down),
Eq. 3 (production limit), Eq. 4 (ramp up / down), Eq. 5 (segment caps and
segment sum; the cost variable c is eliminated into the objective, Eq. 7).
System rows: nodal B-theta balance per (b,t) and a ranged flow row per
(l,t) stand in for the base-case PTDF rows of Eq. 6; the N-1 rows of Eq. 6
are dense PTDF+LODF rows for the K most loaded lines; a 3 % spinning reserve
row per hour.

Instance-aware scaling (Sec. 3.A) is a change of units of the *model
parameters* made before the matrix exists, so it is applied here when
``eta_scaling`` is on: production quantities are divided by eta^P and costs
multiplied by eta^P/eta^C.  ``objective_scale`` (= eta^C) and
``power_scale`` (= eta^P) recover model units.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.sparse.csgraph import connected_components, minimum_spanning_tree
from scipy.spatial import cKDTree

# per-(g,t) variable slots; columns are hour-major: ((t*G + g)*7 + slot)
U, V, W, P, S1, S2, S3 = range(7)
NVU = 7
# per-(g,t) row slots
R_LOGIC, R_VW, R_MINUP, R_MINDN, R_PROD, R_RUP, R_RDN, R_SEG1, R_SEG2, R_SEG3, R_SEGSUM = range(11)
NRU = 11
INF = np.inf


@dataclass
class SCUCConfig:
    """Sizes and distributions of one synthetic instance."""

    buses: int
    lines: int
    units: int
    T: int
    contingencies: int = 0
    seed: int = 1
    eta_scaling: bool = True
    # "pmax": eta^P = max_g P^U_g (the text of Sec. 3.A, which names the
    # maximum production limit); "pmin": max_g P^L_g (its displayed formula).
    eta_reading: str = "pmax"
    ptdf_trunc: float = 1e-3
    reserve_frac: float = 0.03
    load_frac: float = 0.6
    load_amp: float = 0.2
    load_noise: float = 0.1
    penalty: float = 1000.0
    ctg_rating: float = 1.0
    lodf_candidates: int = 20
    # "ptdf": Eq. 6 as written -- one system-wide balance row per hour and
    # PTDF flow rows for the monitored lines (no angle variables);
    # "btheta": nodal balance rows with bus angles and a row per line.
    network: str = "ptdf"
    # base-case monitored lines for "ptdf" (None: the N-1 lines, or L/100
    # when there are no N-1 rows)
    base_lines: int | None = None


PRESETS = {
    # 14 buses, 20 lines, 5 units, T=24, no contingency rows: ~1.5k variables
    "scuc14": SCUCConfig(buses=14, lines=20, units=5, T=24, contingencies=0, seed=1,
                         network="btheta"),
    # 2,000-bus random geometric grid, 300 units, 50 N-1 lines
    "scuc2k": SCUCConfig(buses=2000, lines=2800, units=300, T=36, contingencies=50, seed=2),
    # 6,500 buses, 1,000 units, 100 N-1 lines (successive-fixing loop)
    "scuc6k": SCUCConfig(buses=6500, lines=9000, units=1000, T=36, contingencies=100, seed=3),
    # 13,000 buses, 4,000 units, 200 N-1 lines (the large relaxation)
    "scuc13k": SCUCConfig(buses=13000, lines=18000, units=4000, T=36, contingencies=200, seed=20000),
}


def batch_configs(count: int = 64, first_seed: int = 1000) -> list:
    """Uneven batch: buses log-uniform in [200, 3000], units = 0.15*buses,
    lines = 1.4*buses (mean degree 2.8), T in {24, 36}, no N-1 rows."""
    out = []
    for i in range(count):
        seed = first_seed + i
        r = np.random.default_rng(seed + 7919)
        b = int(round(np.exp(r.uniform(np.log(200), np.log(3000)))))
        out.append(SCUCConfig(buses=b, lines=int(round(1.4 * b)), units=max(1, int(round(0.15 * b))),
                              T=int(r.choice([24, 36])), contingencies=0, seed=seed))
    return out


# ----------------------------------------------------------------------------
# grid
# ----------------------------------------------------------------------------

def _morton(q: np.ndarray) -> np.ndarray:
    def spread(v):
        v = v.astype(np.uint64)
        v = (v | (v << np.uint64(16))) & np.uint64(0x0000FFFF0000FFFF)
        v = (v | (v << np.uint64(8))) & np.uint64(0x00FF00FF00FF00FF)
        v = (v | (v << np.uint64(4))) & np.uint64(0x0F0F0F0F0F0F0F0F)
        v = (v | (v << np.uint64(2))) & np.uint64(0x3333333333333333)
        v = (v | (v << np.uint64(1))) & np.uint64(0x5555555555555555)
        return v
    return spread(q[:, 0]) | (spread(q[:, 1]) << np.uint64(1))


def make_grid(rng: np.random.Generator, B: int, L: int):
    """Random geometric graph: Euclidean MST (connected) plus the shortest
    remaining k-nearest-neighbour edges up to L lines.  Buses are numbered in
    Morton order so that electrically close buses get close indices."""
    if L < B - 1:
        raise ValueError("need at least B-1 lines for a connected grid")
    pts = rng.random((B, 2))
    q = np.clip((pts * 65535).astype(np.int64), 0, 65535)
    pts = pts[np.argsort(_morton(q), kind="stable")]
    tree = cKDTree(pts)
    k = min(B, 16)
    d, idx = tree.query(pts, k=k)
    i = np.repeat(np.arange(B), k - 1)
    j = idx[:, 1:].ravel()
    w = d[:, 1:].ravel()
    a, b = np.minimum(i, j), np.maximum(i, j)
    key = a.astype(np.int64) * B + b
    key, first = np.unique(key, return_index=True)
    a, b, w = a[first], b[first], w[first]
    Gk = sp.coo_matrix((w + 1e-12, (a, b)), shape=(B, B)).tocsr()
    mst = minimum_spanning_tree(Gk).tocoo()
    ea, eb = list(np.minimum(mst.row, mst.col)), list(np.maximum(mst.row, mst.col))
    # join components (rare for k=16) by their nearest pairs
    ncomp, lab = connected_components(
        sp.coo_matrix((np.ones(len(ea)), (ea, eb)), shape=(B, B)), directed=False)
    while ncomp > 1:
        inside = np.flatnonzero(lab == lab[0])
        outside = np.flatnonzero(lab != lab[0])
        t_out = cKDTree(pts[outside])
        dd, jj = t_out.query(pts[inside], k=1)
        s = int(np.argmin(dd))
        u, v = int(inside[s]), int(outside[jj[s]])
        ea.append(min(u, v)); eb.append(max(u, v))
        ncomp, lab = connected_components(
            sp.coo_matrix((np.ones(len(ea)), (ea, eb)), shape=(B, B)), directed=False)
    used = set(zip(ea, eb))
    order = np.argsort(w, kind="stable")
    for o in order:
        if len(ea) >= L:
            break
        e = (int(a[o]), int(b[o]))
        if e not in used:
            used.add(e); ea.append(e[0]); eb.append(e[1])
    if len(ea) < L:
        raise ValueError("not enough candidate edges for the requested line count")
    fr = np.asarray(ea[:L], dtype=np.int64)
    to = np.asarray(eb[:L], dtype=np.int64)
    x = rng.uniform(0.01, 0.2, size=L)
    return pts, fr, to, x


class _DCGrid:
    """DC network of a grid: reduced bus susceptance LU (reference bus 0)."""

    def __init__(self, B, fr, to, x):
        self.B, self.fr, self.to = B, fr, to
        self.y = 1.0 / x
        L = len(fr)
        rows = np.concatenate([fr, to, fr, to])
        cols = np.concatenate([fr, to, to, fr])
        vals = np.concatenate([self.y, self.y, -self.y, -self.y])
        Bbus = sp.coo_matrix((vals, (rows, cols)), shape=(B, B)).tocsc()
        self.lu = spla.splu(Bbus[1:, 1:].tocsc())
        self.L = L

    def angles(self, inj_pu):
        """Bus angles (reference bus 0) for injections inj_pu [B, k]."""
        th = np.zeros_like(inj_pu)
        th[1:] = self.lu.solve(np.ascontiguousarray(inj_pu[1:]))
        return th

    def ptdf_rows(self, lines):
        """PTDF rows (MW on line per MW injected at bus, withdrawn at bus 0)."""
        lines = np.asarray(lines)
        rhs = np.zeros((self.B, len(lines)))
        rhs[self.fr[lines], np.arange(len(lines))] += 1.0
        rhs[self.to[lines], np.arange(len(lines))] -= 1.0
        z = self.angles(rhs)               # B^-1 (e_i - e_j)  (symmetric B)
        return (z * self.y[lines][None, :]).T  # [len(lines), B]


# ----------------------------------------------------------------------------
# instance
# ----------------------------------------------------------------------------

@dataclass
class SCUCInstance:
    cfg: SCUCConfig
    m: int
    n: int
    row_ptr: np.ndarray     # int64 [m+1]
    col: np.ndarray         # int32 [nnz]
    val: np.ndarray         # float64 [nnz]
    c: np.ndarray           # float64 [n]
    xl: np.ndarray          # float64 [n]  (-inf allowed)
    xu: np.ndarray          # float64 [n]  (+inf allowed)
    sense: np.ndarray       # uint8 [m]  b'G', b'L', b'E', b'R'
    rhs: np.ndarray         # float64 [m]
    rng_: np.ndarray        # float64 [m]  range of 'R' rows, 0 elsewhere
    G: int
    T: int
    u_idx: np.ndarray       # int32 [G*T] column of u_{g,t} (g-major)
    v_idx: np.ndarray
    w_idx: np.ndarray
    u_init: np.ndarray      # int8 [G]
    is_int: np.ndarray      # uint8 [n]   1 for the relaxed binaries u, v, w
    power_scale: float
    objective_scale: float
    params: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def row_bounds(self):
        lo = np.full(self.m, -INF)
        hi = np.full(self.m, INF)
        s = self.sense
        g = s == ord("G"); l = s == ord("L"); e = s == ord("E"); r = s == ord("R")
        lo[g] = self.rhs[g]
        hi[l] = self.rhs[l]
        lo[e] = self.rhs[e]; hi[e] = self.rhs[e]
        lo[r] = self.rhs[r]; hi[r] = self.rhs[r] + self.rng_[r]
        return lo, hi

    def csr(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.m, self.n))

    def summary(self) -> dict:
        lens = np.diff(self.row_ptr)
        return {"buses": self.cfg.buses, "lines": self.cfg.lines, "units": self.cfg.units,
                "T": self.cfg.T, "contingencies": self.cfg.contingencies, "seed": self.cfg.seed,
                "m": self.m, "n": self.n, "nnz": self.nnz,
                "max_row_nnz": int(lens.max()) if self.m else 0}


def make_scuc(cfg: SCUCConfig) -> SCUCInstance:
    rng = np.random.default_rng(cfg.seed)
    B, Lr, G, T, K = cfg.buses, cfg.lines, cfg.units, cfg.T, cfg.contingencies

    pts, fr, to, xr = make_grid(rng, B, Lr)
    L = len(fr)
    dc = _DCGrid(B, fr, to, xr)

    # ---- units (MW, $/MWh) ----
    pmax = np.clip(rng.lognormal(np.log(89.4), 0.75, size=G), 20.0, 400.0)
    pmin = 0.3 * pmax
    ru = 0.5 * pmax
    rd = ru.copy()
    su = ru.copy()
    sd = ru.copy()
    ut = rng.integers(1, 5, size=G)
    dt = rng.integers(1, 5, size=G)
    segc = np.sort(rng.uniform(10.0, 80.0, size=(G, 3)), axis=1)
    segw = np.repeat(((pmax - pmin) / 3.0)[:, None], 3, axis=1)
    bus_g = rng.integers(0, B, size=G)

    # ---- load ----
    hours = np.arange(1, T + 1)
    Dt = (cfg.load_frac * pmax.sum() * (1.0 + cfg.load_amp * np.sin(2 * np.pi * (hours - 8) / 24.0))
          * (1.0 + rng.uniform(-cfg.load_noise, cfg.load_noise, size=T)))
    wb = rng.uniform(0.5, 1.5, size=B)
    Dbt = Dt[None, :] * (wb / wb.sum())[:, None]           # [B, T]

    # ---- line limits from a proportional-dispatch DC flow ----
    share = pmax / pmax.sum()
    gen_bt = np.zeros((B, T))
    np.add.at(gen_bt, bus_g, share[:, None] * Dt[None, :])
    th = dc.angles((gen_bt - Dbt) / 100.0)
    flow = 100.0 * dc.y[:, None] * (th[fr] - th[to])         # [L, T] MW
    F = 1.5 * np.abs(flow).max(axis=1)
    F = np.maximum(F, 0.05 * F.mean())

    # ---- initial state: all units on at the proportional dispatch of hour 1,
    # capped at 0.9 x the shut-down capacity so that stopping in hour 1 is
    # always possible (Eq. 4 ramp-down row at t = 1) ----
    u_init = np.ones(G, dtype=np.int8)
    p_init = np.minimum(share * Dt[0], 0.9 * sd)

    # ---- instance-aware scaling (Sec. 3.A) ----
    if cfg.eta_scaling:
        etaP = float(pmax.max() if cfg.eta_reading == "pmax" else pmin.max())
        etaC = float(segc.max())
    else:
        etaP, etaC = 1.0, 1.0
    cs = etaP / etaC
    pmax_s, pmin_s = pmax / etaP, pmin / etaP
    ru_s, rd_s, su_s, sd_s = ru / etaP, rd / etaP, su / etaP, sd / etaP
    segw_s = segw / etaP
    segc_s = segc * cs
    cl_s = pmin_s * segc_s[:, 0]                 # cost of running at P^L
    pen_s = cfg.penalty * cs
    Dbt_s, Dt_s = Dbt / etaP, Dt / etaP
    F_s = F / etaP
    p_init_s = p_init / etaP
    bl = 100.0 * dc.y / etaP                     # (scaled MW)/rad

    # ---- variable layout ----
    nU = NVU * G * T
    ptdf_net = cfg.network == "ptdf"
    if cfg.network not in ("ptdf", "btheta"):
        raise ValueError("network must be 'ptdf' or 'btheta'")
    n = nU + (1 if ptdf_net else 2) * B * T

    def uv(g, t, k):
        return (t * G + g) * NVU + k

    def bv(b, t, k):  # "btheta": (theta, d) per bus-hour
        return nU + (t * B + b) * 2 + k

    def dcol(b, t):   # unserved-load column of bus b, hour t
        return nU + t * B + b if ptdf_net else bv(b, t, 1)

    gg, tt = np.meshgrid(np.arange(G), np.arange(T), indexing="ij")
    gg, tt = gg.ravel(), tt.ravel()          # g-major, t-minor
    GT = G * T

    # ---- bounds and costs ----
    xl = np.zeros(n)
    xu = np.zeros(n)
    c = np.zeros(n)
    base = (tt * G + gg) * NVU
    xu[base + U] = 1.0; xu[base + V] = 1.0; xu[base + W] = 1.0
    xu[base + P] = (pmax_s - pmin_s)[gg]
    for h in range(3):
        xu[base + S1 + h] = segw_s[gg, h]
        c[base + S1 + h] = segc_s[gg, h]
    c[base + U] = cl_s[gg]
    bb, bt = np.meshgrid(np.arange(B), np.arange(T), indexing="ij")
    bb, bt = bb.ravel(), bt.ravel()
    d_col = dcol(bb, bt)
    if not ptdf_net:
        th_col = bv(bb, bt, 0)
        xl[th_col] = -INF; xu[th_col] = INF
        ref = bb == 0
        xl[th_col[ref]] = 0.0; xu[th_col[ref]] = 0.0
    xu[d_col] = Dbt_s[bb, bt]
    c[d_col] = pen_s

    rows, cols, vals = [], [], []

    def add(r, cidx, v):
        r = np.asarray(r, dtype=np.int64)
        cidx = np.asarray(cidx, dtype=np.int64)
        v = np.broadcast_to(np.asarray(v, dtype=np.float64), r.shape)
        rows.append(r.ravel()); cols.append(cidx.ravel()); vals.append(np.array(v).ravel())

    mU = NRU * GT
    if ptdf_net:
        Kb = cfg.base_lines if cfg.base_lines is not None else (K if K > 0 else max(5, L // 100))
        Kb = min(Kb, L)
        m_bus, m_line = T, Kb * T
    else:
        Kb = 0
        m_bus, m_line = B * T, L * T
    m_res = T
    m_ctg = K * T
    m = mU + m_bus + m_line + m_res + m_ctg
    sense = np.zeros(m, dtype=np.uint8)
    rhs = np.zeros(m)
    rngv = np.zeros(m)
    urow = (tt * G + gg) * NRU
    t0 = tt == 0
    t1 = ~t0

    # Eq. 1: u_t - u_{t-1} - v_t + w_t = 0  (t=0: u_init on the right)
    r = urow + R_LOGIC
    add(r, base + U, 1.0); add(r, base + V, -1.0); add(r, base + W, 1.0)
    add(r[t1], uv(gg[t1], tt[t1] - 1, U), -1.0)
    sense[r] = ord("E"); rhs[r[t0]] = u_init[gg[t0]]
    # Eq. 1: v + w <= 1
    r = urow + R_VW
    add(r, base + V, 1.0); add(r, base + W, 1.0)
    sense[r] = ord("L"); rhs[r] = 1.0
    # Eq. 2: sum_{tau=max(1,t-UT+1)}^{t} v_tau - u_t <= 0 ; sum w_tau + u_t <= 1
    r_up = urow + R_MINUP
    r_dn = urow + R_MINDN
    add(r_up, base + U, -1.0)
    add(r_dn, base + U, 1.0)
    for d in range(4):
        ok = (tt - d >= 0) & (d < ut[gg])
        add(r_up[ok], uv(gg[ok], tt[ok] - d, V), 1.0)
        ok = (tt - d >= 0) & (d < dt[gg])
        add(r_dn[ok], uv(gg[ok], tt[ok] - d, W), 1.0)
    sense[r_up] = ord("L"); rhs[r_up] = 0.0
    sense[r_dn] = ord("L"); rhs[r_dn] = 1.0
    # Eq. 3: p' - (P^U - P^L) u <= 0
    r = urow + R_PROD
    add(r, base + P, 1.0); add(r, base + U, -(pmax_s - pmin_s)[gg])
    sense[r] = ord("L")
    # Eq. 4 ramp up: p'_t + P^L u_t - SU v_t - p'_{t-1} - (P^L+RU) u_{t-1} <= 0
    r = urow + R_RUP
    add(r, base + P, 1.0); add(r, base + U, pmin_s[gg]); add(r, base + V, -su_s[gg])
    add(r[t1], uv(gg[t1], tt[t1] - 1, P), -1.0)
    add(r[t1], uv(gg[t1], tt[t1] - 1, U), -(pmin_s + ru_s)[gg[t1]])
    sense[r] = ord("L")
    rhs[r[t0]] = ru_s[gg[t0]] * u_init[gg[t0]] + p_init_s[gg[t0]]
    # Eq. 4 ramp down: p'_{t-1} + P^L u_{t-1} - p'_t - (P^L+RD) u_t - SD w_t <= 0
    r = urow + R_RDN
    add(r, base + P, -1.0); add(r, base + U, -(pmin_s + rd_s)[gg]); add(r, base + W, -sd_s[gg])
    add(r[t1], uv(gg[t1], tt[t1] - 1, P), 1.0)
    add(r[t1], uv(gg[t1], tt[t1] - 1, U), pmin_s[gg[t1]])
    sense[r] = ord("L")
    rhs[r[t0]] = -p_init_s[gg[t0]]
    # Eq. 5: p_h - (P^U_h - P^U_{h-1}) u <= 0 ; sum_h p_h - p' = 0
    for h in range(3):
        r = urow + R_SEG1 + h
        add(r, base + S1 + h, 1.0); add(r, base + U, -segw_s[gg, h])
        sense[r] = ord("L")
    r = urow + R_SEGSUM
    add(r, base + S1, 1.0); add(r, base + S2, 1.0); add(r, base + S3, 1.0); add(r, base + P, -1.0)
    sense[r] = ord("E")

    def add_ptdf_row(r, db, t):
        """Row sum_b db_b (sum_{g in G_b}(p'_gt + P^L_g u_gt) + d_bt); returns
        the load term sum_b db_b D_bt that goes to the row bounds."""
        nzb = np.flatnonzero(db)
        gsel = np.flatnonzero(db[bus_g] != 0.0)
        add(np.full(len(gsel), r), uv(gsel, t, P), db[bus_g[gsel]])
        add(np.full(len(gsel), r), uv(gsel, t, U), db[bus_g[gsel]] * pmin_s[gsel])
        add(np.full(len(nzb), r), dcol(nzb, t), db[nzb])
        return float((db[nzb] * Dbt_s[nzb, t]).sum())

    load = np.abs(flow).max(axis=1)
    rb0 = mU
    rl0 = rb0 + m_bus
    if ptdf_net:
        # Eq. 6, first line: sum_g p_gt + sum_b d_bt = sum_b D_bt
        ones = np.ones(B)
        for t in range(T):
            tot = add_ptdf_row(rb0 + t, ones, t)
            sense[rb0 + t] = ord("E"); rhs[rb0 + t] = tot
        # Eq. 6, second line for c = 0 on the monitored lines (PTDF rows)
        mon_b = np.argsort(-load, kind="stable")[:Kb]
        ptdf_b = dc.ptdf_rows(mon_b) if Kb > 0 else np.zeros((0, B))
        ptdf_b[np.abs(ptdf_b) < cfg.ptdf_trunc] = 0.0
        for kk in range(Kb):
            for t in range(T):
                r = rl0 + t * Kb + kk
                const = add_ptdf_row(r, ptdf_b[kk], t)
                sense[r] = ord("R"); rhs[r] = -F_s[mon_b[kk]] + const; rngv[r] = 2.0 * F_s[mon_b[kk]]
    else:
        # nodal balance (b,t): sum_{g in G_b}(p' + P^L u) + d - sum_l b_l (th_b - th_o) = D_bt
        rowb = rb0 + bt * B + bb
        add(rowb, d_col, 1.0)
        rg = rb0 + tt * B + bus_g[gg]
        add(rg, base + P, 1.0); add(rg, base + U, pmin_s[gg])
        for t in range(T):
            rf = rb0 + t * B + fr
            rt = rb0 + t * B + to
            add(rf, bv(fr, t, 0), -bl); add(rf, bv(to, t, 0), bl)
            add(rt, bv(to, t, 0), -bl); add(rt, bv(fr, t, 0), bl)
        sense[rowb] = ord("E"); rhs[rowb] = Dbt_s[bb, bt]
        # line flow (l,t): -F <= b_l (th_from - th_to) <= F
        ll, lt = np.meshgrid(np.arange(L), np.arange(T), indexing="ij")
        ll, lt = ll.ravel(), lt.ravel()
        r = rl0 + lt * L + ll
        add(r, bv(fr[ll], lt, 0), bl[ll]); add(r, bv(to[ll], lt, 0), -bl[ll])
        sense[r] = ord("R"); rhs[r] = -F_s[ll]; rngv[r] = 2.0 * F_s[ll]

    # spinning reserve (t): sum_g ((P^U - P^L) u - p') >= reserve_frac * D_t
    rr0 = rl0 + m_line
    r = rr0 + tt
    add(r, base + U, (pmax_s - pmin_s)[gg]); add(r, base + P, -1.0)
    sense[rr0:rr0 + T] = ord("G"); rhs[rr0:rr0 + T] = cfg.reserve_frac * Dt_s

    # N-1 rows (k,t): -F^c <= sum_b delta_b (gen_b + d_b - D_b) <= F^c
    rc0 = rr0 + m_res
    ctg_info = None
    if K > 0:
        mon = np.argsort(-load, kind="stable")[:K]
        ptdf_m = dc.ptdf_rows(mon)                          # [K, B]
        num = ptdf_m[:, fr] - ptdf_m[:, to]                 # transfer PTDF of each line c
        for kk in range(K):
            num[kk, mon[kk]] = 0.0
        ncand = min(cfg.lodf_candidates, L - 1)
        cand = np.argsort(-np.abs(num), axis=1, kind="stable")[:, :ncand]
        ucand = np.unique(cand)
        self_tr = np.zeros(L)
        for s0 in range(0, len(ucand), 512):
            cc = ucand[s0:s0 + 512]
            pr = dc.ptdf_rows(cc)
            self_tr[cc] = pr[np.arange(len(cc)), fr[cc]] - pr[np.arange(len(cc)), to[cc]]
        outage = np.zeros(K, dtype=np.int64)
        lodf = np.zeros(K)
        for kk in range(K):
            cc = cand[kk]
            den = 1.0 - self_tr[cc]
            ok = np.abs(den) > 1e-6
            val_ = np.where(ok, num[kk, cc] / np.where(ok, den, 1.0), 0.0)
            j = int(np.argmax(np.abs(val_)))
            outage[kk] = cc[j]
            lodf[kk] = val_[j]
        ptdf_o = dc.ptdf_rows(outage)
        delta = ptdf_m + lodf[:, None] * ptdf_o              # [K, B]
        delta[np.abs(delta) < cfg.ptdf_trunc] = 0.0
        Fc = cfg.ctg_rating * F_s[mon]
        ctg_info = {"monitored": mon, "outage": outage, "lodf": lodf}
        for kk in range(K):
            for t in range(T):
                r = rc0 + t * K + kk
                const = add_ptdf_row(r, delta[kk], t)
                sense[r] = ord("R"); rhs[r] = -Fc[kk] + const; rngv[r] = 2.0 * Fc[kk]

    R_ = np.concatenate(rows)
    C_ = np.concatenate(cols)
    X_ = np.concatenate(vals)
    A = sp.coo_matrix((X_, (R_, C_)), shape=(m, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    A.eliminate_zeros()

    u_idx = uv(gg, tt, U).astype(np.int32)      # indexed g*T + t (g-major)
    is_int = np.zeros(n, dtype=np.uint8)
    is_int[base + U] = 1; is_int[base + V] = 1; is_int[base + W] = 1

    params = dict(pmax=pmax, pmin=pmin, ru=ru, rd=rd, su=su, sd=sd, ut=ut, dt=dt, segc=segc,
                  segw=segw, bus_g=bus_g, Dbt=Dbt, Dt=Dt, F=F, fr=fr, to=to, x=xr, pts=pts,
                  p_init=p_init, etaP=etaP, etaC=etaC, ctg=ctg_info,
                  row_blocks=dict(unit=(0, mU), bus=(rb0, rb0 + m_bus), line=(rl0, rl0 + m_line),
                                  reserve=(rr0, rr0 + m_res), ctg=(rc0, rc0 + m_ctg)),
                  col_blocks=dict(unit=(0, nU), bus=(nU, n)), network=cfg.network,
                  base_lines=Kb)
    return SCUCInstance(cfg=cfg, m=m, n=n, row_ptr=A.indptr.astype(np.int64),
                        col=A.indices.astype(np.int32), val=A.data.astype(np.float64),
                        c=c, xl=xl, xu=xu, sense=sense, rhs=rhs, rng_=rngv, G=G, T=T,
                        u_idx=u_idx, v_idx=(u_idx + 1).astype(np.int32),
                        w_idx=(u_idx + 2).astype(np.int32), u_init=u_init, is_int=is_int,
                        power_scale=etaP, objective_scale=etaC, params=params)


def make_preset(name: str, **overrides) -> SCUCInstance:
    cfg = dataclasses.replace(PRESETS[name], **overrides)
    return make_scuc(cfg)


def split_network_rows(inst: SCUCInstance):
    """The transmission-filtering split of an instance (Fig. 1 of the paper):
    ``base`` holds every row except the network security rows (base-case
    line rows and N-1 rows), ``pool`` holds those rows over the same columns.
    Both are LP dicts (row box form); ``pool_rows`` are the pool rows'
    indices in the full instance.  Pure data selection."""
    lo, hi = inst.row_bounds()
    blocks = inst.params["row_blocks"]
    net = np.zeros(inst.m, dtype=bool)
    for name in ("line", "ctg"):
        a, b = blocks[name]
        net[a:b] = True
    A = inst.csr()

    def part(sel):
        S = A[sel].tocsr()
        S.sort_indices()
        return dict(m=S.shape[0], n=inst.n, row_ptr=S.indptr.astype(np.int64), col=S.indices.astype(np.int32),
                    val=S.data.astype(np.float64), c=inst.c.copy(), xl=inst.xl.copy(), xu=inst.xu.copy(),
                    lo=lo[sel].copy(), hi=hi[sel].copy())

    base_rows = np.flatnonzero(~net)
    pool_rows = np.flatnonzero(net)
    return part(base_rows), part(pool_rows), pool_rows
