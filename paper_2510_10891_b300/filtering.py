"""Transmission filtering (Fig. 1): solve the LP without the network security
rows, add the pool rows its solution violates, re-solve from the previous
point (y = 0 on the new rows), until no violated pool row is outside the LP
(the rows inside are held to the solve's own tolerance).  Host
orchestration of C-ABI calls only: the solves, the violation check and the
row appending run on the GPU."""
from __future__ import annotations

import numpy as np

from .lp import LP


def transmission_filter(base: LP, pool: LP, viol_tol: float = 1e-6, max_rounds: int = 20, **params) -> dict:
    """Returns the last LP (a new handle unless no row was added; the caller
    closes it), its solve, the pool rows in the order they were appended
    (``rows_added``), and per round the LP size, iterations, status, violated
    and added rows and the largest relative violation."""
    lp, x0, y0 = base, None, None
    added = np.zeros(pool.m, dtype=bool)
    rounds, order = [], []
    for _ in range(max_rounds):
        r = lp.solve(x0=x0, y0=y0, **params)
        viol, worst = pool.row_violations(r["x"], viol_tol)
        new = viol[~added[viol]]
        rounds.append(dict(m=lp.m, iters=r["info"]["iters"], status=r["info"]["status"], violated=len(viol),
                           added=len(new), max_violation=worst, solve_ms=r["info"]["solve_ms"]))
        if len(new) == 0:
            # every violated pool row is already in the LP, which holds it to
            # the solve's own tolerance: no round can add anything
            return dict(lp=lp, result=r, rounds=rounds, converged=True, violated_in_model=len(viol),
                        rows_added=np.asarray(order, dtype=np.int32))
        added[new] = True
        order.extend(new.tolist())
        nxt = lp.add_rows(pool, new)
        if lp is not base:
            lp.close()          # an intermediate LP of this loop
        lp = nxt
        x0, y0 = r["x"], np.concatenate([r["y"], np.zeros(len(new))])
    return dict(lp=lp, result=r, rounds=rounds, converged=False, violated_in_model=int(np.sum(added[viol])),
                rows_added=np.asarray(order, dtype=np.int32))
