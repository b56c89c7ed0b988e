"""Seeded random LPs and vectors (inputs for parity tests and warm starts)."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def random_lp(m, n, density=0.2, seed=0, senses="GLER", free_frac=0.1, long_rows=0,
              long_cols=0, feasible=True):
    """A random bounded-feasible LP in the library's input form.

    Rows have random senses; a random interior point x0 makes every row
    satisfiable, and finite boxes on most columns keep it bounded.
    ``long_rows``/``long_cols`` add dense rows/columns to exercise the long
    row path of the sparse kernels.
    """
    rng = np.random.default_rng(seed)
    A = sp.random(m, n, density=density, random_state=rng, format="lil",
                  data_rvs=lambda k: rng.uniform(-2.0, 2.0, size=k))
    for r in rng.choice(m, size=min(long_rows, m), replace=False):
        A[r, :] = rng.uniform(-1.0, 1.0, size=n)
    for cidx in rng.choice(n, size=min(long_cols, n), replace=False):
        A[:, cidx] = rng.uniform(-1.0, 1.0, size=(m, 1))
    A = A.tocsr()
    for r in range(m):  # no empty rows
        if A.indptr[r] == A.indptr[r + 1]:
            A[r, rng.integers(n)] = 1.0
    A = A.tocsr()
    A.sort_indices()
    xl = rng.uniform(-5.0, 0.0, size=n)
    xu = xl + rng.uniform(0.5, 6.0, size=n)
    free = rng.random(n) < free_frac
    xl[free] = -np.inf
    xu[free] = np.inf
    box = np.where(free, 0.0, xl + rng.random(n) * (np.where(free, 1.0, xu - xl)))
    x0 = np.where(free, rng.uniform(-1, 1, size=n), box)
    ax = A @ x0
    sense = rng.choice([ord(s) for s in senses], size=m).astype(np.uint8)
    rhs = np.zeros(m)
    rngv = np.zeros(m)
    slack = rng.uniform(0.1, 2.0, size=m)
    g = sense == ord("G"); l = sense == ord("L"); e = sense == ord("E"); r_ = sense == ord("R")
    rhs[g] = ax[g] - slack[g]
    rhs[l] = ax[l] + slack[l]
    rhs[e] = ax[e]
    rhs[r_] = ax[r_] - slack[r_]
    rngv[r_] = 2.0 * slack[r_]
    # cost: make free columns dual-feasible by giving them A^T y0 costs
    y0 = rng.normal(size=m)
    y0[g] = np.abs(y0[g]); y0[l] = -np.abs(y0[l])
    c = rng.normal(size=n)
    c[free] = (A.T @ y0)[free]
    return dict(m=m, n=n, row_ptr=A.indptr.astype(np.int64), col=A.indices.astype(np.int32),
                val=A.data.astype(np.float64), c=c, xl=xl, xu=xu, sense=sense, rhs=rhs,
                rng_=rngv)


def seeded_vector(n, seed, lo=-1.0, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, size=n)
