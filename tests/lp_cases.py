"""LP cases with a known feasibility verdict and the defining inequalities of
the certificates (Farkas ray, recession direction), shared by the oracle
and GPU tests of infeasibility detection."""
import numpy as np
import scipy.sparse as sp
from scipy.optimize import linprog

PRIMAL_INFEASIBLE, DUAL_INFEASIBLE = 5, 6


def dense_lp(A, lo, hi, c, xl, xu):
    S = sp.csr_matrix(np.atleast_2d(np.asarray(A, float)))
    return dict(m=S.shape[0], n=len(c), row_ptr=S.indptr, col=S.indices, val=S.data,
                c=np.asarray(c, float), xl=np.asarray(xl, float), xu=np.asarray(xu, float),
                lo=np.asarray(lo, float), hi=np.asarray(hi, float))


def highs_status(lp):
    """HiGHS verdict: 0 optimal, 2 infeasible, 3 unbounded."""
    A = sp.csr_matrix((lp["val"], lp["col"], lp["row_ptr"]), shape=(lp["m"], lp["n"]))
    fh, fl = np.isfinite(lp["hi"]), np.isfinite(lp["lo"])
    Aub = sp.vstack([A[fh], -A[fl]]).tocsr()
    bub = np.concatenate([lp["hi"][fh], -lp["lo"][fl]])
    bounds = np.c_[np.where(np.isfinite(lp["xl"]), lp["xl"], None),
                   np.where(np.isfinite(lp["xu"]), lp["xu"], None)]
    r = linprog(lp["c"], A_ub=Aub if Aub.shape[0] else None, b_ub=bub if Aub.shape[0] else None,
                bounds=bounds, method="highs")
    return r.status, r.fun


def farkas(lp, u):
    """Homogeneous dual objective of the ray u (z = -A^T u) over the terms
    whose bounds are finite, and the size of the terms that would need an
    infinite bound."""
    A = sp.csr_matrix((lp["val"], lp["col"], lp["row_ptr"]), shape=(lp["m"], lp["n"]))
    z = -(A.T @ u)
    F, V = 0.0, 0.0
    for v, l, h in list(zip(u, lp["lo"], lp["hi"])) + list(zip(z, lp["xl"], lp["xu"])):
        b = l if v > 0 else h
        if v == 0:
            continue
        if np.isfinite(b):
            F += b * v
        else:
            V += v * v
    return F, np.sqrt(V)


def recession(lp, d):
    """c^T d and the size of the violation of the recession cones of
    [lo, hi] (by A d) and [xl, xu] (by d)."""
    A = sp.csr_matrix((lp["val"], lp["col"], lp["row_ptr"]), shape=(lp["m"], lp["n"]))
    ad = A @ d
    viol = np.concatenate([np.where((d < 0) & np.isfinite(lp["xl"]), d, 0.0),
                           np.where((d > 0) & np.isfinite(lp["xu"]), d, 0.0),
                           np.where((ad < 0) & np.isfinite(lp["lo"]), ad, 0.0),
                           np.where((ad > 0) & np.isfinite(lp["hi"]), ad, 0.0)])
    return float(lp["c"] @ d), float(np.linalg.norm(viol))


def infeasible_box(seed):
    """Rows that no point of a finite box satisfies (primal infeasible; the
    box keeps the dual feasible)."""
    rng = np.random.default_rng(seed)
    m, n = int(rng.integers(2, 6)), int(rng.integers(2, 6))
    A = rng.uniform(-2, 2, (m, n))
    xl, xu = rng.uniform(-2, 0, n), rng.uniform(0.5, 2, n)
    hi = np.full(m, np.inf)
    # row 0 asks for more than its maximum over the box
    amax = np.sum(np.where(A[0] > 0, A[0] * xu, A[0] * xl))
    lo = np.full(m, -np.inf)
    lo[0] = amax + rng.uniform(0.1, 1.0)
    return dense_lp(A, lo, hi, rng.normal(size=n), xl, xu)


def unbounded(seed):
    """A feasible LP plus a column with negative cost and no upper bound whose
    entries only loosen rows with lower bounds (primal unbounded)."""
    rng = np.random.default_rng(seed)
    m, n = int(rng.integers(2, 6)), int(rng.integers(2, 5))
    A = rng.uniform(-2, 2, (m, n))
    xl, xu = rng.uniform(-2, 0, n), rng.uniform(0.5, 2, n)
    x0 = (xl + xu) / 2
    lo = A @ x0 - rng.uniform(0.1, 1, m)
    hi = np.full(m, np.inf)
    A = np.c_[A, rng.uniform(0.2, 1.0, m)]
    return dense_lp(A, lo, hi, np.r_[rng.normal(size=n), -1.0], np.r_[xl, 0.0], np.r_[xu, np.inf])
