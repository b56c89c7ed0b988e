"""FP32 products on 16-bit index offsets (scuc_lp_set_index16,
scuc_lp_layout).

The FP32 iteration products read each matrix entry as its FP32 value plus a
16-bit offset from one of at most two cluster bases where the layout
allows: per 512-entry chunk of a long row, per column of the sliced copy of
A^T.  The sums are the same as with 32-bit indices, so the iterates of a
mixed-precision solve must be bit-identical with the switch on and off.
The LPs below exercise every branch: chunks with one and with two clusters,
chunks that need three and keep 32-bit indices, columns whose rows fall
into two clusters, and a copy of A^T that stays 32-bit because a column has
three clusters."""
import numpy as np
import pytest
import scipy.sparse as sp

pytestmark = pytest.mark.gpu


def _box_lp(A, seed):
    rng = np.random.default_rng(seed)
    A = sp.csr_matrix(A)
    A.sum_duplicates()
    A.sort_indices()
    m, n = A.shape
    return dict(m=m, n=n, row_ptr=A.indptr.astype(np.int64), col=A.indices.astype(np.int32),
                val=A.data.astype(np.float64), c=rng.normal(size=n), xl=np.full(n, -1.0), xu=np.full(n, 1.0),
                lo=np.full(m, -1.0) - rng.random(m), hi=np.full(m, 1.0) + rng.random(m))


def _clustered(seed, clusters):
    """m x n with every column's rows in `clusters` blocks 70,000 apart, five
    dense rows (A's chunks: at most two clusters each, n = 70,000) and three
    columns with 200 rows in each of three blocks at rows 0, 70,000 and m -
    2,000 (A^T's chunks: the first 512 entries need three clusters and keep
    32-bit rows, the last ones lie in one block).  A row left empty gets an
    entry in a column whose block of the same cluster lies within 10,020
    rows of it."""
    rng = np.random.default_rng(seed)
    m, n = 70_000 * clusters, 70_000
    rows, cols = [], []
    for k in range(clusters):
        start = (np.arange(n) * 2) % 60_000 + 70_000 * k
        r = start[:, None] + rng.integers(0, 5_000, size=(n, 12))
        rows.append(r.ravel())
        cols.append(np.repeat(np.arange(n), 12))
    for i in range(5):                                  # dense rows
        cols.append(rng.choice(n, size=600, replace=False))
        rows.append(np.full(600, 1_000 * i + 7))
    long_cols = (11, 222, 3_333)
    for j in long_cols:                                 # long columns: three blocks of 200 rows
        rows.append(np.concatenate([b + rng.choice(2_000, size=200, replace=False)
                                    for b in (0, 70_000, m - 2_000)]))
        cols.append(np.full(600, j))
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    empty = np.setdiff1d(np.arange(m), r)
    off = empty % 70_000
    fill = np.clip((off - 2_500) // 2, 0, 29_999)       # block start 2j within 2,501 rows
    fill = np.where(off > 62_500, 29_990 + empty % 10, fill)   # or a block start in 59,980..59,998
    fill[np.isin(fill, long_cols)] += 1
    r = np.concatenate([r, empty])
    c = np.concatenate([c, fill])
    v = rng.uniform(-1.0, 1.0, size=r.size)
    return _box_lp(sp.coo_matrix((v, (r, c)), shape=(m, n)), seed)


def _solve(P, src, index16):
    lp = P.LP(src)
    if not index16:
        lp.set_index16(0)
    r = lp.solve(want=("x", "y"), tol=0.0, max_iter=192, precision="mixed", polish_stall=10 ** 6,
                 polish_factor=0.0, polish_floor=0.0)
    lay = lp.layout()
    lp.close()
    return r, lay


def _chunked_entries(src):
    """Entries of A's rows and of A^T's rows (A's columns) above 512."""
    rl = np.diff(src["row_ptr"])
    cl = np.bincount(src["col"], minlength=src["n"])
    return int(rl[rl > 512].sum()), int(cl[cl > 512].sum())


def _same_iterates(P, src):
    a, lay = _solve(P, src, True)
    b, lay32 = _solve(P, src, False)
    assert a["info"]["iters"] == b["info"]["iters"] == 192
    assert a["info"]["iters_fp32"] == 192
    np.testing.assert_array_equal(a["x"], b["x"])
    np.testing.assert_array_equal(a["y"], b["y"])
    assert lay32["a_chunk16"] == 0 and lay32["t_chunk16"] == 0 and lay32["t_sell_compressed"] == 0
    return lay


def test_two_clusters_and_wide_chunks():
    import paper_2510_10891_b300 as P
    src = _clustered(1, 2)
    lay = _same_iterates(P, src)
    ea, et = _chunked_entries(src)
    assert lay["t_sell_compressed"] == 1
    assert lay["a_chunk16"] == ea and lay["a_chunk32"] == 0          # two bases cover every chunk of A
    assert lay["t_chunk32"] > 0 and lay["t_chunk16"] > 0             # A^T: some chunks need three
    assert lay["t_chunk16"] + lay["t_chunk32"] == et


def test_three_clusters_keep_32bit_rows():
    import paper_2510_10891_b300 as P
    src = _clustered(2, 3)
    lay = _same_iterates(P, src)
    assert lay["t_sell_compressed"] == 0
    assert lay["a_chunk16"] == _chunked_entries(src)[0]


def test_scuc2k_layout_and_iterates():
    import paper_2510_10891_b300 as P
    from scuc_gen import make_preset
    inst = make_preset("scuc2k")
    src = dict(m=inst.m, n=inst.n, row_ptr=inst.row_ptr, col=inst.col, val=inst.val, c=inst.c, xl=inst.xl,
               xu=inst.xu, sense=inst.sense, rhs=inst.rhs, rng_=inst.rng_)
    lay = _same_iterates(P, src)
    assert lay["t_sell_compressed"] == 1 and lay["a_chunk16"] > 0 and lay["a_chunk32"] == 0


def test_index16_is_set_before_the_first_solve():
    import paper_2510_10891_b300 as P
    from paper_2510_10891_b300 import _lib as L
    from scuc_gen import make_preset
    lp = P.LP(make_preset("scuc14"))
    assert L.lib().scuc_lp_set_index16(lp.h, 2) == L.SCUC_E_INVALID
    lp.solve(tol=1e-4, precision="mixed")
    assert L.lib().scuc_lp_set_index16(lp.h, 0) == L.SCUC_E_INVALID
    lp.close()
