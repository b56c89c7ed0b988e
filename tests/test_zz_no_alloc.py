"""scuc_lp_kkt_noalloc: KKT residuals of a given point with no device
allocation (for callers whose GPU memory is already handed out to another
allocator or pool, or that cannot afford cudaMalloc/cudaFree in their loop).

The solve reports r_p, r_d, gap and both objectives at the point it returns;
the no-allocation entry point, given that same point, must report the same
values (same tolerances as the other parity tests), and two calls in a row
must agree exactly: the shared scratch keeps the previous call's contents,
and none of them may leak into the next result.

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_kkt_noalloc_matches_solve():
    import torch

    import paper_2510_10891_b300 as P
    from paper_2510_10891_b300 import _lib as L
    from scuc_gen import make_preset

    assert torch.cuda.is_available()
    inst = make_preset("scuc2k")
    stream = torch.cuda.current_stream()
    lp = P.LP(inst, stream=stream.cuda_stream)
    x = torch.empty(inst.n, dtype=torch.float64, device="cuda")
    y = torch.empty(inst.m, dtype=torch.float64, device="cuda")
    z = torch.empty(inst.n, dtype=torch.float64, device="cuda")
    info = lp.solve_device(x_out=x, y_out=y, z_out=z, tol=1e-4)
    assert info["status_name"] == "optimal"
    ptr = lambda t: C.c_void_p(t.data_ptr())
    outs = []
    for _ in range(2):
        out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
        L.check(L.lib().scuc_lp_kkt_noalloc(lp.h, ptr(x), ptr(y), ptr(z), ptr(out)))
        stream.synchronize()
        outs.append(out.cpu().numpy())
    for o in outs:
        rp, rd, gap, pobj, dobj, kkt = o
        assert rp == pytest.approx(info["rp"], rel=1e-7, abs=1e-13)
        assert rd == pytest.approx(info["rd"], rel=1e-7, abs=1e-13)
        assert gap == pytest.approx(info["gap"], rel=1e-7, abs=1e-13)
        assert pobj == pytest.approx(info["pobj"], rel=1e-9)
        assert dobj == pytest.approx(info["dobj"], rel=1e-9)
        assert kkt == pytest.approx(info["kkt"], rel=1e-7)
    np.testing.assert_array_equal(outs[0], outs[1])
    # null arguments are refused before any launch
    assert L.lib().scuc_lp_kkt_noalloc(lp.h, None, ptr(y), ptr(z), ptr(out)) == L.SCUC_E_INVALID
