"""scuc_lp_kkt_noalloc: KKT residuals of a given point with no device
allocation, for callers that cannot allocate GPU memory when they check a
point: their device memory is already handed out to another allocator or a
fixed pool, or they run a serving loop that must not pay for cudaMalloc /
cudaFree (cudaFree waits for the whole device).

The entry point must give the residuals that scuc_lp_solve reports for the
point it returns, and the oracle's FP64 evaluation of the same point, also
at points that are not solutions (random, with multipliers of the wrong sign
at infinite bounds).  All calls share one fixed device array that keeps the
previous call's contents: before the calls under test it is filled by a call
on a different LP with other block counts, and two calls in a row must agree
exactly.  Free device memory must not change across the calls.

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _kkt_noalloc(L, lp, x, y, z, stream, out=None):
    import torch
    ptr = lambda t: C.c_void_p(t.data_ptr())
    if out is None:
        out = torch.empty(6, dtype=torch.float64, device="cuda")
    out.fill_(float("nan"))
    L.check(L.lib().scuc_lp_kkt_noalloc(lp.h, ptr(x), ptr(y), ptr(z), ptr(out)))
    stream.synchronize()
    return out.cpu().numpy()


def _agree(o, ref, rel):
    rp, rd, gap, pobj, dobj, kkt = o
    assert rp == pytest.approx(ref["rp"], rel=rel, abs=1e-13)
    assert rd == pytest.approx(ref["rd"], rel=rel, abs=1e-13)
    assert gap == pytest.approx(ref["gap"], rel=rel, abs=1e-13)
    assert pobj == pytest.approx(ref["pobj"], rel=1e-9, abs=1e-9)
    assert dobj == pytest.approx(ref["dobj"], rel=1e-9, abs=1e-9)
    assert kkt == pytest.approx(ref["kkt"], rel=rel, abs=1e-13)


def test_kkt_noalloc_matches_solve_and_oracle():
    import torch

    import paper_2510_10891_b300 as P
    from paper_2510_10891_b300 import _lib as L
    from scuc_gen import make_preset

    assert torch.cuda.is_available()
    stream = torch.cuda.current_stream()
    inst = make_preset("scuc2k")
    lp = P.LP(inst, stream=stream.cuda_stream)
    x = torch.empty(inst.n, dtype=torch.float64, device="cuda")
    y = torch.empty(inst.m, dtype=torch.float64, device="cuda")
    z = torch.empty(inst.n, dtype=torch.float64, device="cuda")
    info = lp.solve_device(x_out=x, y_out=y, z_out=z, tol=1e-4)
    assert info["status_name"] == "optimal"

    # another LP, with other row-block counts, fills the shared array first
    other = make_preset("scuc14")
    lp_o = P.LP(other, stream=stream.cuda_stream)
    g = torch.Generator().manual_seed(3)
    xo = torch.randn(other.n, generator=g, dtype=torch.float64).cuda()
    yo = torch.randn(other.m, generator=g, dtype=torch.float64).cuda()
    zo = torch.randn(other.n, generator=g, dtype=torch.float64).cuda()
    o_other = _kkt_noalloc(L, lp_o, xo, yo, zo, stream)
    _agree(o_other, oracle.kkt(other, xo.cpu().numpy(), yo.cpu().numpy(), zo.cpu().numpy()), 1e-9)

    bufs = [torch.empty(6, dtype=torch.float64, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    outs = [_kkt_noalloc(L, lp, x, y, z, stream, out=b) for b in bufs]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0, "a call allocated device memory"
    np.testing.assert_array_equal(outs[0], outs[1])
    ref = oracle.kkt(inst, x.cpu().numpy(), y.cpu().numpy(), z.cpu().numpy())
    for o in outs:
        _agree(o, info, 1e-7)     # what the solve reported for this point
        _agree(o, ref, 1e-9)      # the oracle's evaluation of the same point

    # a point that is not a solution: random x, y, z (multipliers of both
    # signs, including at infinite bounds, whose dual-objective terms are
    # left out)
    for seed in (5, 6):
        g = torch.Generator().manual_seed(seed)
        xr = torch.randn(inst.n, generator=g, dtype=torch.float64).cuda()
        yr = torch.randn(inst.m, generator=g, dtype=torch.float64).cuda()
        zr = torch.randn(inst.n, generator=g, dtype=torch.float64).cuda()
        o = _kkt_noalloc(L, lp, xr, yr, zr, stream)
        _agree(o, oracle.kkt(inst, xr.cpu().numpy(), yr.cpu().numpy(), zr.cpu().numpy()), 1e-9)

    # null arguments are refused before any launch
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    ptr = lambda t: C.c_void_p(t.data_ptr())
    assert L.lib().scuc_lp_kkt_noalloc(lp.h, None, ptr(y), ptr(z), ptr(out)) == L.SCUC_E_INVALID
    lp_o.close()
    lp.close()
