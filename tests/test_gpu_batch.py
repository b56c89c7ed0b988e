"""Batched solves (scuc_lp_solve_batch) through the C ABI: every LP of a
batch follows its own solve's iteration (same checks, restart decisions and
iteration counts as a solo solve and as the CPU oracle), solutions agree to
rounding, the autotuned partition shapes are valid, outputs land in host and
device buffers, and the 64-LP uneven batch converges faster together than
one by one."""
import multiprocessing as mp
import time

import numpy as np
import pytest

import oracle
from scuc_gen import random_lp
from scuc_gen.scuc import batch_configs, make_scuc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.fixture(scope="module")
def P(torch_cuda):
    import paper_2510_10891_b300 as P
    return P


def _compare_logs(glog, olog, rtol=1e-7):
    assert len(glog) == len(olog), (len(glog), len(olog))
    for g, o in zip(glog, olog):
        assert g["iter"] == o["iter"]
        assert g["restart"] == o["restart"], (g, o)
        for k in ("rp", "rd"):
            assert g[k] == pytest.approx(o[k], rel=rtol, abs=1e-13), (k, g, o)
        assert g["gap"] == pytest.approx(o["gap"], rel=rtol, abs=1e-11), ("gap", g, o)


def _mixed_sizes():
    # uneven LPs: random ones with long rows/columns, empty rows, and SCUC relaxations
    lps = [random_lp(300, 200, density=0.02, seed=1, long_rows=3, long_cols=2),
           random_lp(40, 30, density=0.2, seed=2),
           random_lp(1000, 700, density=0.004, seed=3, long_cols=4, senses="GE"),
           random_lp(513, 1025, density=0.01, seed=4, long_rows=2, senses="LR")]
    lps += [make_scuc(c) for c in batch_configs(3, 1000)[:3]]
    return lps


@pytest.fixture(scope="module")
def mixed_lps():
    return _mixed_sizes()


def test_batch_fp64_follows_each_solo_solve_and_the_oracle(P, mixed_lps):
    kw = dict(tol=1e-6, max_iter=20480, precision="fp64")
    handles = [P.LP(d) for d in mixed_lps]
    res, bi = P.solve_batch(handles, **kw)
    assert bi["blocks_A"] > 0 and bi["blocks_T"] > 0
    converged = 0
    for d, h, r in zip(mixed_lps, handles, res):
        solo = P.LP(d).solve(**kw)
        assert r["info"]["status"] == solo["info"]["status"], (r["info"]["status_name"], solo["info"]["status_name"])
        converged += r["info"]["status"] == 0
        assert r["info"]["iters"] == solo["info"]["iters"]
        _compare_logs(h.log(r["info"]["nlog"]), solo["log"])
        assert r["info"]["pobj"] == pytest.approx(solo["info"]["pobj"], rel=1e-9, abs=1e-12)
        scale = max(1.0, float(np.max(np.abs(solo["x"]))))
        assert float(np.max(np.abs(r["x"] - solo["x"]))) <= 1e-8 * scale
    assert converged >= 4          # the others stop at the iteration limit on both sides
    # the small LPs against the oracle directly
    for d, h, r in list(zip(mixed_lps, handles, res))[:2]:
        o = oracle.hpr_solve(d, **{k: v for k, v in kw.items() if k != "precision"})
        assert r["info"]["iters"] == o["info"]["iters"]
        _compare_logs(h.log(r["info"]["nlog"]), o["log"])


def test_batch_mixed_precision_certified_by_the_oracle(P, mixed_lps):
    handles = [P.LP(d) for d in mixed_lps]
    res, _ = P.solve_batch(handles, tol=1e-4, precision="mixed")
    for d, r in zip(mixed_lps, res):
        assert r["info"]["status"] == 0
        assert r["info"]["iters_fp32"] > 0 or r["info"]["iters"] <= 128
        k = oracle.kkt(d, r["x"], r["y"], r["z"])
        assert k["kkt"] <= 1e-4 * 1.0001, k


def test_autotune_shapes_and_untuned_partition(P, mixed_lps):
    handles = [P.LP(d) for d in mixed_lps]
    r1, b1 = P.solve_batch(handles, autotune=True, tol=1e-6, precision="fp64")
    # tuned now (12 shapes timed) or earlier in this process (same sizes)
    assert (b1["candidates"], b1["tune_cached"]) in ((12, 0), (0, 1))
    assert b1["ept_A"] in (8, 12, 16) and b1["ept_T"] in (8, 12, 16)
    assert b1["run_A"] in (16, 64) and b1["run_T"] in (16, 64)
    # a second batch of the same sizes reuses the tuned shapes without timing
    r2, b2 = P.solve_batch(handles, autotune=True, tol=1e-6, precision="fp64")
    assert b2["tune_cached"] == 1 and b2["candidates"] == 0
    assert [b2[k] for k in ("ept_A", "run_A", "ept_T", "run_T")] == [b1[k] for k in ("ept_A", "run_A", "ept_T",
                                                                                        "run_T")]
    for a, b in zip(r1, r2):
        assert a["info"]["iters"] == b["info"]["iters"] and a["info"]["pobj"] == b["info"]["pobj"]
    r0, b0 = P.solve_batch(handles, autotune=False, tol=1e-6, precision="fp64")
    assert b0["candidates"] == 2 and (b0["ept_A"], b0["run_A"]) == (12, 32)
    for a, b in zip(r1, r0):
        # another partition only changes the rounding order of the sums
        assert a["info"]["iters"] == b["info"]["iters"]
        assert a["info"]["pobj"] == pytest.approx(b["info"]["pobj"], rel=1e-9, abs=1e-12)


def test_batch_device_outputs_match_host_outputs(P, torch_cuda, mixed_lps):
    torch = torch_cuda
    handles = [P.LP(d) for d in mixed_lps]
    rh, _ = P.solve_batch(handles, autotune=False, tol=1e-5, precision="fp64")
    outs = [(torch.empty(h.n, dtype=torch.float64, device="cuda"), None,
             torch.empty(h.n, dtype=torch.float64, device="cuda")) for h in handles]
    rd, _ = P.solve_batch(handles, outputs=outs, autotune=False, tol=1e-5, precision="fp64")
    for a, b, (x, _, z) in zip(rh, rd, outs):
        np.testing.assert_array_equal(a["x"], x.cpu().numpy())
        np.testing.assert_array_equal(a["z"], z.cpu().numpy())
        assert a["info"]["iters"] == b["info"]["iters"]


def test_batch_rejects_a_repeated_handle(P, mixed_lps):
    h = P.LP(mixed_lps[0])
    with pytest.raises(P._lib.ScucError) as e:
        P.solve_batch([h, P.LP(mixed_lps[1]), h], tol=1e-4)
    assert e.value.code == P._lib.SCUC_E_INVALID
    res, _ = P.solve_batch([], tol=1e-4)
    assert res == []


def test_64_uneven_scuc_relaxations_batched(P):
    """The uneven batch family (64 instances, 200-3,000 buses, T in {24, 36},
    seeds 1000-1063): all reach 1e-4 together; the batch beats solving them
    one by one on the same GPU."""
    cfgs = batch_configs(64, 1000)
    with mp.get_context("spawn").Pool(16) as pool:
        insts = pool.map(make_scuc, cfgs)
    handles = [P.LP(i) for i in insts]
    kw = dict(tol=1e-4, precision="mixed")
    P.solve_batch(handles[:2], **kw)                         # warm-up (module load, first launches)
    t0 = time.perf_counter()
    res, bi = P.solve_batch(handles, **kw)
    t_batch = time.perf_counter() - t0
    assert all(r["info"]["status"] == 0 for r in res), [r["info"]["status_name"] for r in res]
    t0 = time.perf_counter()
    solo = [h.solve(want=("x",), **kw) for h in handles]
    t_solo = time.perf_counter() - t0
    print("64 LPs: batched %.2f s (setup %.0f ms, tune %.0f ms, iterations %.0f ms, shapes A %d/%d, "
          "A^T %d/%d), one by one %.2f s" % (t_batch, bi["setup_ms"], bi["tune_ms"], bi["solve_ms"],
                                            bi["ept_A"], bi["run_A"], bi["ept_T"], bi["run_T"], t_solo))
    for r, s in zip(res, solo):
        # same iteration; FP32 sums in another order can move a check across the tolerance
        assert abs(r["info"]["iters"] - s["info"]["iters"]) <= 256
    for i in (0, 17, 63):
        k = oracle.kkt(insts[i], res[i]["x"], res[i]["y"], res[i]["z"])
        assert k["kkt"] <= 1e-4 * 1.0001
    assert t_batch < t_solo
