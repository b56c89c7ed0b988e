"""GPU parity of the learned warm start (include/scuc_ws.h) against the CPU
oracle, through the C ABI: network forward and gradients within the error of
BF16 operands, Adam and determinism, the assembled starting point and the
training targets bit for bit, the warm solve with its cold-start fallback,
and the gain of the trained network on the 13k-bus relaxation."""
import numpy as np
import pytest

import oracle
from oracle import ws_oracle as O

pytestmark = pytest.mark.gpu

DIMS = (12, 256, 256, 256, 3)


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.fixture(scope="module")
def P(torch_cuda):
    import paper_2510_10891_b300 as P
    return P


@pytest.fixture(scope="module")
def W(P):
    from paper_2510_10891_b300 import warmstart as W
    return W


def _bf16(a, torch):
    """Round to BF16 (nearest even) and back, as the kernels stage operands."""
    return torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _features(rows, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 1, (rows, DIMS[0])).astype(np.float32) * 2.0 + 0.5
    Y = np.stack([rng.uniform(0, 1, rows), rng.uniform(0, 1, rows), rng.normal(0.5, 0.2, rows)],
                 1).astype(np.float32)
    return X, Y


def _net(W, seed, mean, scale):
    net = W.WarmStartNet(DIMS)
    vec = W.init_params(DIMS, seed)
    # non-zero biases exercise the bias paths
    rng = np.random.default_rng(seed + 100)
    params = O.unflatten(vec.astype(np.float64), DIMS)
    params = [(Wl, rng.normal(0, 0.1, bl.shape)) for Wl, bl in params]
    vec = O.flatten(params).astype(np.float32)
    net.set_params(vec)
    net.set_input_norm(mean, scale)
    return net, vec


def _oracle_params(vec, torch):
    """Oracle parameters as the kernels see them: BF16 weights, FP32 biases."""
    ps = O.unflatten(vec.astype(np.float64), DIMS)
    return [(_bf16(Wl, torch), bl) for Wl, bl in ps]


def _std_bf16(X, mean, scale, torch):
    return _bf16((X - mean) / scale, torch)


@pytest.mark.parametrize("rows", [1, 777, 4096 + 37])
def test_predict_matches_oracle(W, torch_cuda, rows):
    torch = torch_cuda
    X, _ = _features(rows, 1)
    mean = X.mean(0).astype(np.float32) if rows > 1 else np.zeros(DIMS[0], np.float32)
    scale = np.full(DIMS[0], 2.0, np.float32)
    net, vec = _net(W, 3, mean, scale)
    out = net.predict(torch.as_tensor(X, device="cuda")).cpu().numpy()
    # oracle on the BF16 operands the kernels use (standardised input, weights)
    o, _ = O.forward(_oracle_params(vec, torch), np.zeros(DIMS[0]), np.ones(DIMS[0]),
                     _std_bf16(X, mean, scale, torch))
    ref = np.stack([O.sigmoid(o[:, 0]), O.sigmoid(o[:, 1]), o[:, 2]], 1)
    err = np.abs(out - ref)
    # hidden activations are rounded to BF16 (relative 2^-9) before each product
    assert err.max() < 0.03, err.max(axis=0)
    assert np.median(err) < 0.004


@pytest.mark.parametrize("rows", [1, 127, 128, 4096 + 37])
def test_tcgen05_forward_matches_mma_sync(W, torch_cuda, rows):
    """The hidden layers' products on tcgen05 (TMA, tensor-memory accumulator,
    fused bias and ReLU: the default) against the same network on mma.sync:
    both multiply the same BF16 operands with FP32 accumulation, so they
    differ by the order of the FP32 sums (and a rare BF16 rounding of an
    activation that this moves); ragged row counts around the 128-row tile.
    Gradients of a batch agree the same way."""
    torch = torch_cuda
    X, Y = _features(rows, 11)
    mean = X.mean(0).astype(np.float32) if rows > 1 else np.zeros(DIMS[0], np.float32)
    scale = np.full(DIMS[0], 2.0, np.float32)
    net, _ = _net(W, 13, mean, scale)
    Xd = torch.as_tensor(X, device="cuda")
    net.set_gemm("mma_sync")
    ref = net.predict(Xd).cpu().numpy()
    net.set_gemm("tcgen05")
    out = net.predict(Xd).cpu().numpy()
    err = np.abs(out - ref)
    assert err.max() < 5e-3 and err.mean() < 1e-4, (err.max(), err.mean())
    if rows > 1:
        Yd = torch.as_tensor(Y, device="cuda")
        l1, g1 = net.gradients(Xd, Yd)
        net.set_gemm("mma_sync")
        l0, g0 = net.gradients(Xd, Yd)
        assert l1 == pytest.approx(l0, rel=1e-4)
        assert np.linalg.norm(g1 - g0) <= 1e-3 * np.linalg.norm(g0)


def test_gradients_match_oracle(W, torch_cuda):
    torch = torch_cuda
    rows = 1000 + 13
    X, Y = _features(rows, 5)
    mean, scale = X.mean(0), X.std(0)
    net, vec = _net(W, 7, mean.astype(np.float32), scale.astype(np.float32))
    loss, g = net.gradients(torch.as_tensor(X, device="cuda"), torch.as_tensor(Y, device="cuda"),
                            w_dispatch=0.8, w_price=1.5)
    lo, go = O.gradients(_oracle_params(vec, torch), np.zeros(DIMS[0]), np.ones(DIMS[0]),
                         _std_bf16(X, mean.astype(np.float32), scale.astype(np.float32), torch), Y, 0.8, 1.5)
    assert loss == pytest.approx(lo, rel=5e-3)
    gg = O.unflatten(g.astype(np.float64), DIMS)
    for l, ((gW, gb), (oW, ob)) in enumerate(zip(gg, go)):
        for a, b in ((gW, oW), (gb, ob)):
            rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
            # BF16 operands in every product of the backward pass
            assert rel < 0.03, (l, rel)
            cos = float((a * b).sum() / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30))
            assert cos > 0.999, (l, cos)


def test_adam_step_matches_oracle_and_training_is_deterministic(W, torch_cuda):
    torch = torch_cuda
    rows = 512
    X, Y = _features(rows, 11)
    mean, scale = X.mean(0).astype(np.float32), X.std(0).astype(np.float32)
    Xd, Yd = torch.as_tensor(X, device="cuda"), torch.as_tensor(Y, device="cuda")
    net, vec = _net(W, 13, mean, scale)
    _, g = net.gradients(Xd, Yd)
    idx = torch.arange(rows, dtype=torch.int32, device="cuda")
    net.train(Xd, Yd, idx, rows, 1, lr=1e-3)
    new = net.get_params()
    ps = O.unflatten(vec.astype(np.float64), DIMS)
    zeros = [(np.zeros_like(a), np.zeros_like(b)) for a, b in ps]
    po, _, _ = O.adam_step(ps, O.unflatten(g.astype(np.float64), DIMS), zeros, zeros, 1, lr=1e-3)
    np.testing.assert_allclose(new, O.flatten(po), rtol=1e-5, atol=2e-7)
    # determinism: the same start and draws give the same parameters, bit for bit
    rng = np.random.default_rng(0)
    draws = torch.as_tensor(rng.integers(0, rows, 64 * 50).astype(np.int32), device="cuda")
    a, _ = _net(W, 13, mean, scale)
    b, _ = _net(W, 13, mean, scale)
    la = a.train(Xd, Yd, draws, 64, 50)
    lb = b.train(Xd, Yd, draws, 64, 50)
    np.testing.assert_array_equal(a.get_params(), b.get_params())
    np.testing.assert_array_equal(la, lb)


def test_training_reduces_the_loss(W, torch_cuda):
    torch = torch_cuda
    rows = 20000
    rng = np.random.default_rng(21)
    X = rng.normal(0, 1, (rows, DIMS[0])).astype(np.float32)
    # a learnable target: commitment from a threshold, dispatch and price smooth
    Y = np.stack([(X[:, 0] - X[:, 1] > 0).astype(np.float32), 1 / (1 + np.exp(-X[:, 2])),
                  0.5 + 0.1 * np.tanh(X[:, 3])], 1).astype(np.float32)
    Xd, Yd = torch.as_tensor(X, device="cuda"), torch.as_tensor(Y, device="cuda")
    net = W.WarmStartNet(DIMS)
    net.set_params(W.init_params(DIMS, 0))
    net.set_input_norm(np.zeros(DIMS[0], np.float32), np.ones(DIMS[0], np.float32))
    draws = torch.as_tensor(rng.integers(0, rows, 400 * 1024).astype(np.int32), device="cuda")
    losses = net.train(Xd, Yd, draws, 1024, 400)
    assert np.all(np.isfinite(losses))
    assert losses[-20:].mean() < 0.35 * losses[:5].mean(), (losses[:5], losses[-20:])


def test_train_rejects_out_of_range_sample_index(P, W, torch_cuda):
    torch = torch_cuda
    X, Y = _features(100, 1)
    net = W.WarmStartNet(DIMS)
    idx = torch.as_tensor(np.array([0, 5, 100, 3], np.int32), device="cuda")
    with pytest.raises(P._lib.ScucError) as e:
        net.train(torch.as_tensor(X, device="cuda"), torch.as_tensor(Y, device="cuda"), idx, 4, 1)
    assert e.value.code == P._lib.SCUC_E_INVALID


# ---------------------------------------------------------------------------
# assembly, targets, warm solve
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def instances():
    from scuc_gen import make_preset
    from scuc_gen.scuc import batch_configs, make_scuc
    return {"scuc14": make_preset("scuc14"), "batch0": make_scuc(batch_configs(1, 10003)[0])}


def _pred(GT, seed, nan=False):
    rng = np.random.default_rng(seed)
    pred = np.stack([rng.uniform(-0.3, 1.3, GT), rng.uniform(-0.3, 1.3, GT), rng.normal(0.5, 0.2, GT)],
                    1).astype(np.float32)
    pred[::17, 0] = 1.0
    pred[::19, 0] = 0.0
    if nan:
        pred[::23, 0] = np.nan
        pred[::29, 1] = np.nan
    return pred


@pytest.mark.parametrize("name", ["scuc14", "batch0"])
@pytest.mark.parametrize("fill", [0, 1, 2, 4, 7])
def test_assemble_matches_oracle_bitwise(P, W, torch_cuda, instances, name, fill):
    torch = torch_cuda
    from scuc_gen.features import ws_layout_arrays
    inst = instances[name]
    arr = ws_layout_arrays(inst)
    lp = P.LP(inst)
    lay = W.Layout(arr, fill)
    pred = _pred(inst.G * inst.T, fill + 3, nan=(fill == 7))
    y0 = torch.full((inst.m,), 7.0, dtype=torch.float64, device="cuda")
    x0, y0 = W.assemble(lp, lay, torch.as_tensor(pred, device="cuda"), y0=y0)
    xo, yo = O.assemble(arr, pred, inst.xl, inst.xu, inst.m, fill)
    np.testing.assert_array_equal(x0.cpu().numpy(), xo)
    np.testing.assert_array_equal(y0.cpu().numpy(), yo)


@pytest.mark.parametrize("name", ["scuc14", "batch0"])
def test_targets_match_oracle_bitwise(P, W, torch_cuda, instances, name):
    torch = torch_cuda
    from scuc_gen.features import ws_layout_arrays
    inst = instances[name]
    arr = ws_layout_arrays(inst)
    lp = P.LP(inst)
    r = lp.solve(tol=1e-4)
    Yg = W.targets(lp, W.Layout(arr), torch.as_tensor(r["x"], device="cuda"),
                   torch.as_tensor(r["y"], device="cuda")).cpu().numpy()
    np.testing.assert_array_equal(Yg, O.targets(arr, r["x"], r["y"]))


def test_layout_index_errors_are_rejected(P, W, torch_cuda, instances):
    torch = torch_cuda
    from scuc_gen.features import ws_layout_arrays
    inst = instances["scuc14"]
    lp = P.LP(inst)
    pred = torch.as_tensor(_pred(inst.G * inst.T, 1), device="cuda")
    arr = dict(ws_layout_arrays(inst))
    bad = arr["u_col"].copy(); bad[5] = inst.n
    with pytest.raises(P._lib.ScucError) as e:
        W.assemble(lp, W.Layout(dict(arr, u_col=bad)), pred)
    assert e.value.code == P._lib.SCUC_E_INVALID
    badm = arr["price_member"].copy(); badm[-1] = inst.G * inst.T
    with pytest.raises(P._lib.ScucError):
        W.assemble(lp, W.Layout(dict(arr, price_member=badm), P._lib.WS_FILL_PRICES), pred)
    badr = arr["unit_price_row"].copy(); badr[0] = inst.m
    x = torch.zeros(inst.n, dtype=torch.float64, device="cuda")
    y = torch.zeros(inst.m, dtype=torch.float64, device="cuda")
    with pytest.raises(P._lib.ScucError):
        W.targets(lp, W.Layout(dict(arr, unit_price_row=badr)), x, y)


def test_reference_period_is_the_cold_first_check(P, instances):
    inst = instances["batch0"]
    lp = P.LP(inst)
    cold = lp.solve(tol=1e-4, precision="fp64")
    first = cold["log"][0]
    r = lp.solve_warm(cold["x"], tol=1e-4, precision="fp64")
    assert r["info"]["ref_iters"] == 64
    assert r["info"]["cold_first_kkt"] == max(first["rp"], first["rd"], first["gap"])


def test_warm_solve_from_the_solution_is_fast(P, instances):
    inst = instances["batch0"]
    lp = P.LP(inst)
    cold = lp.solve(tol=1e-6, precision="fp64")
    assert cold["info"]["status"] == 0
    warm = lp.solve_warm(cold["x"], cold["y"], tol=1e-6, precision="fp64")
    info = warm["info"]
    assert info["status"] == 0 and info["warm_iters"] == 0
    assert info["iters"] - info["ref_iters"] <= cold["info"]["iters"] // 4
    assert info["pobj"] == pytest.approx(cold["info"]["pobj"], rel=1e-5)


@pytest.mark.parametrize("first_check", [0, 1])
def test_warm_solve_falls_back_to_cold(P, instances, first_check):
    inst = instances["batch0"]
    lp = P.LP(inst)
    cold = lp.solve(tol=1e-4, precision="fp64")
    x_bad = np.where(np.isfinite(inst.xu), inst.xu, 0.0)     # every column at its upper bound
    r = lp.solve_warm(x_bad, warm_max_iter=64, first_check=first_check, tol=1e-4, precision="fp64")
    info = r["info"]
    assert info["status"] == 4          # SCUC_ST_FALLBACK_COLD
    assert info["warm_iters"] == 64
    assert info["ref_iters"] == 64 * first_check
    assert info["iters"] == 64 + 64 * first_check + cold["info"]["iters"]
    # the cold rerun is the plain cold solve (same lambda, same decisions)
    np.testing.assert_array_equal(r["x"], cold["x"])
    assert info["pobj"] == cold["info"]["pobj"]


def test_first_check_rejection_is_consistent(P, instances):
    inst = instances["batch0"]
    lp = P.LP(inst)
    x_bad = np.where(np.isfinite(inst.xu), inst.xu, 0.0)
    kmax = lambda e: max(e["rp"], e["rd"], e["gap"])
    kw = kmax(lp.solve(x0=x_bad, max_iter=64, tol=1e-12, precision="fp64")["log"][0])
    kc = kmax(lp.solve(max_iter=64, tol=1e-12, precision="fp64")["log"][0])
    r = lp.solve_warm(x_bad, tol=1e-4, precision="fp64")
    info = r["info"]
    assert info["cold_first_kkt"] == kc
    if kw >= kc:
        assert info["status"] == 4 and info["warm_iters"] == 64
    else:
        assert info["warm_iters"] != 64
    assert info["kkt"] <= 1e-4
    # a caller-supplied reference skips the reference period
    r2 = lp.solve_warm(x_bad, cold_first_kkt=kc, tol=1e-4, precision="fp64")
    assert r2["info"]["ref_iters"] == 0
    assert r2["info"]["iters"] == info["iters"] - 64


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_warm_solve_reuses_the_reference_period_scaling(P, instances, precision):
    """The warm solve after the cold reference period keeps the scaled data
    that period set up (nothing changed in between): its result is
    bit-identical to a warm solve given the same reference KKT, which sets
    the scaling (and lambda) up afresh."""
    inst = instances["batch0"]
    lp = P.LP(inst)
    cold = lp.solve(tol=1e-4, precision=precision)
    x0 = 0.9 * cold["x"] + 0.1 * np.clip(0.0, inst.xl, inst.xu)
    r1 = lp.solve_warm(x0, tol=1e-4, precision=precision)
    kc = r1["info"]["cold_first_kkt"]
    r2 = lp.solve_warm(x0, cold_first_kkt=kc, tol=1e-4, precision=precision)
    assert r1["info"]["ref_iters"] == 64 and r2["info"]["ref_iters"] == 0
    assert r1["info"]["status"] == r2["info"]["status"]
    assert r1["info"]["iters"] - 64 == r2["info"]["iters"]
    for k in ("x", "y", "z"):
        np.testing.assert_array_equal(r1[k], r2[k])


def test_warm_solve_matches_oracle_warm_solve(P, W, torch_cuda, instances):
    torch = torch_cuda
    from scuc_gen.features import ws_layout_arrays
    inst = instances["scuc14"]
    arr = ws_layout_arrays(inst)
    lp = P.LP(inst)
    # predictions near the optimum: the oracle's solution with noise
    sol = oracle.hpr_solve(inst, tol=1e-6)
    rng = np.random.default_rng(5)
    pred = O.targets(arr, sol["x"], sol["y"]) + rng.normal(0, 0.05, (inst.G * inst.T, 3)).astype(np.float32)
    x0, _ = W.assemble(lp, W.Layout(arr, 3), torch.as_tensor(pred, device="cuda"))
    x0h = x0.cpu().numpy()
    g = lp.solve_warm(x0h, tol=1e-6, precision="fp64")
    o = oracle.hpr_solve(inst, x_init=x0h, tol=1e-6)
    assert g["info"]["status"] == 0 and g["info"]["warm_iters"] == 0, g["info"]
    assert g["info"]["iters"] - g["info"]["ref_iters"] == o["info"]["iters"]
    assert g["info"]["pobj"] == pytest.approx(o["info"]["pobj"], rel=1e-9)
    np.testing.assert_allclose(g["x"], o["x"], rtol=0, atol=1e-7 * max(1.0, np.abs(o["x"]).max()))


# ---------------------------------------------------------------------------
# what the trained network buys
# ---------------------------------------------------------------------------

def test_trained_network_gains_on_the_13k_bus_relaxation(P, W, torch_cuda):
    """Trained on cold solutions of 32 smaller instances (the uneven batch
    family, seeds 10000-10031), evaluated on the held-out 13k-bus relaxation
    (seed 20000): the trained network's warm start must beat the cold start,
    an untrained (random-init) network and the feature-mean predictor."""
    torch = torch_cuda
    from paper_2510_10891_b300 import ws_train as T
    from scuc_gen import make_preset
    from scuc_gen.features import ws_features, ws_layout_arrays
    from scuc_gen.scuc import batch_configs
    items = T.generate(batch_configs(32, 10000), workers=16)
    X, Y, infos = T.collect(items)
    assert len(infos) >= 30
    net, losses = T.fit(X, Y, steps=2000, batch=4096, seed=0)
    assert losses[-100:].mean() < 0.5 * losses[:10].mean()
    inst = make_preset("scuc13k")
    lp = P.LP(inst)
    lay = W.Layout(ws_layout_arrays(inst))
    Xe = torch.as_tensor(ws_features(inst), device="cuda")
    kw = dict(tol=1e-4, precision="mixed")
    xc = torch.empty(lp.n, dtype=torch.float64, device="cuda")
    cold = lp.solve_device(x_out=xc, **kw)
    assert cold["status"] == 0
    untrained = W.WarmStartNet()
    untrained.set_params(W.init_params(W.DEFAULT_DIMS, 1))
    untrained.set_input_norm(net.mean, net.scale)
    preds = {"trained": net.predict(Xe), "untrained": untrained.predict(Xe),
             "feature_mean": T.mean_predictor(Y, Xe.shape[0])}
    res = {"cold": cold["iters"]}
    d = oracle.as_lp(inst)
    for name, pred in preds.items():
        x0, _ = W.assemble(lp, lay, pred)
        xw = torch.empty(lp.n, dtype=torch.float64, device="cuda")
        yw = torch.empty(lp.m, dtype=torch.float64, device="cuda")
        zw = torch.empty(lp.n, dtype=torch.float64, device="cuda")
        info = lp.solve_warm(x0, x_out=xw, y_out=yw, z_out=zw, **kw)["info"]
        assert info["kkt"] <= 1e-4
        # the oracle's FP64 evaluation of the returned point agrees
        k = oracle.kkt(d, xw.cpu().numpy(), yw.cpu().numpy(), zw.cpu().numpy())
        assert k["kkt"] <= 1e-4 * 1.0001 and k["kkt"] == pytest.approx(info["kkt"], rel=1e-6), (name, k, info)
        dist = float(torch.linalg.vector_norm(xw - xc) / torch.linalg.vector_norm(xc))
        res[name] = info["iters"]
        print("%s: %d iterations (%s), |x - x_cold| / |x_cold| = %.3g" % (name, info["iters"],
                                                                      info["status_name"], dist))
    print(res)
    assert res["trained"] <= 0.6 * res["cold"], res
    assert res["trained"] < res["untrained"], res
    assert res["trained"] < res["feature_mean"], res
