"""Pins of the warm-start oracle (CPU, FP64): finite differences, an
independent autograd implementation, closed forms and invariants."""
import numpy as np
import pytest

from oracle import ws_oracle as O


def _net(dims, seed):
    rng = np.random.default_rng(seed)
    params = [(rng.normal(0, 1.0 / np.sqrt(a), (a, b)), rng.normal(0, 0.1, b))
              for a, b in zip(dims[:-1], dims[1:])]
    mean = rng.normal(0, 1, dims[0])
    scale = rng.uniform(0.5, 2.0, dims[0])
    return params, mean, scale


def _data(rows, F, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 1, (rows, F))
    Y = np.stack([rng.uniform(0, 1, rows), rng.uniform(0, 1, rows), rng.normal(0.5, 0.2, rows)], 1)
    return X, Y


def test_gradients_match_central_differences():
    dims = (5, 7, 6, 3)
    params, mean, scale = _net(dims, 1)
    X, Y = _data(9, 5, 2)
    wd, wp = 0.7, 1.3
    _, grads = O.gradients(params, mean, scale, X, Y, wd, wp)
    vec = O.flatten(params)
    gvec = O.flatten(grads)
    h = 1e-6
    num = np.zeros_like(vec)
    for i in range(len(vec)):
        e = np.zeros_like(vec); e[i] = h
        lp = O.loss(O.unflatten(vec + e, dims), mean, scale, X, Y, wd, wp)
        lm = O.loss(O.unflatten(vec - e, dims), mean, scale, X, Y, wd, wp)
        num[i] = (lp - lm) / (2 * h)
    # ReLU kinks are away from the sampled points with probability 1
    assert np.max(np.abs(num - gvec)) <= 1e-7 * max(1.0, np.max(np.abs(gvec)))


def test_gradients_match_torch_autograd():
    torch = pytest.importorskip("torch")
    dims = (4, 8, 8, 3)
    params, mean, scale = _net(dims, 3)
    X, Y = _data(13, 4, 4)
    loss, grads = O.gradients(params, mean, scale, X, Y, 0.5, 2.0)
    tp = [(torch.tensor(W, dtype=torch.float64, requires_grad=True),
           torch.tensor(b, dtype=torch.float64, requires_grad=True)) for W, b in params]
    h = (torch.tensor(X) - torch.tensor(mean)) / torch.tensor(scale)
    for l, (W, b) in enumerate(tp):
        h = h @ W + b
        if l < len(tp) - 1:
            h = torch.relu(h)
    y = torch.tensor(Y)
    per = (torch.nn.functional.softplus(h[:, 0]) - y[:, 0] * h[:, 0]
           + 0.5 * (torch.sigmoid(h[:, 1]) - y[:, 1]) ** 2 + 2.0 * (h[:, 2] - y[:, 2]) ** 2)
    tl = per.mean()
    tl.backward()
    assert abs(tl.item() - loss) <= 1e-12 * max(1.0, abs(loss))
    for (gW, gb), (W, b) in zip(grads, tp):
        np.testing.assert_allclose(gW, W.grad.numpy(), rtol=1e-10, atol=1e-13)
        np.testing.assert_allclose(gb, b.grad.numpy(), rtol=1e-10, atol=1e-13)


def test_zero_weight_network_loss_closed_form():
    # all weights zero: every output equals the last layer's bias, so the loss
    # is the per-target closed form of constant predictions
    dims = (3, 4, 3)
    b = np.array([0.3, -1.2, 0.8])
    params = [(np.zeros((3, 4)), np.zeros(4)), (np.zeros((4, 3)), b)]
    X, Y = _data(6, 3, 5)
    l = O.loss(params, np.zeros(3), np.ones(3), X, Y, 1.0, 1.0)
    s1 = 1.0 / (1.0 + np.exp(1.2))
    expect = np.mean(np.log(1.0 + np.exp(0.3)) - Y[:, 0] * 0.3 + (s1 - Y[:, 1]) ** 2 + (0.8 - Y[:, 2]) ** 2)
    assert abs(l - expect) < 1e-13
    # and the bias gradient of the last layer is the mean residual of each head
    _, g = O.gradients(params, np.zeros(3), np.ones(3), X, Y)
    s0 = 1.0 / (1.0 + np.exp(-0.3))
    np.testing.assert_allclose(g[1][1], [np.mean(s0 - Y[:, 0]), np.mean(2 * (s1 - Y[:, 1]) * s1 * (1 - s1)),
                                         np.mean(2 * (0.8 - Y[:, 2]))], rtol=1e-12)


def test_adam_first_step_is_lr_times_sign():
    # with zero moments the bias-corrected first step is -lr g / (|g| + eps)
    params = [(np.array([[1.0, -2.0]]), np.array([0.5, 0.0]))]
    grads = [(np.array([[0.3, -4.0]]), np.array([1e-3, -7.0]))]
    zeros = [(np.zeros((1, 2)), np.zeros(2))]
    p1, m1, v1 = O.adam_step(params, grads, zeros, zeros, 1, lr=0.01, eps=1e-8)
    for (W0, b0), (W1, b1), (gW, gb) in zip(params, p1, grads):
        np.testing.assert_allclose(W1 - W0, -0.01 * gW / (np.abs(gW) + 1e-8), rtol=1e-12)
        np.testing.assert_allclose(b1 - b0, -0.01 * gb / (np.abs(gb) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m1[0][0], 0.1 * grads[0][0])
    np.testing.assert_allclose(v1[0][0], 0.001 * grads[0][0] ** 2)


@pytest.fixture(scope="module")
def small_inst():
    from scuc_gen import make_preset
    return make_preset("scuc14")


def _lay(inst):
    from scuc_gen.features import ws_layout_arrays
    return ws_layout_arrays(inst)


def test_assemble_invariants(small_inst):
    inst = small_inst
    lay = _lay(inst)
    G, T = inst.G, inst.T
    rng = np.random.default_rng(7)
    pred = np.stack([rng.uniform(-0.2, 1.2, G * T), rng.uniform(-0.2, 1.2, G * T),
                     rng.normal(0.5, 0.1, G * T)], 1).astype(np.float32)
    x0, y0 = O.assemble(lay, pred, inst.xl, inst.xu, inst.m, 7)
    assert np.all(x0 >= inst.xl) and np.all(x0 <= inst.xu)
    u = x0[lay["u_col"]].reshape(G, T)
    np.testing.assert_array_equal(u.ravel(), np.clip(pred[:, 0].astype(np.float64), 0, 1))
    prev = np.concatenate([inst.u_init[:, None].astype(float), u[:, :-1]], 1)
    v = x0[lay["v_col"]].reshape(G, T)
    w = x0[lay["w_col"]].reshape(G, T)
    np.testing.assert_allclose(v - w, u - prev, atol=1e-15)      # Eq. 1 logic row holds
    assert np.all(v * w == 0)
    p = x0[lay["p_col"]]
    assert np.all(p <= lay["p_cap"] * u.ravel() + 1e-15)          # Eq. 3 production limit holds
    seg = x0[lay["seg_col"]]
    np.testing.assert_allclose(seg.sum(axis=1), p, rtol=1e-14, atol=1e-15)  # Eq. 5 segment sum
    assert np.all(seg <= lay["seg_cap"] * u.ravel()[:, None] + 1e-15)
    # segments fill in order: a later segment is used only when the earlier are full
    full = np.isclose(seg, lay["seg_cap"] * u.ravel()[:, None], rtol=1e-14, atol=1e-15)
    for h in range(1, seg.shape[1]):
        assert np.all((seg[:, h] == 0) | full[:, h - 1])
    # price rows: price_scale times the mean prediction of their members
    for q, row in enumerate(lay["price_row"]):
        mem = lay["price_member"][lay["price_ptr"][q]:lay["price_ptr"][q + 1]]
        np.testing.assert_allclose(y0[row], lay["price_scale"] * pred[mem, 2].astype(np.float64).mean(),
                                   rtol=1e-14)
    others = np.setdiff1d(np.arange(inst.m), lay["price_row"])
    assert np.all(y0[others] == 0)
    # columns outside the unit-hours start at the projection of 0
    unit_cols = np.concatenate([lay["u_col"], lay["v_col"], lay["w_col"], lay["p_col"], lay["seg_col"].ravel()])
    rest = np.setdiff1d(np.arange(inst.n), unit_cols)
    np.testing.assert_array_equal(x0[rest], np.clip(0.0, inst.xl[rest], inst.xu[rest]))


def test_assemble_without_fill_leaves_v_w_segments_at_zero(small_inst):
    inst = small_inst
    lay = _lay(inst)
    pred = np.full((inst.G * inst.T, 3), 0.5, np.float32)
    x0, y0 = O.assemble(lay, pred, inst.xl, inst.xu, inst.m, 0)
    assert np.all(x0[lay["v_col"]] == 0) and np.all(x0[lay["seg_col"]] == 0)
    np.testing.assert_array_equal(x0[lay["p_col"]], 0.5 * lay["p_cap"])
    assert np.all(y0 == 0)


def test_targets_invert_assembly(small_inst):
    # targets of an assembled point give back the predictions (u, min(r, u))
    inst = small_inst
    lay = _lay(inst)
    rng = np.random.default_rng(9)
    GT = inst.G * inst.T
    pred = np.stack([rng.uniform(0, 1, GT), rng.uniform(0, 1, GT), rng.normal(0.5, 0.1, GT)], 1).astype(np.float32)
    x0, y0 = O.assemble(lay, pred, inst.xl, inst.xu, inst.m, 7)
    Y = O.targets(lay, x0, y0)
    np.testing.assert_array_equal(Y[:, 0], pred[:, 0])
    np.testing.assert_allclose(Y[:, 1], np.minimum(pred[:, 1], pred[:, 0]), rtol=2e-7, atol=1e-7)
    # each unit-hour's price target is the mean predicted price of its row
    for k in range(GT):
        row = lay["unit_price_row"][k]
        q = np.searchsorted(lay["price_row"], row)
        mem = lay["price_member"][lay["price_ptr"][q]:lay["price_ptr"][q + 1]]
        assert abs(Y[k, 2] - pred[mem, 2].astype(np.float64).mean()) < 1e-6
