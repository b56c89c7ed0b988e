"""CPU oracle (plain FP64 numpy) for the learned warm start.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check of
``__graft_entry__`` and by ``bench.py``'s CPU legs.  It shares no code with
the CUDA library: every function below is the plain definition, written out
with numpy array operations and loops.

The paper has no learned component; these are the definitions of the
network, its loss and gradients, Adam, and the construction of a starting
point for the iteration of Eq. 9 from per generator-hour predictions of the
commitment u (Eq. 1), the output above minimum p' (Eq. 3) and the price of
the balance row of Eq. 6.

Network (``params``: list of (W_l, b_l), W_l of shape [d_l, d_{l+1}]):
    h_0 = (x - mean) / scale
    z_l = h_{l-1} W_l + b_l,  h_l = max(z_l, 0) for hidden layers
    o   = z_{L-1};  predictions (sigmoid(o_0), sigmoid(o_1), o_2)
Loss of a batch (mean over samples) with targets (u*, r*, q*):
    softplus(o_0) - u* o_0 + w_d (sigmoid(o_1) - r*)^2 + w_p (o_2 - q*)^2
Adam (Kingma and Ba): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
    w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Pins (tests/test_oracle_ws.py): central finite differences of the loss;
torch.autograd on the same network in FP64; the closed-form loss of a network
whose weights are all zero; the closed-form first Adam step; invariants of
the assembled starting point (bounds, Eq. 1 logic, segment sums, price means).
"""
from __future__ import annotations

import numpy as np


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def softplus(z):
    return np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))


def forward(params, mean, scale, X):
    """Outputs o [rows, 3] and the hidden activations [h_0, h_1, ...]."""
    h = (np.asarray(X, np.float64) - mean) / scale
    hs = [h]
    L = len(params)
    for l, (W, b) in enumerate(params):
        z = h @ W + b
        if l < L - 1:
            z = np.maximum(z, 0.0)
        h = z
        hs.append(h)
    return h, hs


def predict(params, mean, scale, X):
    o, _ = forward(params, mean, scale, X)
    return np.stack([sigmoid(o[:, 0]), sigmoid(o[:, 1]), o[:, 2]], axis=1)


def loss(params, mean, scale, X, Y, w_d=1.0, w_p=1.0):
    o, _ = forward(params, mean, scale, X)
    Y = np.asarray(Y, np.float64)
    per = (softplus(o[:, 0]) - Y[:, 0] * o[:, 0] + w_d * (sigmoid(o[:, 1]) - Y[:, 1]) ** 2
           + w_p * (o[:, 2] - Y[:, 2]) ** 2)
    return float(per.mean())


def gradients(params, mean, scale, X, Y, w_d=1.0, w_p=1.0):
    """(loss, [(dW_l, db_l)]) by backpropagation through the definitions above."""
    o, hs = forward(params, mean, scale, X)
    Y = np.asarray(Y, np.float64)
    n = o.shape[0]
    su, sr = sigmoid(o[:, 0]), sigmoid(o[:, 1])
    lval = float((softplus(o[:, 0]) - Y[:, 0] * o[:, 0] + w_d * (sr - Y[:, 1]) ** 2
                  + w_p * (o[:, 2] - Y[:, 2]) ** 2).mean())
    d = np.zeros_like(o)
    d[:, 0] = (su - Y[:, 0]) / n                       # d/do0 of softplus(o0) - y o0
    d[:, 1] = 2.0 * w_d * (sr - Y[:, 1]) * sr * (1.0 - sr) / n
    d[:, 2] = 2.0 * w_p * (o[:, 2] - Y[:, 2]) / n
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        h_in = hs[l]
        grads[l] = (h_in.T @ d, d.sum(axis=0))
        if l > 0:
            d = (d @ W.T) * (hs[l] > 0.0)
    return lval, grads


def adam_step(params, grads, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t = step number, from 1); returns new (params, m, v)."""
    out_p, out_m, out_v = [], [], []
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        new = []
        for w_, g_, m_, v_ in ((W, gW, mW, vW), (b, gb, mb, vb)):
            m2 = b1 * m_ + (1.0 - b1) * g_
            v2 = b2 * v_ + (1.0 - b2) * g_ * g_
            w2 = w_ - lr * (m2 / (1.0 - b1 ** t)) / (np.sqrt(v2 / (1.0 - b2 ** t)) + eps)
            new.append((w2, m2, v2))
        out_p.append((new[0][0], new[1][0]))
        out_m.append((new[0][1], new[1][1]))
        out_v.append((new[0][2], new[1][2]))
    return out_p, out_m, out_v


def unflatten(vec, dims):
    """Parameter vector (W_0 row-major, b_0, W_1, b_1, ...) -> [(W, b)]."""
    vec = np.asarray(vec, np.float64)
    out, off = [], 0
    for a, b in zip(dims[:-1], dims[1:]):
        W = vec[off:off + a * b].reshape(a, b); off += a * b
        bb = vec[off:off + b]; off += b
        out.append((W, bb))
    assert off == len(vec)
    return out


def flatten(params):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


# ---------------------------------------------------------------------------
# starting point and targets
# ---------------------------------------------------------------------------

def _unit(q):
    """A prediction as a value in [0, 1]; NaN counts as 0."""
    q = float(q)
    if q > 0.0:
        return q if q < 1.0 else 1.0
    return 0.0


def _clamp(v, lo, hi):
    return lo if v < lo else (hi if v > hi else v)


def assemble(lay, pred, xl, xu, m, fill):
    """Starting point (x0, y0) from predictions pred [G*T, 3] (float32).

    ``lay`` holds host arrays: G, T, u_col, v_col, w_col, p_col, seg_col
    [G*T, nseg], p_cap, seg_cap [G*T, nseg], u_init, price_row, price_ptr,
    price_member, price_scale.  fill bits: 1 = v, w from the change of u
    (Eq. 1), 2 = p' over the cost segments in order (Eq. 5), 4 = duals of the
    price rows.  Loops over unit-hours, in the order of the definitions."""
    G, T = lay["G"], lay["T"]
    n = len(xl)
    x0 = np.array([_clamp(0.0, xl[j], xu[j]) for j in range(n)], dtype=np.float64)
    y0 = np.zeros(m)
    pred = np.asarray(pred, np.float32)
    for g in range(G):
        for t in range(T):
            k = g * T + t
            u = _unit(pred[k, 0])
            r = min(_unit(pred[k, 1]), u)
            p = r * float(lay["p_cap"][k])
            j = lay["u_col"][k]; x0[j] = _clamp(u, xl[j], xu[j])
            j = lay["p_col"][k]; x0[j] = _clamp(p, xl[j], xu[j])
            if fill & 1:
                prev = _unit(pred[k - 1, 0]) if t > 0 else float(lay["u_init"][g])
                d = u - prev
                j = lay["v_col"][k]; x0[j] = _clamp(max(d, 0.0), xl[j], xu[j])
                j = lay["w_col"][k]; x0[j] = _clamp(max(-d, 0.0), xl[j], xu[j])
            if fill & 2:
                rem = p
                for h in range(lay["seg_col"].shape[1]):
                    cap = float(lay["seg_cap"][k, h]) * u
                    s = min(rem, cap)
                    rem = rem - s
                    j = lay["seg_col"][k, h]; x0[j] = _clamp(s, xl[j], xu[j])
    if fill & 4:
        for q in range(len(lay["price_row"])):
            a, b = lay["price_ptr"][q], lay["price_ptr"][q + 1]
            s = 0.0
            for e in range(a, b):
                s = s + float(pred[lay["price_member"][e], 2])
            mean = s / (b - a) if b > a else 0.0
            y0[lay["price_row"][q]] = lay["price_scale"] * mean
    return x0, y0


def targets(lay, x, y):
    """Training targets [G*T, 3] (float32) of a solution (x, y)."""
    GT = lay["G"] * lay["T"]
    Y = np.zeros((GT, 3), np.float32)
    for k in range(GT):
        Y[k, 0] = np.float32(x[lay["u_col"][k]])
        Y[k, 1] = np.float32(x[lay["p_col"][k]] / lay["p_cap"][k])
        row = lay["unit_price_row"][k]
        Y[k, 2] = np.float32(y[row] / lay["price_scale"]) if row >= 0 else np.float32(0.0)
    return Y
