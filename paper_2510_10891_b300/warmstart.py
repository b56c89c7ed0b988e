"""Learned warm start: Python face of include/scuc_ws.h (argument marshalling
only; the network's forward and backward passes, Adam, the assembly of the
starting point and the extraction of targets run in the CUDA library).
Device buffers are torch CUDA tensors."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L

DEFAULT_DIMS = (12, 256, 256, 256, 3)


def _dp(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _torch():
    import torch
    return torch


def train_params(**kw) -> L.WsTrainParams:
    p = L.WsTrainParams()
    L.lib().scuc_ws_default_train_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError("unknown training parameter %r" % k)
        setattr(p, k, v)
    return p


def init_params(dims, seed: int) -> np.ndarray:
    """Seeded initial parameters: W_l ~ N(0, 2/d_l) (1/d_l for the output
    layer), b_l = 0, flattened in the library's layout."""
    rng = np.random.default_rng(seed)
    parts = []
    for l, (a, b) in enumerate(zip(dims[:-1], dims[1:])):
        gain = 1.0 if l == len(dims) - 2 else 2.0
        parts.append(rng.normal(0.0, np.sqrt(gain / a), size=(a, b)).ravel())
        parts.append(np.zeros(b))
    return np.concatenate(parts).astype(np.float32)


class WarmStartNet:
    """The network of scuc_ws_create on the current CUDA device."""

    def __init__(self, dims=DEFAULT_DIMS, stream: int | None = None):
        self.dims = tuple(int(d) for d in dims)
        arr = (C.c_int32 * len(self.dims))(*self.dims)
        h = C.c_void_p()
        L.check(L.lib().scuc_ws_create(C.byref(h), len(self.dims) - 1, arr,
                                       C.c_void_p(stream) if stream else None))
        self.h = h
        cnt = C.c_int64()
        L.check(L.lib().scuc_ws_num_params(self.h, C.byref(cnt)))
        self.nparams = cnt.value
        self.mean = np.zeros(self.dims[0], np.float32)
        self.scale = np.ones(self.dims[0], np.float32)

    def close(self):
        if getattr(self, "h", None):
            L.lib().scuc_ws_destroy(self.h)
            self.h = None

    __del__ = close

    def set_params(self, vec):
        vec = np.ascontiguousarray(vec, dtype=np.float32)
        if vec.size != self.nparams:
            raise ValueError("expected %d parameters, got %d" % (self.nparams, vec.size))
        L.check(L.lib().scuc_ws_set_params(self.h, C.c_void_p(vec.ctypes.data)))

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.nparams, np.float32)
        L.check(L.lib().scuc_ws_get_params(self.h, C.c_void_p(out.ctypes.data)))
        return out

    def set_gemm(self, kind):
        """Forward-product kernels: "tcgen05" (default: the eligible hidden
        layers on the fifth-generation tensor cores) or "mma_sync" (all
        layers on mma.sync)."""
        L.check(L.lib().scuc_ws_set_gemm(self.h, {"tcgen05": 0, "mma_sync": 1}[kind]))

    def set_input_norm(self, mean, scale):
        self.mean = np.ascontiguousarray(mean, dtype=np.float32)
        self.scale = np.ascontiguousarray(scale, dtype=np.float32)
        L.check(L.lib().scuc_ws_set_input_norm(self.h, C.c_void_p(self.mean.ctypes.data),
                                               C.c_void_p(self.scale.ctypes.data)))

    def predict(self, X, out=None):
        """X: CUDA float32 [rows, dims[0]] -> CUDA float32 [rows, 3] (u, r, price)."""
        torch = _torch()
        rows = int(X.shape[0])
        if out is None:
            out = torch.empty((rows, 3), dtype=torch.float32, device=X.device)
        L.check(L.lib().scuc_ws_predict(self.h, _dp(X), rows, _dp(out)))
        return out

    def gradients(self, X, Y, **tp):
        """(loss, gradient vector) of the mean loss over all rows of X, Y."""
        p = train_params(**tp)
        g = np.zeros(self.nparams, np.float32)
        loss = C.c_double()
        L.check(L.lib().scuc_ws_gradients(self.h, _dp(X), _dp(Y), int(X.shape[0]), C.byref(p),
                                          C.c_void_p(g.ctypes.data), C.byref(loss)))
        return loss.value, g

    def train(self, X, Y, idx, batch: int, steps: int, **tp) -> np.ndarray:
        """steps Adam steps; idx: CUDA int32 [steps*batch] sample indices.
        Returns the loss of every step's batch."""
        p = train_params(**tp)
        losses = np.zeros(max(steps, 1))
        L.check(L.lib().scuc_ws_train(self.h, _dp(X), _dp(Y), int(X.shape[0]), _dp(idx), int(batch),
                                      int(steps), C.byref(p), C.c_void_p(losses.ctypes.data)))
        return losses[:steps]

    # ----- persistence -----
    def save(self, path, **meta):
        np.savez_compressed(path, dims=np.asarray(self.dims, np.int32), params=self.get_params(),
                            mean=self.mean, scale=self.scale,
                            meta=np.asarray(repr(meta)))

    @classmethod
    def load(cls, path, stream: int | None = None):
        z = np.load(path, allow_pickle=False)
        net = cls(tuple(int(d) for d in z["dims"]), stream)
        net.set_params(z["params"])
        net.set_input_norm(z["mean"], z["scale"])
        return net


class Layout:
    """scuc_ws_layout with its arrays resident on the GPU.  ``arrays`` is the
    dict of scuc_gen.features.ws_layout_arrays; ``fill`` the SCUC_WS_FILL_*
    bits of the parts assembled beyond u and p'."""

    def __init__(self, arrays: dict, fill: int = 0, device="cuda"):
        torch = _torch()
        self.arrays = arrays
        t = {}
        for k in ("u_col", "v_col", "w_col", "p_col", "seg_col", "unit_price_row", "price_row",
                  "price_ptr", "price_member"):
            t[k] = torch.as_tensor(np.ascontiguousarray(arrays[k], dtype=np.int32), device=device)
        for k in ("p_cap", "seg_cap", "u_init"):
            t[k] = torch.as_tensor(np.ascontiguousarray(arrays[k], dtype=np.float64), device=device)
        self.t = t
        s = L.WsLayout()
        s.G, s.T = int(arrays["G"]), int(arrays["T"])
        s.nseg = int(np.asarray(arrays["seg_col"]).shape[1]) if np.asarray(arrays["seg_col"]).ndim == 2 else 0
        s.fill = int(fill)
        for k, v in t.items():
            setattr(s, k, v.data_ptr())
        s.nprice = int(len(arrays["price_row"]))
        s.price_scale = float(arrays["price_scale"])
        self.s = s

    @property
    def GT(self):
        return self.s.G * self.s.T

    def with_fill(self, fill: int) -> "Layout":
        other = Layout.__new__(Layout)
        other.arrays, other.t = self.arrays, self.t
        s = L.WsLayout()
        C.pointer(s)[0] = self.s
        s.fill = int(fill)
        other.s = s
        return other


def launches_predict(dims) -> int:
    """Kernels one scuc_ws_predict launches: standardisation, a product and a
    bias/activation kernel per layer, the output maps."""
    return 2 + 2 * (len(dims) - 1)


def launches_assemble(layout: "Layout") -> int:
    """Kernels one scuc_ws_assemble launches: the index checks of the arrays
    the fill bits use, the base point, the unit-hours and the price rows."""
    f = layout.s.fill
    checks = 2 + (2 if f & L.WS_FILL_VW else 0) + (1 if f & L.WS_FILL_SEGMENTS else 0)
    prices = f & L.WS_FILL_PRICES and layout.s.nprice > 0
    if prices:
        checks += 3                       # rows, pointers, members
    return checks + 2 + (1 if prices else 0)


def assemble(lp, layout: Layout, pred, x0=None, y0=None):
    """Starting point from predictions (scuc_ws_assemble); returns (x0, y0)
    CUDA float64 tensors (y0 only when given or when FILL_PRICES is set)."""
    torch = _torch()
    if x0 is None:
        x0 = torch.empty(lp.n, dtype=torch.float64, device=pred.device)
    if y0 is None and layout.s.fill & L.WS_FILL_PRICES:
        y0 = torch.empty(lp.m, dtype=torch.float64, device=pred.device)
    L.check(L.lib().scuc_ws_assemble(lp.h, C.byref(layout.s), _dp(pred), _dp(x0), _dp(y0)))
    return x0, y0


def targets(lp, layout: Layout, x, y, out=None):
    """Training targets of a solution (scuc_ws_targets): CUDA float32 [G*T, 3]."""
    torch = _torch()
    if out is None:
        out = torch.empty((layout.GT, 3), dtype=torch.float32, device=x.device)
    L.check(L.lib().scuc_ws_targets(lp.h, C.byref(layout.s), _dp(x), _dp(y), _dp(out)))
    return out
