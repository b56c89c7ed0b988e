"""Training set and training of the warm-start network.

The training data are solutions the method itself produces: seeded synthetic
SCUC instances (the uneven batch family of scuc_gen.batch_configs: 200-3,000
buses, 0.15 units per bus, T in {24, 36}) solved from cold start on the GPU
to 1e-4 KKT; the targets of every unit-hour are extracted from the solution
on the GPU (scuc_ws_targets).  Training runs the library's own forward,
backward and Adam kernels (scuc_ws_train).

    python -m paper_2510_10891_b300.ws_train --instances 2000 --steps 20000 \\
        --out paper_2510_10891_b300/weights/ws_mlp.npz
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import time

import numpy as np

from . import warmstart as W
from .lp import LP

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "weights", "ws_mlp.npz")


def _make(cfg):
    from scuc_gen.features import ws_features, ws_layout_arrays
    from scuc_gen.scuc import make_scuc
    inst = make_scuc(cfg)
    return inst, ws_features(inst), ws_layout_arrays(inst)


def generate(cfgs, workers: int = 16):
    """Instances with their features and layouts, built in spawned worker
    processes (no CUDA state is shared)."""
    if workers <= 1 or len(cfgs) <= 1:
        return [_make(c) for c in cfgs]
    with mp.get_context("spawn").Pool(min(workers, len(cfgs))) as pool:
        return pool.map(_make, cfgs)


def solve_targets(inst, feats, arrays, tol=1e-4, precision="mixed"):
    """Cold solve on the GPU; returns (X, Y, info) as CUDA tensors."""
    import torch
    lp = LP(inst)
    x = torch.empty(lp.n, dtype=torch.float64, device="cuda")
    y = torch.empty(lp.m, dtype=torch.float64, device="cuda")
    info = lp.solve_device(x_out=x, y_out=y, tol=tol, precision=precision)
    lay = W.Layout(arrays)
    Y = W.targets(lp, lay, x, y)
    X = torch.as_tensor(feats, device="cuda")
    lp.close()
    return X, Y, info


def collect(items, tol=1e-4, precision="mixed"):
    import torch
    Xs, Ys, infos = [], [], []
    for inst, feats, arrays in items:
        X, Y, info = solve_targets(inst, feats, arrays, tol, precision)
        if info["status"] != 0:
            continue  # only solutions that reached the tolerance are kept
        Xs.append(X); Ys.append(Y); infos.append(info)
    return torch.cat(Xs), torch.cat(Ys), infos


def collect_batched(items, group=64, tol=1e-4, precision="mixed"):
    """The same targets from batched cold solves (scuc_lp_solve_batch) of
    consecutive groups of instances, in order, on the default partition
    shapes (timed shapes could differ between runs and change the rounding
    of the solutions, so the weights would not be reproducible)."""
    import torch
    from .lp import solve_batch
    Xs, Ys, infos = [], [], []
    for g0 in range(0, len(items), group):
        grp = items[g0:g0 + group]
        lps = [LP(inst) for inst, _, _ in grp]
        outs = [(torch.empty(lp.n, dtype=torch.float64, device="cuda"),
                 torch.empty(lp.m, dtype=torch.float64, device="cuda"), None) for lp in lps]
        res, _ = solve_batch(lps, outputs=outs, autotune=False, tol=tol, precision=precision)
        for (inst, feats, arrays), lp, (x, y, _), r in zip(grp, lps, outs, res):
            if r["info"]["status"] != 0:
                continue  # only solutions that reached the tolerance are kept
            Ys.append(W.targets(lp, W.Layout(arrays), x, y))
            Xs.append(torch.as_tensor(feats, device="cuda"))
            infos.append(r["info"])
        for lp in lps:
            lp.close()
    return torch.cat(Xs), torch.cat(Ys), infos


def fit(X, Y, steps=3000, batch=4096, seed=0, dims=W.DEFAULT_DIMS, **tp):
    """Standardisation from the training features, seeded initial weights and
    sample draws (one permutation per epoch), then training on the GPU."""
    import torch
    Xh = X.double().cpu().numpy()
    mean = Xh.mean(axis=0)
    scale = Xh.std(axis=0)
    scale[scale < 1e-6] = 1.0
    net = W.WarmStartNet(dims)
    net.set_params(W.init_params(dims, seed))
    net.set_input_norm(mean.astype(np.float32), scale.astype(np.float32))
    rng = np.random.default_rng(seed + 1)
    n = X.shape[0]
    need = steps * batch
    draws = np.concatenate([rng.permutation(n) for _ in range((need + n - 1) // n)])[:need]
    idx = torch.as_tensor(draws.astype(np.int32), device="cuda")
    losses = net.train(X, Y, idx, batch, steps, **tp)
    return net, losses


def mean_predictor(Y, rows):
    """The feature-independent baseline: every unit-hour gets the mean target
    of the training set."""
    import torch
    mean = Y.double().cpu().numpy().mean(axis=0).astype(np.float32)
    return torch.as_tensor(np.tile(mean, (rows, 1)), device="cuda")


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--instances", type=int, default=2000)
    ap.add_argument("--first-seed", type=int, default=10000)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--workers", type=int, default=16)
    ap.add_argument("--out", default=WEIGHTS)
    a = ap.parse_args(argv)
    from scuc_gen.scuc import batch_configs
    t0 = time.time()
    items = generate(batch_configs(a.instances, a.first_seed), a.workers)
    t1 = time.time()
    X, Y, infos = collect_batched(items)
    t2 = time.time()
    net, losses = fit(X, Y, a.steps, a.batch, a.seed)
    t3 = time.time()
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    meta = dict(instances=a.instances, kept=len(infos), first_seed=a.first_seed, steps=a.steps,
                batch=a.batch, seed=a.seed, samples=int(X.shape[0]), final_loss=float(losses[-100:].mean()),
                gen_s=round(t1 - t0, 1), solve_s=round(t2 - t1, 1), train_s=round(t3 - t2, 1))
    net.save(a.out, **meta)
    print(meta)


if __name__ == "__main__":
    main()
