"""Train the filter MLP on the GPU with the library's own forward/backward/Adam kernels.

Input: the train_data*.npz files next to this file (features, and per graph the normalised
quadratic (Gn, bn) of the loss ||sum_j c_j T_j(A_hat) X - P X||^2 / ||P X||^2; written by the
oracle's data script): train_data.npz (SBMs and kNN graphs, n = 10^3 .. 10^5),
train_data_large.npz (SBMs with n up to 2^21), train_data_many_k.npz (SBMs with k = 25 .. 100)
and train_data_large_knn.npz (kNN graphs with 2 10^4 .. 8 10^4 points).  Output: mlp_weights.npz (5833 float32 parameters that take the raw features)
and train_summary.json.

Features are standardised for training (mean / std of the training split) and the affine map is
folded into the first layer when saving.  The output bias starts at the best constant
coefficient vector over the training graphs (the minimiser of the summed quadratics), so the
network starts from one fixed degree-8 filter and learns per-graph corrections.

Usage: python -m paper_2310_10939_gb300.filter.train [--epochs 300] [--out DIR]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    import torch

    import paper_2310_10939_gb300 as fsc

    ap = argparse.ArgumentParser()
    ap.add_argument("--data", default=",".join(p for p in (os.path.join(HERE, "train_data.npz"),
                                                            os.path.join(HERE, "train_data_large.npz"),
                                                            os.path.join(HERE, "train_data_many_k.npz"),
                                                            os.path.join(HERE, "train_data_large_knn.npz"))
                                               if os.path.exists(p)))
    ap.add_argument("--out", default=HERE)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--eval-every", type=int, default=10)
    ap.add_argument("--val-frac", type=float, default=0.15)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()

    parts = [np.load(f) for f in args.data.split(",") if f]
    d = {key: np.concatenate([q[key] for q in parts]) for key in ("f", "G", "b", "loss8", "loss22", "best", "n", "k")}
    F, Gn, bn = d["f"], d["G"], d["b"]
    N = F.shape[0]
    ok = np.isfinite(F).all(1) & np.isfinite(Gn.reshape(N, -1)).all(1) & np.isfinite(bn).all(1)
    idx = np.random.default_rng(args.seed + 1).permutation(np.nonzero(ok)[0])
    nval = int(round(args.val_frac * idx.size))
    val, tr = np.sort(idx[:nval]), np.sort(idx[nval:])
    mu = F[tr].mean(0)
    sd = F[tr].std(0)
    sd[sd < 1e-8] = 1.0
    dev = torch.device("cuda")
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    Fn_tr, G_tr, b_tr = T((F[tr] - mu) / sd), T(Gn[tr].reshape(-1, 81)), T(bn[tr])
    Fn_va, G_va, b_va = T((F[val] - mu) / sd), T(Gn[val].reshape(-1, 81)), T(bn[val])

    rng = np.random.default_rng(args.seed)
    W1 = rng.normal(0, math.sqrt(2.0 / 16), (64, 16))
    W2 = rng.normal(0, math.sqrt(2.0 / 64), (64, 64))
    W3 = rng.normal(0, 1e-3, (9, 64))
    c0 = np.linalg.solve(Gn[tr].sum(0), bn[tr].sum(0))      # best single filter for the training set
    theta = np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), W3.ravel(), c0])
    P = T(theta)
    grad = torch.zeros_like(P)
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    loss_buf = torch.zeros(1, dtype=torch.float32, device=dev)

    def eval_loss(Fn, G, b):
        g = torch.zeros_like(P)
        l = torch.zeros(1, dtype=torch.float32, device=dev)
        fsc.mlp_train_step(P, g, m, v, 1, 0.0, Fn, G, b, loss=l, apply_update=False)
        return float(l.item())

    start = {"train": eval_loss(Fn_tr, G_tr, b_tr), "val": eval_loss(Fn_va, G_va, b_va)}
    steps_per_epoch = max(1, tr.size // args.batch)
    total = args.epochs * steps_per_epoch
    step = 0
    t0 = time.time()
    history = []
    best_val, best_params, best_epoch = float("inf"), P.clone(), -1
    for ep in range(args.epochs):
        perm = torch.as_tensor(rng.permutation(tr.size), device=dev)
        for s in range(steps_per_epoch):
            sel = perm[s * args.batch:(s + 1) * args.batch]
            step += 1
            lr = args.lr * 0.5 * (1.0 + math.cos(math.pi * step / total))
            fsc.mlp_train_step(P, grad, m, v, step, lr, Fn_tr[sel].contiguous(), G_tr[sel].contiguous(),
                               b_tr[sel].contiguous(), loss=loss_buf, apply_update=True)
        if ep % args.eval_every == 0 or ep == args.epochs - 1:
            vl = eval_loss(Fn_va, G_va, b_va)
            if vl < best_val:                      # keep the best validation snapshot
                best_val, best_epoch = vl, ep
                best_params.copy_(P)
            if ep % (10 * args.eval_every) == 0 or ep == args.epochs - 1:
                history.append({"epoch": ep, "train": eval_loss(Fn_tr, G_tr, b_tr), "val": vl})
    torch.cuda.synchronize()
    secs = time.time() - t0
    P.copy_(best_params)

    # fold the standardisation into the first layer: W1' = W1 / sd, b1' = b1 - W1' mu
    th = P.cpu().numpy().astype(np.float64)
    W1 = th[:1024].reshape(64, 16) / sd[None, :]
    th[:1024] = W1.ravel()
    th[1024:1088] = th[1024:1088] - W1 @ mu
    params = th.astype(np.float32)
    np.savez(os.path.join(args.out, "mlp_weights.npz"), params=params)

    # validation report: raw-feature inference through the library, loss per graph
    Pw = torch.as_tensor(params, device=dev)
    c = fsc.mlp_forward(Pw, T(F[val])).cpu().numpy().astype(np.float64)
    lv = np.array([c[i] @ Gn[val][i] @ c[i] - 2 * bn[val][i] @ c[i] + 1.0 for i in range(val.size)])
    summary = {
        "graphs": int(N), "train": int(tr.size), "val": int(val.size), "epochs": args.epochs, "steps": step,
        "train_seconds": round(secs, 2), "start": start, "history": history, "best_epoch": best_epoch,
        "val_mean_loss_learned": float(lv.mean()),
        "val_mean_loss_plain_t8": float(d["loss8"][val].mean()),
        "val_mean_loss_plain_t22": float(d["loss22"][val].mean()),
        "val_mean_loss_best_degree8": float(np.nanmean(d["best"][val])),
        "val_frac_learned_beats_t8": float((lv < d["loss8"][val]).mean()),
        "val_frac_learned_beats_t22": float((lv < d["loss22"][val]).mean()),
    }
    big = d["n"][val] >= 100_000
    if big.any():
        summary.update({
            "val_large_graphs": int(big.sum()),
            "val_large_mean_loss_learned": float(lv[big].mean()),
            "val_large_mean_loss_plain_t22": float(d["loss22"][val][big].mean()),
            "val_large_mean_loss_best_degree8": float(np.nanmean(d["best"][val][big])),
            "val_large_frac_learned_beats_t22": float((lv[big] < d["loss22"][val][big]).mean()),
        })
    with open(os.path.join(args.out, "train_summary.json"), "w") as fh:
        json.dump(summary, fh, indent=1)
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
