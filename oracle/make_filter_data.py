"""Training and validation data for the learned filter, computed by the float64 oracle.

Writes paper_2310_10939_gb300/filter/train_data.npz.  For each graph (seeded SBMs and
Gaussian-mixture kNN graphs, sizes spanning n = 10^3 .. 10^5, k = 2 .. 100): the 16
features of its start block X (Philox stream of its seed, l = max(1, ceil(log2 k)) columns),
and the filter-loss quadratic normalised by e0 = ||PX||^2: Gn = G / e0, bn = b / e0, so
loss(c) = c^T Gn c - 2 bn^T c + 1.  Also stored: the loss of the plain power method with
t = 8 and t = 22 (Chebyshev coefficients of gamma^t are exact only for t <= 8, so t = 22 is
evaluated directly), and the best possible degree-8 loss 1 - bn^T Gn^-1 bn.

With --large the graphs are SBMs with n = 10^5 .. 2^21 and k = 2 .. 24 (written to
train_data_large.npz): there n / k, the number of bulk eigen-directions per signal one, reaches
10^5, the range in which the filter must suppress the bulk by 10^-3 or more.  With --many-k
they are SBMs with n = 10^5 .. 6 10^5, k = 25 .. 100 and mean degree 20 .. 40
(train_data_many_k.npz), for many clusters at large n.  With --large-knn they are 10-NN graphs of
Gaussian mixtures with 2 10^4 .. 8 10^4 points (train_data_large_knn.npz).

Usage: python -m oracle.make_filter_data [--graphs 3000] [--workers 8] [--large | --many-k | --large-knn]
(the committed files: defaults; --large --graphs 360; --many-k --graphs 72; --large-knn --graphs 90)
"""
from __future__ import annotations

import argparse
import math
import multiprocessing as mp
import os
import time

import numpy as np

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2310_10939_gb300", "filter", "train_data.npz")
OUT_LARGE = OUT.replace("train_data.npz", "train_data_large.npz")
OUT_MANY_K = OUT.replace("train_data.npz", "train_data_many_k.npz")
OUT_LARGE_KNN = OUT.replace("train_data.npz", "train_data_large_knn.npz")


def _draw(i: int, base_seed: int):
    rng = np.random.default_rng(base_seed * 1_000_003 + i)
    if rng.random() < 0.75:
        n = int(round(math.exp(rng.uniform(math.log(1000), math.log(100_000)))))
        kmax = min(100, n // 30, 50 if n > 40_000 else 100)
        k = int(round(math.exp(rng.uniform(math.log(2), math.log(kmax)))))
        deg_in = float(rng.uniform(10, 40))
        deg_out = deg_in * float(rng.uniform(0.03, 0.15))
        return ("sbm", n, k, deg_in, deg_out, int(rng.integers(1, 2**31)))
    npts = int(round(math.exp(rng.uniform(math.log(1000), math.log(20_000)))))
    k = int(rng.integers(3, 21))
    dim = int(rng.choice([8, 16, 32]))
    return ("knn", npts, k, dim, 10, int(rng.integers(1, 2**31)))


def _draw_large(i: int, base_seed: int):
    rng = np.random.default_rng(base_seed * 1_000_003 + 500_000_000 + i)
    n = int(round(math.exp(rng.uniform(math.log(100_000), math.log(2 ** 21)))))
    kmax = min(24, n // 2000)
    k = int(round(math.exp(rng.uniform(math.log(2), math.log(kmax)))))
    deg_in = float(rng.uniform(10, 40))
    deg_out = deg_in * float(rng.uniform(0.03, 0.15))
    return ("sbm", n, k, deg_in, deg_out, int(rng.integers(1, 2**31)))


def _draw_many_k(i: int, base_seed: int):
    rng = np.random.default_rng(base_seed * 1_000_003 + 900_000_000 + i)
    n = int(round(math.exp(rng.uniform(math.log(100_000), math.log(600_000)))))
    k = int(round(math.exp(rng.uniform(math.log(25), math.log(100)))))
    deg_in = float(rng.uniform(18, 36))
    deg_out = deg_in * float(rng.uniform(0.05, 0.15))
    return ("sbm", n, k, deg_in, deg_out, int(rng.integers(1, 2**31)))


def _draw_large_knn(i: int, base_seed: int):
    rng = np.random.default_rng(base_seed * 1_000_003 + 700_000_000 + i)
    npts = int(round(math.exp(rng.uniform(math.log(20_000), math.log(80_000)))))
    k = int(rng.integers(3, 21))
    dim = int(rng.choice([8, 16, 32]))
    return ("knn", npts, k, dim, 10, int(rng.integers(1, 2**31)))


def _record(spec):
    import workloads as W
    from oracle import filter as fl
    from oracle import spectral
    from oracle.rng import gaussian_block
    kind, n, k, a, b, seed = spec
    g = W.sbm_by_degree(n, k, a, b, seed=seed) if kind == "sbm" else W.knn_mixture(n, a, k, b, seed=seed)
    l = max(1, math.ceil(math.log2(k))) if k > 1 else 1
    X = gaussian_block(g.n, l, seed)
    f = fl.features(g, k, l, X)
    G, bb, e0 = fl.target(g, k, X)
    Gn, bn = G / e0, bb / e0
    loss8 = fl.filter_loss(fl.power_coefficients(8), G, bb, e0)
    PX = fl.top_projection(g, k, X)
    Y22 = spectral.power_method(spectral.signless_laplacian(g), X, 22)
    loss22 = float(((Y22 - PX) ** 2).sum() / e0)
    try:
        best = float(1.0 - bn @ np.linalg.solve(Gn, bn))
    except np.linalg.LinAlgError:
        best = float("nan")
    return dict(f=f, G=Gn, b=bn, loss8=loss8, loss22=loss22, best=best, n=g.n, k=k, l=l, seed=seed,
                kind=0 if kind == "sbm" else 1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--graphs", type=int, default=3000)
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 4)
    ap.add_argument("--seed", type=int, default=2023)
    ap.add_argument("--out", default=None)
    ap.add_argument("--large", action="store_true")
    ap.add_argument("--many-k", action="store_true")
    ap.add_argument("--large-knn", action="store_true")
    args = ap.parse_args()
    big = args.large or args.many_k or args.large_knn
    if args.out is None:
        args.out = (OUT_LARGE_KNN if args.large_knn else OUT_MANY_K if args.many_k else
                    OUT_LARGE if args.large else OUT)
    draw = (_draw_large_knn if args.large_knn else _draw_many_k if args.many_k else
            _draw_large if args.large else _draw)
    specs = [draw(i, args.seed) for i in range(args.graphs)]
    if big:   # largest first, so the pool ends on short jobs
        specs.sort(key=lambda sp: -sp[1])
    t0 = time.time()
    with mp.get_context("spawn").Pool(args.workers) as pool:
        recs = pool.map(_record, specs, chunksize=1 if big else 4)
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    np.savez_compressed(
        args.out,
        f=np.stack([r["f"] for r in recs]), G=np.stack([r["G"] for r in recs]), b=np.stack([r["b"] for r in recs]),
        loss8=np.array([r["loss8"] for r in recs]), loss22=np.array([r["loss22"] for r in recs]),
        best=np.array([r["best"] for r in recs]), n=np.array([r["n"] for r in recs]),
        k=np.array([r["k"] for r in recs]), l=np.array([r["l"] for r in recs]),
        seed=np.array([r["seed"] for r in recs]), kind=np.array([r["kind"] for r in recs]))
    print(f"{len(recs)} graphs in {time.time() - t0:.1f}s -> {args.out}")


if __name__ == "__main__":
    main()
