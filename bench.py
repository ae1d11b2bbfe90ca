#!/usr/bin/env python3
"""Benchmark of fast spectral clustering (Algorithm 2) on one GB300 per rank.

A step is one pass of the hot path over the resident CSR graph: fsc_create_graph (validation +
degrees) followed by the clustering call of the workload's path (start block, the sparse steps,
k-means++ seeding, Lloyd to convergence).

Default workload: SBM with n = 2^22 vertices, 100 equal blocks, expected intra-/inter-block
degree 36/4 (~84M undirected edges, unit weights), k = 100, l = 7.  The timed path is the learned
degree-8 polynomial filter in place of M^t (basis stored in float16, float32 accumulation), the
variants include the plain t = 22 power method in float32 it is compared against.

Prints one JSON line (rank 0).  `--impl reference` times the float64 oracle (plain C + OpenMP on
all host cores) on the same workload instead.  Under torchrun with N > 1 every rank runs its own
replica (one graph does not shard in this library), value = max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "sbm_n2p22_k100": dict(kind="sbm_gpu", n=2 ** 22, k=100, deg_in=36.0, deg_out=4.0, l=7, t=22, path="learned_f16",
                           seed=19,
                           desc="SBM n=2^22, 100 equal blocks, intra-degree 36, inter-degree 4 (GPU generator), "
                                "k=100, l=7: learned degree-8 filter, float16 basis (value) vs plain t=22 power "
                                "method in float32 and bfloat16 (variants)"),
    "sbm_n2p20_k100": dict(kind="sbm_gpu", n=2 ** 20, k=100, deg_in=36.0, deg_out=4.0, l=7, t=22, path="learned_f16",
                           seed=19,
                           desc="SBM n=2^20, 100 equal blocks, intra-degree 36, inter-degree 4 (GPU generator), "
                                "k=100, l=7: the 2^22-vertex configuration at a quarter of its size (ncu captures)"),
    "sbm_n2p20_k16": dict(kind="sbm", n=2 ** 20, k=16, deg_in=20.0, deg_out=2.0, l=4, t=20, path="plain_f32", seed=7,
                          desc="SBM n=2^20, 16 equal blocks, intra-degree 20, inter-degree 2, unit weights; "
                               "k=16, l=4, t=20, plain power method in float32"),
    "knn_2e5_k10": dict(kind="knn", npts=200_000, dim=32, ncomp=10, knn=10, k=10, l=4, t=20, path="plain_f32",
                        seed=5, desc="10-NN graph of 200,000 points in R^32 from a 10-component Gaussian mixture; "
                                     "k=10, l=4, t=20, plain power method in float32"),
    "image_481x321_bf16": dict(kind="image", k=8, l=3, t=30, path="plain_bf16", seed=3,
                               desc="481x321 Voronoi image graph, radius 3; k=8, l=3, t=30, plain power method, "
                                    "bfloat16 storage"),
    "sbm_batch_4096": dict(kind="batch", G=4096, n_range=(500, 50_000), k_range=(2, 20), deg_in=15.0, deg_out=1.5,
                           store="bf16", seed=13,
                           desc="4096 SBM graphs, n~U[500,50000], k~U[2,20], intra-degree 15, inter-degree 1.5, "
                                "l=ceil(log2 k), t=ceil(log2 n), bfloat16 iterates, float32 weights; one persistent "
                                "launch in a captured CUDA graph vs one fsc_cluster per graph"),
}
METRIC = "cluster ms & SpMM HBM GB/s (% peak) at matched ARI, learned/BF16 vs plain"
UNIT = "ms per clustering (create_graph + cluster)"
E2E_UNIT = "ms per clustering"
DEFAULT_WORKLOAD = "sbm_n2p22_k100"
PATH_DTYPE = {"learned_f16": "f16-store/f32-accumulate", "learned_f32": "f32", "learned_bf16": "bf16-store/f32-accumulate",
              "plain_f32": "f32", "plain_bf16": "bf16-store/f32-accumulate"}


def make_graph(w, device="cuda"):
    """workloads.Graph (host CSR) of the workload; the 2^22-vertex SBM comes from the GPU generator."""
    import workloads as W
    if w["kind"] == "sbm":
        return W.sbm_by_degree(w["n"], w["k"], w["deg_in"], w["deg_out"], seed=w["seed"])
    if w["kind"] == "knn":
        return W.knn_mixture(w["npts"], w["dim"], w["ncomp"], w["knn"], seed=w["seed"], device=device)
    if w["kind"] == "image":
        return W.image_grid(321, 481, 8, seed=w["seed"])
    if w["kind"] == "sbm_gpu":
        gb = W.sbm_batch_gpu(1, (w["n"], w["n"]), (w["k"], w["k"]), w["deg_in"], w["deg_out"], seed=w["seed"],
                             with_weights=False, device=device)
        return W.Graph(w["n"], gb.row_ptr.cpu().numpy(), gb.col.cpu().numpy(), None, gb.labels.cpu().numpy(),
                       f"sbm_n{w['n']}_k{w['k']}")
    raise ValueError(w["kind"])


# ---- algorithmic bytes per launch of the sparse kernels -------------------------------------

def csr_bytes(g):
    """CSR once (col, weights when present, int64 row_ptr) and 1/d once."""
    return 4 * g.nnz + (4 * g.nnz if g.w is not None else 0) + 8 * (g.n + 1) + 4 * g.n


def power_step_bytes(g, lp, s):
    """k_power_step: CSR + read the iterate once + write it once."""
    return csr_bytes(g) + 2 * g.n * lp * s


def cheb_step_bytes(g, lp, s):
    """k_cheb_step, mean over the 8 launches of one filter: CSR each launch; iterate rows read once
    (T_j) and written once (T_{j+1}); T_{j-1} read in launches 2..8; d(v) (float64) read in the four
    launches that also form the moments."""
    total = 8 * csr_bytes(g) + (2 + 7 * 3) * g.n * lp * s + 4 * 8 * g.n
    return total / 8.0


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy burst)"
    return 6800.0, "fallback 6.8 TB/s"


def read_traffic(summary_name, sources):
    """Per-launch DRAM bytes from a committed ncu summary, while the kernel sources it names still hash
    to the value recorded in it; None otherwise."""
    h = hashlib.sha256()
    for src in sources:
        h.update(open(os.path.join(ROOT, "paper_2310_10939_gb300", "csrc", src), "rb").read())
    sha = h.hexdigest()[:16]
    summ = os.path.join(ROOT, "profiles", f"{summary_name}.md")
    if not os.path.exists(summ):
        return None
    vals = {}
    for line in open(summ):
        if line.startswith("traffic_per_launch_bytes:") or line.startswith("kernel_source_sha:"):
            key, v = line.split(":", 1)
            vals[key.strip()] = v.strip()
    if vals.get("kernel_source_sha") != sha or "traffic_per_launch_bytes" not in vals:
        return None
    return float(vals["traffic_per_launch_bytes"])


def max_over_ranks(values, device):
    """Element-wise maximum of a list of floats over all ranks of the default process group
    (the timing rule for N > 1: the slowest rank's time is the job's)."""
    import torch
    x = torch.tensor(list(values), dtype=torch.float64, device=device)
    torch.distributed.all_reduce(x, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in x.cpu()]


# ---- the GPU arm -------------------------------------------------------------------------------

class Runner:
    """One clustering of the resident graph along a named path, through the C ABI."""

    def __init__(self, fsc, rp, col, wt, k, l, t, params):
        self.fsc, self.rp, self.col, self.wt = fsc, rp, col, wt
        self.k, self.l, self.t, self.params = k, l, t, params

    def run(self, path, seed, labels=None, events=None, mid=None, stream=None):
        """Returns (labels, stats, sparse launches bracketed by `events`)."""
        fsc = self.fsc
        G = fsc.Graph(self.rp, self.col, self.wt)
        if mid is not None:
            mid.record(stream)
        if path.startswith("learned"):
            store = {"learned_f16": fsc.F16, "learned_f32": fsc.F32, "learned_bf16": fsc.BF16}[path]
            lab, st = fsc.cluster_filtered(G, self.k, self.l, seed, self.params, store=store, labels=labels,
                                           events=events)
            launches = st["fallback_t"] if st["fallback"] else 8
        else:
            store = fsc.F32 if path == "plain_f32" else fsc.BF16
            lab, st = fsc.cluster(G, self.k, self.l, self.t, seed, store=store, labels=labels, rescale=True,
                                  events=events)
            launches = self.t
        G.close()
        return lab, st, launches


def timed_launch(fn, reps=10, warm=3):
    """Mean device time (ms) of fn() on the current stream, CUDA events after warm-up."""
    import torch
    for _ in range(warm):
        fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def gpu_arm(args, w, rank, world, local_rank):
    import torch
    import paper_2310_10939_gb300 as fsc

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    g = make_graph(w, device=f"cuda:{local_rank}")
    k, l, t, seed, path = w["k"], w["l"], w["t"], w["seed"], args.path or w["path"]
    rp = torch.as_tensor(g.row_ptr, device=dev)
    col = torch.as_tensor(g.col, device=dev)
    wt = None if g.w is None else torch.as_tensor(g.w, device=dev)
    planted = torch.as_tensor(g.labels.astype(np.int32), device=dev)
    kp = int(g.labels.max()) + 1
    params = fsc.load_filter_params(device=dev) if os.path.exists(fsc.FILTER_WEIGHTS) else None
    if path.startswith("learned") and params is None:
        raise RuntimeError("the learned path needs the trained filter weights")
    R = Runner(fsc, rp, col, wt, k, l, t, params)
    labels = torch.empty(g.n, dtype=torch.int32, device=dev)
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=dev)   # 512 MB > L2
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        R.run(path, seed, labels)
    torch.cuda.synchronize()

    ev = lambda: torch.cuda.Event(enable_timing=True)   # noqa: E731
    starts, ends, mids = [ev() for _ in range(args.steps)], [ev() for _ in range(args.steps)], \
        [ev() for _ in range(args.steps)]
    brackets = [(ev(), ev()) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    stats, nsparse = None, []
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        _, stats, nl = R.run(path, seed, labels, events=brackets[i], mid=mids[i], stream=stream)
        ends[i].record(stream)
        nsparse.append(nl)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = float(np.mean([s.elapsed_time(e) for s, e in zip(starts, ends)]))
    create_ms = float(np.mean([s.elapsed_time(m) for s, m in zip(starts, mids)]))
    sparse_ms = float(np.mean([a.elapsed_time(b) for a, b in brackets]))
    launch_ms = float(np.mean([a.elapsed_time(b) / n for (a, b), n in zip(brackets, nsparse)]))
    if world > 1:
        ms, launch_ms = max_over_ranks([ms, launch_ms], dev)
    ari = fsc.partition_scores(labels, planted, k, kp)[0]

    # end to end through the public API with host buffers: H2D of the CSR, create, cluster, D2H of labels
    rp_h = torch.as_tensor(g.row_ptr).pin_memory()
    col_h = torch.as_tensor(g.col).pin_memory()
    w_h = None if g.w is None else torch.as_tensor(g.w).pin_memory()
    lab_h = torch.empty(g.n, dtype=torch.int32).pin_memory()
    rp_d, col_d = torch.empty_like(rp), torch.empty_like(col)
    w_d = None if wt is None else torch.empty_like(wt)
    R_e2e = Runner(fsc, rp_d, col_d, w_d, k, l, t, params)
    h2d = rp_h.numel() * 8 + col_h.numel() * 4 + (0 if w_h is None else w_h.numel() * 4)
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rp_d.copy_(rp_h, non_blocking=True)
        col_d.copy_(col_h, non_blocking=True)
        if w_d is not None:
            w_d.copy_(w_h, non_blocking=True)
        lab_d, _, _ = R_e2e.run(path, seed)
        lab_h.copy_(lab_d, non_blocking=True)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e = float(np.mean(e2e_ms))
    if world > 1:
        e2e, = max_over_ranks([e2e], dev)
    del rp_d, col_d, w_d, R_e2e

    variants = None if args.no_variants else time_variants(R, g, planted, kp, seed, flush)
    lp = fsc.pad_l(l)
    peak, peak_src = read_peaks()
    floors = gather_floors(fsc, torch, rp, col, wt, l, dev)

    def roofline(kernel, variant, bytes_launch, ms_launch, s_name):
        achieved = bytes_launch / (ms_launch * 1e-3) / 1e9
        fl = floors.get(s_name)
        summary = f"{'cheb' if kernel == 'k_cheb_step' else 'spmm'}_{args.workload}_{s_name}"
        srcs = ["spmm.cuh", "filter.cu"] if kernel == "k_cheb_step" else ["spmm.cuh"]
        return {"kernel": kernel, "variant": variant, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": peak_src,
                "traffic": read_traffic(summary, srcs), "bytes_per_launch": int(bytes_launch),
                "launch_ms": round(ms_launch, 5),
                "gather_floor_ms": None if fl is None else round(fl, 5),
                "frac_of_gather_floor": None if fl is None else round(fl / ms_launch, 4)}

    value_store = {"learned_f16": "f16", "learned_f32": "f32", "learned_bf16": "bf16", "plain_f32": "f32",
                   "plain_bf16": "bf16"}[path]
    s_bytes = 4 if value_store == "f32" else 2
    if path.startswith("learned") and not stats["fallback"]:
        main_roof = roofline("k_cheb_step", path, cheb_step_bytes(g, lp, s_bytes), launch_ms, value_store)
    else:
        main_roof = roofline("k_power_step", path, power_step_bytes(g, lp, s_bytes), launch_ms, value_store)
    others = []
    for name, rec in (variants or {}).items():
        if not isinstance(rec, dict) or "sparse_launch_ms" not in rec or name == path:
            continue
        st_name = name.split("_")[-1]
        sb = 4 if st_name == "f32" else 2
        if name.startswith("learned") and not rec.get("fallback"):
            others.append(roofline("k_cheb_step", name, cheb_step_bytes(g, lp, sb), rec["sparse_launch_ms"], st_name))
        elif name.startswith("plain") or (name.startswith("learned") and rec.get("fallback")):
            others.append(roofline("k_power_step", name, power_step_bytes(g, lp, sb), rec["sparse_launch_ms"],
                                   st_name))

    out = {
        "metric": METRIC,
        "value": round(ms, 4),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 4),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": PATH_DTYPE[path],
        "data": "synthetic (seeded generator)",
        "config": {"workload": f"{args.workload}: {w['desc']}", "path": path, "n": g.n, "nnz": g.nnz, "k": k, "l": l,
                   "t": t if path.startswith("plain") else 8,
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "512 MB buffer written between timed steps (flush)"},
        "e2e": {"value": round(e2e, 4), "unit": E2E_UNIT,
                "region": "pinned host CSR -> device, create_graph, cluster, labels -> pinned host",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(g.n * 4)},
        "roofline": main_roof,
        "rooflines_other": others,
        "breakdown_ms": {"create_graph": round(create_ms, 4), "cluster": round(ms - create_ms, 4),
                         "sparse_steps": round(sparse_ms, 4)},
        "ari_vs_planted": round(ari, 4),
        "lloyd_iterations": stats["iterations"] if stats else None,
        "wall_s": round(wall, 3),
        "gpu_launches": args.steps * launches_per_step(path, stats, t),
        "clocks": clk,
        "variants": variants,
    }
    if path.startswith("learned"):
        out["filter"] = {"energy_ratio": round(stats["filter_energy_ratio"], 4),
                         "threshold": round(stats["filter_threshold"], 4), "fallback": int(stats["fallback"])}
    return out, g


def launches_per_step(path, stats, t):
    """Kernels of this library launched per step: degrees (1); plain: start block + t power steps;
    learned: start block + 8 Chebyshev steps + coefficients + combine (+ start block and t power
    steps on a fallback); k-means: k-means++ and Lloyd (2)."""
    if path.startswith("learned"):
        n = 1 + 1 + 8 + 1 + 1 + 2
        if stats and stats.get("fallback"):
            n += 1 + stats["fallback_t"]
        return n
    return 1 + 1 + t + 2


def gather_floors(fsc, torch, rp, col, wt, l, dev):
    """Mean duration (ms) of fsc_gather_floor on this graph for each storage type: the random-gather
    floor of one sparse step at this row width."""
    G = fsc.Graph(rp, col, wt)
    lp = fsc.pad_l(l)
    out = {}
    for name, st, dt in (("f32", fsc.F32, torch.float32), ("bf16", fsc.BF16, torch.bfloat16),
                         ("f16", fsc.F16, torch.float16)):
        z = torch.randn((G.n, lp), device=dev).to(dt)
        acc = torch.empty(1, dtype=torch.float32, device=dev)
        out[name] = timed_launch(lambda: fsc.gather_floor(G, l, z, store=st, out=acc), reps=10, warm=3)
        del z
    G.close()
    return out


def time_variants(R, g, planted, kp, seed, flush, steps=5):
    """Every path on the same graph: ms per clustering (create_graph + cluster), ARI against the planted
    labels, the mean sparse-step launch time, and for the filter the guard's energy ratio and whether it
    fell back; the median over 8 seeds of the time of one clustering and of its Lloyd iteration count;
    for every embedding, the ARI over 8 k-means seeds (median) and of the best of 8 by inertia."""
    import torch
    fsc = R.fsc
    out = {}
    paths = ["plain_f32", "plain_bf16"] + (["learned_f32", "learned_f16", "learned_bf16"] if R.params is not None else [])
    paths += ["orthogonal_f32", "pm_k_vectors_f32", "k_eigs_f32"]

    def one(path, sd, events=None):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        if path in ("orthogonal_f32", "pm_k_vectors_f32", "k_eigs_f32"):
            # orthogonal iteration (D-orthonormal every 4 steps) on the method's l columns, or on
            # l = k columns ("PM k Vectors"), or Rayleigh-Ritz on that basis ("k Eigenvectors")
            G = fsc.Graph(R.rp, R.col, R.wt)
            lw = R.l if path == "orthogonal_f32" else R.k
            if path == "k_eigs_f32":
                E = fsc.top_eigenvectors(G, lw, R.t, sd, every=4, events=events)[1]
            else:
                E = fsc.embed_orthogonal(G, lw, R.t, sd, every=4, events=events)
            lab, st, _, _ = fsc.kmeans(E, lw, R.k, sd)
            G.close()
            nl = R.t
        else:
            lab, st, nl = R.run(path, sd, events=events)
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b), lab, st, nl

    for path in paths:
        first = one(path, seed)[0]
        slow = first > 100.0          # the l = k variants at k = 100: fewer repetitions
        for _ in range(0 if slow else 2):
            one(path, seed)
        times, launch = [], []
        for _ in range(2 if slow else steps):
            evs = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            ms, lab, st, nl = one(path, seed, evs)
            times.append(ms)
            launch.append(evs[0].elapsed_time(evs[1]) / nl)
        rec = {"ms": round(float(np.mean(times)), 4),
               "ari_vs_planted": round(fsc.partition_scores(lab, planted, R.k, kp)[0], 4),
               "sparse_launch_ms": round(float(np.mean(launch)), 5)}
        if "filter_energy_ratio" in st:
            rec.update(energy_ratio=round(st["filter_energy_ratio"], 4), fallback=int(st["fallback"]))
        per_seed = [one(path, seed + s) for s in range(3 if slow else 8)]
        rec["ms_median_8_seeds" if not slow else "ms_median_3_seeds"] = round(float(np.median([x[0] for x in per_seed])), 4)
        rec["lloyd_iterations_median_8_seeds" if not slow else "lloyd_iterations_median_3_seeds"] = \
            float(np.median([x[2]["iterations"] for x in per_seed]))
        rec["lloyd_iterations"] = st["iterations"]
        out[path] = rec
    # k-means++ draws decide which local optimum Lloyd reaches, so one clustering per variant says
    # little about the embedding: ARI over 8 seeds (median) and of the best of 8 by inertia
    G = fsc.Graph(R.rp, R.col, R.wt)
    l, t, k = R.l, R.t, R.k
    embs = {"plain_f32": lambda: fsc.embed(G, l, t, seed),
            "plain_bf16": lambda: fsc.embed(G, l, t, seed, store=fsc.BF16, rescale=True),
            "orthogonal_f32": lambda: fsc.embed_orthogonal(G, l, t, seed, every=4),
            "pm_k_vectors_f32": lambda: fsc.embed_orthogonal(G, k, t, seed, every=4)}
    if R.params is not None:
        for name, st in (("learned_f32", fsc.F32), ("learned_f16", fsc.F16), ("learned_bf16", fsc.BF16)):
            embs[name] = (lambda st=st: fsc.filter_embed(G, l, k, seed, params=R.params, store=st)[0])
    for name, mk in embs.items():
        E = mk()
        le = k if name == "pm_k_vectors_f32" else l   # (k Eigs: a rotation of the same rows, same clusterings)
        aris = [fsc.partition_scores(fsc.kmeans(E, le, k, seed + s)[0], planted, k, kp)[0] for s in range(8)]
        lab = fsc.kmeans_best(E, le, k, seed, 8)[0]
        rec = out.setdefault(name, {})
        rec["ari_median_8_seeds"] = round(float(np.median(aris)), 4)
        rec["ari_best_of_8"] = round(fsc.partition_scores(lab, planted, k, kp)[0], 4)
        del E
    G.close()
    return out


# ---- the oracle on the host cores (CPU baseline and reference arm) -----------------------------

def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model", "hardware")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def oracle_sample(g, w, lloyd_iters, csr=None, threads=None):
    """Times a bounded sample of the float64 oracle's Algorithm 2 (plain power method) on the host
    cores and scales it to one clustering: degrees, the start block and the float32 embedding once;
    2 of the t power steps (x t/2); 3 of the k-1 k-means++ rounds (x (k-1)/3); one Lloyd iteration
    with k centres (x the clustering's Lloyd iteration count).  Returns (ms, detail)."""
    from oracle import omp
    if threads is not None:
        omp.set_threads(threads)
    csr = csr or omp.Csr(g)
    k, l, t, seed = w["k"], w["l"], w["t"], w["seed"]
    tm = {}
    t0 = time.perf_counter()
    deg, dinv = omp.degrees(csr)
    tm["degrees"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    x = omp.gaussian_block(g.n, l, seed)
    tm["start_block"] = time.perf_counter() - t0
    S = min(2, t)
    t0 = time.perf_counter()
    omp.power_method(csr, deg, dinv, x, S)
    tm["power_steps"] = (time.perf_counter() - t0) * (t / S if S else 0.0)
    t0 = time.perf_counter()
    B = omp.embedding_f32(dinv, x)
    tm["embedding"] = time.perf_counter() - t0
    rounds = min(4, k)
    t0 = time.perf_counter()
    omp.kmeanspp(B, k, seed, rounds=rounds)
    tm["kmeanspp"] = (time.perf_counter() - t0) * ((k - 1) / (rounds - 1) if rounds > 1 else 0.0)
    centres = np.linspace(0, g.n - 1, k).astype(np.int64)
    t0 = time.perf_counter()
    omp.lloyd(B, centres, max_iter=1)
    tm["lloyd"] = (time.perf_counter() - t0) * lloyd_iters
    ms = 1e3 * sum(tm.values())
    return ms, {key: round(v * 1e3, 2) for key, v in tm.items()}


def cpu_baseline(g, w, lloyd_iters):
    """The all-core leg and a single-core leg of the same sample."""
    from oracle import omp
    cores = omp.threads()
    csr = omp.Csr(g)
    ms, parts = oracle_sample(g, w, lloyd_iters, csr=csr, threads=cores)
    ms1, _ = oracle_sample(g, w, lloyd_iters, csr=csr, threads=1)
    omp.set_threads(cores)
    return {"value": round(ms, 1), "unit": E2E_UNIT, "cores": cores, "kind": "oracle",
            "sample": f"float64 oracle (plain C + OpenMP), plain power method t={w['t']}: degrees, start block and "
                      f"embedding once, 2 power steps x t/2, 3 k-means++ rounds x (k-1)/3, 1 Lloyd iteration x "
                      f"{lloyd_iters} (the clustering's count)",
            "phases_ms": parts, "single_core_ms": round(ms1, 1), "cpu": cpu_model()}


def reference_arm(args, w):
    """The float64 oracle on the host cores (the comparison arm): a full oracle clustering once, then per
    step the bounded sample of oracle_sample scaled to one clustering."""
    from oracle import metrics, omp
    dev = "cpu"
    try:
        import torch
        if torch.cuda.is_available():
            dev = "cuda"
    except ImportError:
        pass
    g = make_graph(w, device=dev)
    cores = omp.threads()
    t0 = time.perf_counter()
    full = omp.fast_spectral_cluster(g, w["k"], w["l"], w["t"], w["seed"])
    full_ms = (time.perf_counter() - t0) * 1e3
    iters = full["iters"]
    csr = omp.Csr(g)
    for _ in range(args.warmup):
        oracle_sample(g, w, iters, csr=csr)
    times = []
    parts = None
    for _ in range(args.steps):
        ms, parts = oracle_sample(g, w, iters, csr=csr)
        times.append(ms)
    ms = float(np.mean(times))
    return {
        "impl": "reference",
        "metric": METRIC,
        "value": round(ms, 2),
        "unit": UNIT,
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 2),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64 (k-means decisions in f32)",
        "data": "synthetic (seeded generator)",
        "config": {"workload": f"{args.workload}: {w['desc']}", "path": "plain power method (the paper's Algorithm 2)",
                   "n": g.n, "nnz": g.nnz, "k": w["k"], "l": w["l"], "t": w["t"]},
        "cpu_baseline": {"value": round(ms, 2), "unit": E2E_UNIT, "cores": cores, "kind": "oracle",
                         "sample": "per step: degrees, start block and embedding once, 2 power steps x t/2, 3 "
                                   "k-means++ rounds x (k-1)/3, 1 Lloyd iteration x the Lloyd iteration count of "
                                   "one full oracle clustering run before the steps",
                         "phases_ms": parts, "cpu": cpu_model(), "full_clustering_ms": round(full_ms, 1)},
        "e2e": {"value": round(ms, 2), "unit": E2E_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "ari_vs_planted": round(metrics.ari(full["labels"], g.labels), 4),
        "lloyd_iterations": iters,
    }


def batch_arm(args, w):
    """Batched clustering of thousands of graphs: one plan run (CUDA graph) per step."""
    import torch
    import paper_2310_10939_gb300 as fsc
    import workloads as W
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    gb = W.sbm_batch_gpu(w["G"], w["n_range"], w["k_range"], w["deg_in"], w["deg_out"], seed=w["seed"])
    gen_s = time.perf_counter() - t0
    store = fsc.BF16 if w["store"] == "bf16" else fsc.F32
    seeds = np.arange(gb.num_graphs, dtype=np.uint64) + 1
    t0 = time.perf_counter()
    plan = fsc.Batch(gb.vertex_offset, gb.row_ptr, gb.col, gb.k, seeds, w=gb.w, store=store, autotune=True)
    plan_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        plan.run()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(0)
    clocks.start()
    stream = torch.cuda.current_stream()
    for a, b in evs:
        a.record(stream)
        plan.run()
        b.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    stats, _, _ = plan.results()
    # per-graph launches: one fsc_create_graph + fsc_cluster per graph on the same CSR, its per-graph
    # views (local row pointers and column ids) prepared before the timed loop
    voff = gb.vertex_offset
    views = []
    for g in range(gb.num_graphs):
        lo, hi = int(voff[g]), int(voff[g + 1])
        rp = gb.row_ptr[lo:hi + 1]
        e0, e1 = int(rp[0]), int(rp[-1])
        views.append((rp - e0, gb.col[e0:e1] - lo, gb.w[e0:e1] if gb.w is not None else None,
                      fsc.default_params(hi - lo, int(gb.k[g]))))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g, (rp, col, wv, (l, t)) in enumerate(views):
        G = fsc.Graph(rp, col, wv)
        fsc.cluster(G, int(gb.k[g]), l, t, int(seeds[g]), store=store, rescale=True)
        G.close()
    torch.cuda.synchronize()
    per_graph_s = time.perf_counter() - t0
    del views
    nnz = int(gb.col.numel())
    out = {
        "metric": "graphs/s (batched clustering of many graphs)",
        "value": round(gb.num_graphs / (ms * 1e-3), 2),
        "unit": "graphs/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16-store/f32-accumulate" if store == fsc.BF16 else "f32",
        "data": "synthetic (seeded GPU generator)",
        "config": {"workload": f"{args.workload}: {w['desc']}", "graphs": gb.num_graphs,
                   "total_vertices": int(voff[-1]), "total_nnz": nnz,
                   "l2": "inputs (~14 GB CSR) far larger than L2"},
        "per_graph_launches": {"value": round(gb.num_graphs / per_graph_s, 2), "unit": "graphs/s",
                               "seconds": round(per_graph_s, 3)},
        "speedup_vs_per_graph": round(per_graph_s / (ms * 1e-3), 2),
        "mean_lloyd_iterations": round(float(np.mean([s_["iterations"] for s_ in stats])), 2),
        "generate_s": round(gen_s, 2), "plan_s": round(plan_s, 2),
        # per step: an embedding and a k-means kernel for each row width l_pad present
        "gpu_launches": args.steps * 2 * len({fsc.pad_l(fsc.default_params(int(voff[g + 1] - voff[g]), int(gb.k[g]))[0])
                                              for g in range(gb.num_graphs)}),
        "clocks": clk,
    }
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["fsc", "reference"], default="fsc")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--path", choices=sorted(PATH_DTYPE), default=None, help="override the workload's timed path")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    w = WORKLOADS[args.workload]
    if w["kind"] == "batch":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batched mode has no CPU reference arm"}))
        else:
            print(json.dumps(batch_arm(args, w)), flush=True)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(reference_arm(args, w)), flush=True)
        return

    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    out, g = gpu_arm(args, w, rank, world, local_rank)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        plain = (out.get("variants") or {}).get("plain_f32", {})
        iters = plain.get("lloyd_iterations") or out["lloyd_iterations"] or 1
        out["cpu_baseline"] = cpu_baseline(g, w, iters)
    if world > 1:
        import torch
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
