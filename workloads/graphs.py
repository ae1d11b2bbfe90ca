"""Seeded generators of undirected weighted graphs in CSR form.

Every generator returns a :class:`Graph` whose CSR holds both directions of
each undirected edge, column indices sorted within each row, no self-loops and
no duplicate entries.  ``w`` is ``None`` for unit weights, else float32 weights
computed in float64 and rounded once; edges whose float32 weight underflows to
zero are dropped, so every consumer sees the identical graph.

The workloads follow the paper's experiments (stochastic block model, Sec. 4.1;
k-nearest-neighbour graphs of labelled point sets, Sec. 4.2) and a pixel-grid
graph for image segmentation.  Vertex ids are assigned block by block
(cluster by cluster) as the generators build them; :func:`permuted` relabels.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Graph:
    n: int
    row_ptr: np.ndarray          # int64, n + 1
    col: np.ndarray              # int32, nnz
    w: np.ndarray | None         # float32, nnz, or None for unit weights
    labels: np.ndarray | None    # int32 planted cluster of each vertex, or None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @property
    def k_planted(self) -> int:
        return 0 if self.labels is None else int(self.labels.max()) + 1


def from_edges(n: int, u, v, w=None, labels=None, name: str = "", meta=None) -> Graph:
    """CSR of the undirected graph with edges {u[e], v[e]} (u != v, each pair once)."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    if u.size and (u == v).any():
        raise ValueError("self-loop in edge list")
    rows = np.concatenate([u, v])
    cols = np.concatenate([v, u])
    ww = None
    if w is not None:
        w = np.asarray(w, dtype=np.float32)
        ww = np.concatenate([w, w])
    key = rows * np.int64(n) + cols
    order = np.argsort(key)
    key = key[order]
    if key.size > 1 and (np.diff(key) == 0).any():
        raise ValueError("duplicate edge in edge list")
    rows = rows[order]
    cols = cols[order].astype(np.int32)
    if ww is not None:
        ww = ww[order]
    counts = np.bincount(rows, minlength=n).astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    lab = None if labels is None else np.asarray(labels, dtype=np.int32)
    return Graph(n, row_ptr, cols, ww, lab, name, dict(meta or {}))


def _sorted_unique(a: np.ndarray) -> np.ndarray:
    a = np.sort(a)
    if a.size:
        a = a[np.concatenate([[True], a[1:] != a[:-1]])]
    return a


def _block_starts(sizes):
    sizes = np.asarray(sizes, dtype=np.int64)
    starts = np.zeros(sizes.size + 1, dtype=np.int64)
    np.cumsum(sizes, out=starts[1:])
    return sizes, starts


def sbm(sizes, p_in: float, p_out: float, seed: int, name: str = "sbm") -> Graph:
    """Stochastic block model (Sec. 4.1): each within-block pair is an edge with
    probability ``p_in``, each cross-block pair with probability ``p_out``.

    Sampled exactly: for every block pair the edge count is Binomial(#pairs, p)
    and the edges are a uniform subset of that size (rejection of repeats).
    """
    rng = np.random.default_rng(seed)
    sizes, starts = _block_starts(sizes)
    k = sizes.size
    n = int(starts[-1])
    bi, bj = np.triu_indices(k)
    npairs = np.where(bi == bj, sizes[bi] * (sizes[bi] - 1) // 2, sizes[bi] * sizes[bj])
    prob = np.where(bi == bj, p_in, p_out)
    counts = rng.binomial(npairs, prob).astype(np.int64)
    group_of = -np.ones((k, k), dtype=np.int64)
    group_of[bi, bj] = np.arange(bi.size)
    block_of = np.repeat(np.arange(k, dtype=np.int64), sizes)

    keys = np.empty(0, dtype=np.int64)
    # dense block pairs (many of their pairs are edges): choose the subset from the full enumeration
    dense = (npairs <= 20000) | (counts * 4 >= npairs)
    dense_keys = []
    for gi in np.nonzero(dense & (counts > 0))[0]:
        b1, b2 = int(bi[gi]), int(bj[gi])
        if b1 == b2:
            iu, ju = np.triu_indices(int(sizes[b1]), 1)
            lo_c, hi_c = iu + starts[b1], ju + starts[b1]
        else:
            ii, jj = np.meshgrid(np.arange(sizes[b1]), np.arange(sizes[b2]), indexing="ij")
            lo_c, hi_c = ii.ravel() + starts[b1], jj.ravel() + starts[b2]
        pick = rng.choice(lo_c.size, int(counts[gi]), replace=False)
        dense_keys.append(lo_c[pick].astype(np.int64) * n + hi_c[pick].astype(np.int64))
    if dense_keys:
        keys = _sorted_unique(np.concatenate(dense_keys))
    need = np.where(dense, 0, counts)
    for _ in range(64):
        if need.sum() == 0:
            break
        g = np.repeat(np.arange(bi.size), need)
        a = starts[bi[g]] + rng.integers(0, sizes[bi[g]])
        b = starts[bj[g]] + rng.integers(0, sizes[bj[g]])
        ok = a != b
        lo = np.minimum(a, b)[ok]
        hi = np.maximum(a, b)[ok]
        keys = _sorted_unique(np.concatenate([keys, lo * n + hi]))
        lo_all = keys // n
        hi_all = keys % n
        have = np.bincount(group_of[block_of[lo_all], block_of[hi_all]], minlength=bi.size)
        need = np.where(dense, 0, counts - have)
        assert (need >= 0).all()
    else:
        raise RuntimeError("SBM sampler did not converge")
    labels = block_of.astype(np.int32)
    return from_edges(n, keys // n, keys % n, None, labels, name,
                      {"sizes": sizes.tolist(), "p_in": p_in, "p_out": p_out, "seed": seed})


def equal_sizes(n: int, k: int):
    """k blocks covering n vertices; the first n mod k blocks get one extra vertex."""
    base, extra = divmod(n, k)
    return [base + (1 if i < extra else 0) for i in range(k)]


def sbm_by_degree(n: int, k: int, deg_in: float, deg_out: float, seed: int, name: str = "sbm") -> Graph:
    """SBM with k near-equal blocks and expected within/cross-block degrees.

    p_in = deg_in / (s - 1) and p_out = deg_out / (n - s) with s = n / k.
    """
    s = n / k
    p_in = min(1.0, deg_in / (s - 1))
    p_out = min(1.0, deg_out / (n - s)) if k > 1 else 0.0
    g = sbm(equal_sizes(n, k), p_in, p_out, seed, name)
    g.meta.update({"deg_in": deg_in, "deg_out": deg_out})
    return g


def disjoint_cliques(k: int, s: int, name: str = "cliques") -> Graph:
    """Disjoint union of k complete graphs K_s (unit weights)."""
    iu, ju = np.triu_indices(s, 1)
    u = np.concatenate([iu + b * s for b in range(k)])
    v = np.concatenate([ju + b * s for b in range(k)])
    labels = np.repeat(np.arange(k), s)
    return from_edges(k * s, u, v, None, labels, name, {"k": k, "s": s})


def cycle(n: int) -> Graph:
    """Cycle C_n (unit weights), n >= 3."""
    u = np.arange(n)
    v = (u + 1) % n
    return from_edges(n, np.minimum(u, v), np.maximum(u, v), None, None, "cycle")


def complete(n: int) -> Graph:
    """Complete graph K_n (unit weights)."""
    iu, ju = np.triu_indices(n, 1)
    return from_edges(n, iu, ju, None, None, "complete")


def with_isolated(g: Graph, extra: int) -> Graph:
    """Append ``extra`` isolated vertices (label -1 is not used: they get label 0)."""
    n = g.n + extra
    row_ptr = np.concatenate([g.row_ptr, np.full(extra, g.row_ptr[-1], dtype=np.int64)])
    labels = None if g.labels is None else np.concatenate([g.labels, np.zeros(extra, np.int32)])
    return Graph(n, row_ptr, g.col.copy(), None if g.w is None else g.w.copy(), labels,
                 g.name + f"+{extra}iso", dict(g.meta))


def permuted(g: Graph, seed: int) -> Graph:
    """The same graph with vertex ids relabelled by a seeded random permutation."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(g.n)                  # new id of old vertex i
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    keep = rows < g.col
    u = perm[rows[keep]]
    v = perm[g.col[keep].astype(np.int64)]
    w = None if g.w is None else g.w[keep]
    labels = None
    if g.labels is not None:
        labels = np.empty_like(g.labels)
        labels[perm] = g.labels
    return from_edges(g.n, u, v, w, labels, g.name + "-perm", dict(g.meta))


def _weighted_edges(n, u, v, w64, labels, name, meta):
    w32 = w64.astype(np.float32)
    keep = w32 > 0
    return from_edges(n, u[keep], v[keep], w32[keep], labels, name, meta)


def mixture_points(npts: int, dim: int, ncomp: int, seed: int):
    """The points of knn_mixture: ``ncomp`` equally likely unit-variance Gaussian components with
    means drawn from N(0, 4 I).  Returns (points float64 npts x dim, component labels)."""
    rng = np.random.default_rng(seed)
    means = rng.normal(0.0, 2.0, size=(ncomp, dim))
    labels = rng.integers(0, ncomp, size=npts)
    x = means[labels] + rng.normal(0.0, 1.0, size=(npts, dim))
    return x, labels


def knn_mixture(npts: int, dim: int, ncomp: int, knn: int, seed: int, device: str = "cpu",
                name: str = "knn") -> Graph:
    """k-nearest-neighbour graph of a Gaussian mixture (the Sec. 4.2 pre-processing).

    Points: ``ncomp`` equally likely isotropic unit-variance components with
    means drawn from N(0, 4 I).  Each point is joined to its ``knn`` nearest
    neighbours; the directed lists are symmetrised by union.  The weight of
    {i, j} is exp(-||x_i - x_j||^2 / sigma^2) with sigma the median of all
    npts * knn directed neighbour distances.  ``device='cuda'`` finds the
    neighbours with torch on the GPU (for large point sets); the weights are
    always computed in float64 on the host.
    """
    x, labels = mixture_points(npts, dim, ncomp, seed)
    nbr = _knn_indices(x, knn, device)                   # npts x knn, excludes self
    d_dir = np.sqrt(((x[:, None, :] - x[nbr]) ** 2).sum(-1)) if npts * knn * dim <= 5e7 else \
        np.concatenate([np.sqrt(((x[s:s + 4096, None, :] - x[nbr[s:s + 4096]]) ** 2).sum(-1))
                        for s in range(0, npts, 4096)])
    sigma = float(np.median(d_dir))
    a = np.repeat(np.arange(npts, dtype=np.int64), knn)
    b = nbr.reshape(-1).astype(np.int64)
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    key = _sorted_unique(lo * npts + hi)
    lo = key // npts
    hi = key % npts
    d2 = ((x[lo] - x[hi]) ** 2).sum(-1)
    w64 = np.exp(-d2 / sigma ** 2)
    return _weighted_edges(npts, lo, hi, w64, labels.astype(np.int32), name,
                           {"npts": npts, "dim": dim, "ncomp": ncomp, "knn": knn, "sigma": sigma,
                            "seed": seed})


def _knn_indices(x: np.ndarray, knn: int, device: str) -> np.ndarray:
    npts = x.shape[0]
    if device != "cpu":
        import torch
        xt = torch.as_tensor(x, dtype=torch.float32, device=device)
        sq = (xt * xt).sum(1)
        out = torch.empty((npts, knn), dtype=torch.int64, device=device)
        for s in range(0, npts, 2048):
            blk = xt[s:s + 2048]
            d = sq[s:s + 2048, None] + sq[None, :] - 2.0 * (blk @ xt.T)
            idx = torch.arange(s, min(s + 2048, npts), device=device)
            d[idx - s, idx] = float("inf")
            out[s:s + 2048] = torch.topk(d, knn, dim=1, largest=False).indices
        return out.cpu().numpy()
    sq = (x * x).sum(1)
    out = np.empty((npts, knn), dtype=np.int64)
    for s in range(0, npts, 512):
        blk = x[s:s + 512]
        d = sq[s:s + 512, None] + sq[None, :] - 2.0 * (blk @ x.T)
        r = np.arange(blk.shape[0])
        d[r, r + s] = np.inf
        part = np.argpartition(d, knn, axis=1)[:, :knn]
        dp = np.take_along_axis(d, part, 1)
        order = np.argsort(dp, axis=1, kind="stable")
        out[s:s + 512] = np.take_along_axis(part, order, 1)
    return out


def image_grid(height: int = 321, width: int = 481, nsites: int = 8, noise: float = 0.05,
               radius: float = 3.0, seed: int = 0, name: str = "image") -> Graph:
    """Pixel graph of a synthetic image of ``nsites`` Voronoi regions.

    Each region has a uniform random RGB colour; every pixel adds N(0, noise^2)
    per channel.  Vertices are pixels in raster order; pixels within Euclidean
    distance ``radius`` are joined with weight
    exp(-||d_rgb||^2 / 0.01) * exp(-||d_xy||^2 / radius^2).
    Planted labels are the Voronoi regions.
    """
    rng = np.random.default_rng(seed)
    sites = np.stack([rng.uniform(0, height, nsites), rng.uniform(0, width, nsites)], 1)
    colours = rng.uniform(0.0, 1.0, size=(nsites, 3))
    yy, xx = np.meshgrid(np.arange(height), np.arange(width), indexing="ij")
    pix = np.stack([yy.ravel(), xx.ravel()], 1).astype(np.float64)
    d2 = ((pix[:, None, :] - sites[None, :, :]) ** 2).sum(-1)
    region = d2.argmin(1)
    rgb = colours[region] + rng.normal(0.0, noise, size=(height * width, 3))
    n = height * width
    r = int(np.floor(radius))
    us, vs, ws = [], [], []
    for dy in range(0, r + 1):
        for dx in range(-r, r + 1):
            if dy == 0 and dx <= 0:
                continue                      # each unordered offset once
            dist2 = dy * dy + dx * dx
            if dist2 > radius * radius:
                continue
            y0 = np.arange(height - dy)
            x0 = np.arange(max(0, -dx), min(width, width - dx))
            Y, X = np.meshgrid(y0, x0, indexing="ij")
            a = (Y * width + X).ravel()
            b = ((Y + dy) * width + (X + dx)).ravel()
            drgb = ((rgb[a] - rgb[b]) ** 2).sum(1)
            ws.append(np.exp(-drgb / 0.01) * np.exp(-dist2 / radius ** 2))
            us.append(a)
            vs.append(b)
    u = np.concatenate(us).astype(np.int64)
    v = np.concatenate(vs).astype(np.int64)
    w64 = np.concatenate(ws)
    lo = np.minimum(u, v)
    hi = np.maximum(u, v)
    return _weighted_edges(n, lo, hi, w64, region.astype(np.int32), name,
                           {"height": height, "width": width, "nsites": nsites, "noise": noise,
                            "radius": radius, "seed": seed})


@dataclass
class GraphBatch:
    """Disjoint union of graphs as one CSR with global vertex ids."""
    vertex_offset: np.ndarray    # int64, G + 1
    row_ptr: np.ndarray          # int64, total vertices + 1
    col: np.ndarray              # int32, global ids
    w: np.ndarray | None
    labels: np.ndarray           # planted labels (local ids)
    k: np.ndarray                # int32 planted clusters per graph
    graphs: list                 # the member Graph objects (kept for per-graph checks), or None

    @property
    def num_graphs(self) -> int:
        return int(self.k.size)

    def member(self, g: int) -> Graph:
        """Graph g alone (local vertex ids), as host numpy arrays."""
        if self.graphs is not None:
            return self.graphs[g]
        lo, hi = int(self.vertex_offset[g]), int(self.vertex_offset[g + 1])
        rp = _host(self.row_ptr[lo:hi + 1])
        e0, e1 = int(rp[0]), int(rp[-1])
        col = (_host(self.col[e0:e1]).astype(np.int64) - lo).astype(np.int32)
        w = None if self.w is None else _host(self.w[e0:e1])
        return Graph(hi - lo, (rp - e0).astype(np.int64), col, w, _host(self.labels[lo:hi]).astype(np.int32),
                     f"member{g}")


def union(graphs, with_weights: bool = False) -> GraphBatch:
    """Concatenate graphs into one block-diagonal CSR (global vertex and edge ids)."""
    ns = np.array([g.n for g in graphs], dtype=np.int64)
    voff = np.zeros(len(graphs) + 1, dtype=np.int64)
    np.cumsum(ns, out=voff[1:])
    nnz = np.array([g.nnz for g in graphs], dtype=np.int64)
    eoff = np.zeros(len(graphs) + 1, dtype=np.int64)
    np.cumsum(nnz, out=eoff[1:])
    row_ptr = np.concatenate([g.row_ptr[:-1] + eoff[i] for i, g in enumerate(graphs)] + [eoff[-1:]])
    col = np.concatenate([g.col.astype(np.int64) + voff[i] for i, g in enumerate(graphs)]).astype(np.int32)
    w = None
    if with_weights or any(g.w is not None for g in graphs):
        w = np.concatenate([g.w if g.w is not None else np.ones(g.nnz, np.float32) for g in graphs])
    labels = np.concatenate([g.labels for g in graphs]).astype(np.int32)
    k = np.array([g.k_planted for g in graphs], dtype=np.int32)
    return GraphBatch(voff, row_ptr.astype(np.int64), col, w, labels, k, list(graphs))


def sbm_batch(num_graphs: int, n_range, k_range, deg_in: float, deg_out: float, seed: int,
              with_weights: bool = False) -> GraphBatch:
    """Many SBMs: n ~ U[n_range], k ~ U[k_range] per graph (seeded), expected degrees given."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_range[0], n_range[1] + 1, num_graphs)
    ks = rng.integers(k_range[0], k_range[1] + 1, num_graphs)
    graphs = [sbm_by_degree(int(n), int(k), deg_in, deg_out, seed=int(seed * 100003 + i)) for i, (n, k) in
              enumerate(zip(ns, ks))]
    return union(graphs, with_weights)


def _host(a):
    return a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a)


def sbm_batch_gpu(num_graphs: int, n_range, k_range, deg_in: float, deg_out: float, seed: int,
                  with_weights: bool = True, device: str = "cuda") -> GraphBatch:
    """Large batches of SBM-like graphs generated on the GPU with torch (input plumbing only).

    Per graph: n ~ U[n_range], k ~ U[k_range] (numpy, seeded) and k near-equal blocks.  The
    number of within-block edges is Poisson(deg_in * n / 2), of cross-block edges
    Poisson(deg_out * n / 2); each edge has a uniform first endpoint and a uniform second
    endpoint in (respectively outside) its block; repeated pairs are dropped.  This is the SBM
    of the same expected degrees up to the dropped repeats (a vanishing fraction at these
    densities).  Row pointers, columns (global ids) and weights (all 1.0 if ``with_weights``)
    stay on the device as torch tensors.
    """
    import torch
    rng = np.random.default_rng(seed)
    G = num_graphs
    ns = rng.integers(n_range[0], n_range[1] + 1, G).astype(np.int64)
    ks = rng.integers(k_range[0], k_range[1] + 1, G).astype(np.int64)
    m_in = rng.poisson(deg_in * ns / 2.0).astype(np.int64)
    m_out = rng.poisson(deg_out * ns / 2.0).astype(np.int64)
    voff = np.zeros(G + 1, dtype=np.int64)
    np.cumsum(ns, out=voff[1:])
    NV = int(voff[-1])
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    dev = torch.device(device)
    t_ns = torch.as_tensor(ns, device=dev)
    t_ks = torch.as_tensor(ks, device=dev)
    t_voff = torch.as_tensor(voff, device=dev)

    def blocks(g, u):                       # block id, start and size of local vertex u of graph g
        n, k = t_ns[g], t_ks[g]
        base, extra = n // k, n % k
        big = extra * (base + 1)
        b = torch.where(u < big, u // (base + 1), extra + (u - big) // torch.clamp(base, min=1))
        start = torch.where(b < extra, b * (base + 1), big + (b - extra) * base)
        size = base + (b < extra).to(torch.int64)
        return b, start, size

    keys = []
    for counts, inside in ((m_in, True), (m_out, False)):
        g = torch.repeat_interleave(torch.arange(G, device=dev), torch.as_tensor(counts, device=dev))
        n = t_ns[g]
        u = torch.floor(torch.rand(g.numel(), generator=gen, device=dev, dtype=torch.float64) * n).to(torch.int64)
        _, start, size = blocks(g, u)
        r = torch.rand(g.numel(), generator=gen, device=dev, dtype=torch.float64)
        if inside:
            v = start + torch.floor(r * (size - 1)).to(torch.int64)
            v = v + (v >= u).to(torch.int64)
        else:
            v = torch.floor(r * (n - size)).to(torch.int64)
            v = v + (v >= start).to(torch.int64) * size
        off = t_voff[g]
        a, c = u + off, v + off
        keys.append(torch.minimum(a, c) * NV + torch.maximum(a, c))
        del g, n, u, start, size, r, v, off, a, c
    key = torch.unique(torch.cat(keys))
    del keys
    lo, hi = key // NV, key % NV
    del key
    rows = torch.cat([lo, hi])
    cols = torch.cat([hi, lo])
    del lo, hi
    order = torch.argsort(rows * NV + cols)
    rows, cols = rows[order], cols[order].to(torch.int32)
    del order
    counts = torch.bincount(rows, minlength=NV)
    del rows
    row_ptr = torch.zeros(NV + 1, dtype=torch.int64, device=dev)
    row_ptr[1:] = torch.cumsum(counts, 0)
    w = torch.ones(cols.numel(), dtype=torch.float32, device=dev) if with_weights else None
    gv = torch.repeat_interleave(torch.arange(G, device=dev), t_ns)
    local = torch.arange(NV, device=dev) - t_voff[gv]
    labels, _, _ = blocks(gv, local)
    return GraphBatch(voff, row_ptr, cols, w, labels.to(torch.int32), ks.astype(np.int32), None)
