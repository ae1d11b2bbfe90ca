"""Batched Algorithm 2 (one persistent launch over many graphs) against per-graph runs and the oracle.

Per graph, the batch must give exactly the labels of fsc_cluster with the same parameters
and lanes per row (same per-row arithmetic, exact integer k-means sums); against the float64
oracle the bar is the usual one: ARI within 0.01 of the oracle's on the same graph.
"""
import numpy as np
import pytest

import workloads as W
from _helpers import require_cuda
from oracle import cluster as ocluster
from oracle import metrics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def _batch(torch, gb, store, **kw):
    import paper_2310_10939_gb300 as fsc
    rp = torch.as_tensor(gb.row_ptr, device="cuda")
    col = torch.as_tensor(gb.col, device="cuda")
    w = None if gb.w is None else torch.as_tensor(gb.w, device="cuda")
    seeds = np.arange(gb.num_graphs, dtype=np.uint64) * 7 + 3
    b = fsc.Batch(gb.vertex_offset, rp, col, gb.k, seeds, w=w, store=store, **kw)
    return b, seeds


@pytest.mark.parametrize("store_name", ["bf16", "f32"])
@pytest.mark.parametrize("weighted", [True, False])
def test_batch_equals_per_graph_cluster(torch, store_name, weighted):
    import paper_2310_10939_gb300 as fsc
    store = fsc.BF16 if store_name == "bf16" else fsc.F32
    gb = W.sbm_batch(24, (300, 6000), (2, 20), 15.0, 1.5, seed=11, with_weights=weighted)
    b, seeds = _batch(torch, gb, store)
    labels = b.run().cpu().numpy()
    stats, picks, cents = b.results()
    for g in range(gb.num_graphs):
        m = gb.member(g)
        lo, hi = gb.vertex_offset[g], gb.vertex_offset[g + 1]
        wt = None if gb.w is None else torch.as_tensor(gb.w[gb.row_ptr[lo]:gb.row_ptr[hi]], device="cuda")
        G = fsc.Graph(torch.as_tensor(m.row_ptr, device="cuda"), torch.as_tensor(m.col, device="cuda"), wt)
        l, t = fsc.default_params(m.n, int(gb.k[g]))
        ref, st = fsc.cluster(G, int(gb.k[g]), l, t, int(seeds[g]), store=store, rescale=True, threads_per_row=4)
        assert np.array_equal(labels[lo:hi], ref.cpu().numpy()), g
        assert stats[g]["iterations"] == st["iterations"]
        assert np.isclose(stats[g]["inertia"], st["inertia"], rtol=1e-12)
        assert len(picks[g]) == gb.k[g] and cents[g].shape == (gb.k[g], l)
    b.close()


@pytest.mark.parametrize("store_name", ["f32", "bf16"])
def test_batch_matches_oracle_on_sampled_members(torch, store_name):
    """Embedding error per member (1e-5 f32, 2e-2 bf16) and ARI within 0.01 of the oracle's
    (every member in f32; in bf16 the members the oracle itself separates, ARI >= 0.9, and the
    k-means stage of the others on the oracle's own float32 embedding)."""
    import paper_2310_10939_gb300 as fsc
    from _helpers import rel_fro
    from oracle import spectral
    store = fsc.F32 if store_name == "f32" else fsc.BF16
    gb = W.sbm_batch(30, (500, 8000), (2, 12), 15.0, 1.5, seed=5, with_weights=True)
    b, seeds = _batch(torch, gb, store)
    labels = b.run().cpu().numpy()
    for g in range(0, gb.num_graphs, 3):
        m = gb.member(g)
        lo, hi = gb.vertex_offset[g], gb.vertex_offset[g + 1]
        l, t = fsc.default_params(m.n, int(gb.k[g]))
        emb = b.embedding(g, m.n, l).cpu().numpy()
        err = rel_fro(emb[:, :l], spectral.embed(m, l, t, int(seeds[g])))
        assert err <= (1e-5 if store == fsc.F32 else 2e-2), (g, err)
        ref = ocluster.fast_spectral_cluster(m, int(gb.k[g]), l, t, int(seeds[g]))
        a_gpu = metrics.ari(labels[lo:hi], m.labels)
        a_ref = metrics.ari(ref["labels"], m.labels)
        if store == fsc.F32 or a_ref >= 0.9:
            assert abs(a_gpu - a_ref) <= 0.01, (g, a_gpu, a_ref)
        else:
            # a member the oracle itself separates poorly: its k-means lands in a local optimum that
            # a 2e-2 change of the points can move, so the ARI is not comparable; the k-means stage
            # is then checked on the oracle's float32 embedding, labels equal up to near-ties
            _kmeans_parity_on_oracle_embedding(torch, m, int(gb.k[g]), l, t, int(seeds[g]))
    b.close()


def _kmeans_parity_on_oracle_embedding(torch, m, k, l, t, seed):
    import paper_2310_10939_gb300 as fsc
    from _helpers import near_boundary, oracle_embedding_f32
    from oracle import kmeans as km
    _, X = oracle_embedding_f32(m, l, t, seed, fsc.pad_l(l))
    lab, _, _, sd = fsc.kmeans(torch.as_tensor(X, device="cuda"), l, k, seed, want_seeds=True)
    ref = km.kmeans(X[:, :l], k, seed)
    if not np.array_equal(sd.cpu().numpy(), ref["seeds"]):
        assert near_boundary(X[:, :l], k, seed, ref["seeds"])
        return
    margin = km.relative_margin(ref["best"], ref["second"])
    assert not ((lab.cpu().numpy() != ref["labels"]) & (margin >= 1e-6)).any()


def test_batch_edge_cases(torch):
    """Tiny and degenerate members: n = 1 (k = 1, t = 0), l = 8, isolated vertices, k = n."""
    import paper_2310_10939_gb300 as fsc
    members = [
        W.from_edges(1, [], [], labels=[0]),
        W.with_isolated(W.sbm([40, 60], 0.3, 0.02, 1), 5),
        W.disjoint_cliques(3, 9),
        W.sbm([200] * 5, 0.1, 0.005, 2),
        W.cycle(50),
    ]
    members[-1].labels = np.zeros(50, np.int32)
    gb = W.union(members)
    k = np.array([1, 2, 3, 5, 50], dtype=np.int32)
    l = np.array([1, 2, 8, 3, 1], dtype=np.int32)
    t = np.array([0, 5, 20, 12, 3], dtype=np.int32)
    rp = torch.as_tensor(gb.row_ptr, device="cuda")
    col = torch.as_tensor(gb.col, device="cuda")
    seeds = np.arange(5, dtype=np.uint64) + 100
    b = fsc.Batch(gb.vertex_offset, rp, col, k, seeds, l=l, t=t, store=fsc.F32)
    labels = b.run().cpu().numpy()
    for g, m in enumerate(members):
        lo, hi = gb.vertex_offset[g], gb.vertex_offset[g + 1]
        G = fsc.Graph(torch.as_tensor(m.row_ptr, device="cuda"), torch.as_tensor(m.col, device="cuda"))
        ref, _ = fsc.cluster(G, int(k[g]), int(l[g]), int(t[g]), int(seeds[g]), threads_per_row=4, rescale=True)
        assert np.array_equal(labels[lo:hi], ref.cpu().numpy()), g
    assert metrics.ari(labels[gb.vertex_offset[2]:gb.vertex_offset[3]], members[2].labels) == 1.0
    b.close()


def test_batch_rejects_cross_graph_edges(torch):
    import paper_2310_10939_gb300 as fsc
    gb = W.sbm_batch(3, (100, 200), (2, 3), 10.0, 1.0, seed=2)
    col = gb.col.copy()
    col[0] = gb.vertex_offset[2]              # an edge of graph 0 into graph 2
    with pytest.raises(fsc.FscError) as e:
        fsc.Batch(gb.vertex_offset, torch.as_tensor(gb.row_ptr, device="cuda"), torch.as_tensor(col, device="cuda"),
                  gb.k, np.ones(3, np.uint64))
    assert e.value.name == "FSC_ERR_INDEX_RANGE"


def test_autotune_then_batch(torch):
    """The autotuner picks a lane count; batches built with it still match their members' results."""
    import paper_2310_10939_gb300 as fsc
    g = W.sbm_by_degree(200_000, 8, 15.0, 1.5, seed=4)
    G = fsc.Graph.from_workload(g)
    best, us = fsc.autotune(G, 3, fsc.BF16)
    assert best in (4, 8, 16, 32) and us > 0
    gb = W.sbm_batch(8, (1000, 4000), (5, 8), 15.0, 1.5, seed=9)
    b, seeds = _batch(torch, gb, fsc.BF16, autotune=True)
    labels = b.run().cpu().numpy()
    stats, _, _ = b.results()
    assert all(s["iterations"] >= 1 for s in stats)
    for q in range(gb.num_graphs):
        lo, hi = gb.vertex_offset[q], gb.vertex_offset[q + 1]
        assert labels[lo:hi].min() >= 0 and labels[lo:hi].max() < gb.k[q]
    b.close()


def test_full_scale_batch_4096_sampled(torch):
    """The full batch (4096 SBMs, n ~ U[500, 50000], k ~ U[2, 20], degrees 15 / 1.5, bf16 iterates,
    float32 weights) in one plan; sampled members against per-graph fsc_cluster (exact) and the
    oracle (embedding within 2e-2; ARI within 0.01 where the oracle separates the graph)."""
    import paper_2310_10939_gb300 as fsc
    from _helpers import rel_fro
    from oracle import spectral
    gb = W.sbm_batch_gpu(4096, (500, 50_000), (2, 20), 15.0, 1.5, seed=13)
    seeds = np.arange(gb.num_graphs, dtype=np.uint64) + 1
    b = fsc.Batch(gb.vertex_offset, gb.row_ptr, gb.col, gb.k, seeds, w=gb.w, store=fsc.BF16)
    labels = b.run().cpu().numpy()
    stats, _, _ = b.results()
    assert all(1 <= s["iterations"] <= 100 for s in stats)
    rng = np.random.default_rng(0)
    for i, g in enumerate(rng.choice(gb.num_graphs, 6, replace=False)):
        m = gb.member(int(g))
        lo, hi = gb.vertex_offset[g], gb.vertex_offset[g + 1]
        l, t = fsc.default_params(m.n, int(gb.k[g]))
        G = fsc.Graph(torch.as_tensor(m.row_ptr, device="cuda"), torch.as_tensor(m.col, device="cuda"),
                      torch.as_tensor(m.w, device="cuda"))
        ref, _ = fsc.cluster(G, int(gb.k[g]), l, t, int(seeds[g]), store=fsc.BF16, rescale=True, threads_per_row=4)
        assert np.array_equal(labels[lo:hi], ref.cpu().numpy()), g
        # every sampled member's embedding against the oracle, whatever its clustering quality
        emb = b.embedding(int(g), m.n, l).cpu().numpy()
        assert rel_fro(emb[:, :l], spectral.embed(m, l, t, int(seeds[g]))) <= 2e-2, g
        if i < 2:
            oref = ocluster.fast_spectral_cluster(m, int(gb.k[g]), l, t, int(seeds[g]))
            a_ref = metrics.ari(oref["labels"], m.labels)
            if a_ref >= 0.9:
                assert abs(metrics.ari(labels[lo:hi], m.labels) - a_ref) <= 0.01
            else:
                _kmeans_parity_on_oracle_embedding(torch, m, int(gb.k[g]), l, t, int(seeds[g]))
    b.close()
