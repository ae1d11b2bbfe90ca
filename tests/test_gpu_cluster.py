"""Algorithm 2 end to end on the GPU against the oracle, at the small SBM size and at full scale.

Bar: embedding relative Frobenius error <= 1e-5 (float32) / 2e-2 (bfloat16)
against float64; k-means labels equal to the oracle's on a shared float32
input except near-ties (margin < 1e-6); ARI against the planted labels within
0.01 of the oracle's.
"""
import numpy as np
import pytest

import workloads as W
from _helpers import near_boundary, rel_fro, require_cuda
from oracle import cluster as ocluster
from oracle import kmeans as km
from oracle import metrics, spectral

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


@pytest.mark.parametrize("seed", range(1, 11))
def test_cluster_sbm_n1000_k4_matches_oracle_ari(torch, seed):
    """SBM n=1000, 4 blocks of 250, p=0.1, q=0.002, l=2, t=20 (ten seeds, the paper's trial count)."""
    import paper_2310_10939_gb300 as fsc
    g = W.sbm([250] * 4, 0.1, 0.002, seed)
    G = fsc.Graph.from_workload(g)
    labels, st = fsc.cluster(G, 4, 2, 20, seed)
    ref = ocluster.fast_spectral_cluster(g, 4, 2, 20, seed)
    a_gpu = metrics.ari(labels.cpu().numpy(), g.labels)
    a_ref = metrics.ari(ref["labels"], g.labels)
    assert abs(a_gpu - a_ref) <= 0.01
    assert st["device_status"] == 0 and st["changed"] == 0


def _full_scale_check(torch, g, k, l, t, seed, store, emb_tol):
    import paper_2310_10939_gb300 as fsc
    G = fsc.Graph.from_workload(g)
    lp = fsc.pad_l(l)
    emb = fsc.embed(G, l, t, seed, store=store, rescale=True).cpu().numpy()
    B = spectral.embed(g, l, t, seed)
    err = rel_fro(emb[:, :l], B)
    assert err <= emb_tol, err
    # k-means parity on the oracle's float32 embedding (shared input)
    X = np.zeros((g.n, lp), dtype=np.float32)
    X[:, :l] = B.astype(np.float32)
    lab_gpu, st, _, sd = fsc.kmeans(torch.as_tensor(X, device="cuda"), l, k, seed, want_seeds=True)
    ref = km.kmeans(X[:, :l], k, seed)
    lab_gpu = lab_gpu.cpu().numpy()
    if np.array_equal(sd.cpu().numpy(), ref["seeds"]):
        margin = km.relative_margin(ref["best"], ref["second"])
        assert not ((lab_gpu != ref["labels"]) & (margin >= 1e-6)).any()
    else:
        # picks may part only where a draw lies within the documented error window of a boundary
        assert near_boundary(X[:, :l], k, seed, ref["seeds"]), (sd.cpu().numpy(), ref["seeds"])
    # the whole GPU pipeline against the oracle pipeline: ARI within 0.01
    labels, st = fsc.cluster(G, k, l, t, seed, store=store, rescale=True)
    a_gpu = metrics.ari(labels.cpu().numpy(), g.labels)
    a_ref = metrics.ari(ref["labels"], g.labels)
    assert abs(a_gpu - a_ref) <= 0.01, (a_gpu, a_ref)
    return a_gpu, a_ref, err


def test_full_scale_sbm_2pow20_k16(torch):
    """SBM n=2^20, 16 equal blocks, expected intra-degree 20, inter-degree 2, l=4, t=20, float32."""
    g = W.sbm_by_degree(2 ** 20, 16, 20.0, 2.0, seed=7)
    a_gpu, a_ref, _ = _full_scale_check(torch, g, 16, 4, 20, 7, 0, 1e-5)
    assert a_ref >= 0.9


def test_full_scale_knn_mixture(torch):
    """200,000 points in R^32, 10-component mixture, 10-NN graph, k=10, l=4, t=20, float32."""
    g = W.knn_mixture(200_000, 32, 10, 10, seed=5, device="cuda")
    _full_scale_check(torch, g, 10, 4, 20, 5, 0, 1e-5)


def test_full_scale_image_grid_bf16_and_f32(torch):
    """481x321 Voronoi image graph, radius 3, k=8, l=3, t=30: bfloat16 and float32 storage."""
    import paper_2310_10939_gb300 as fsc
    g = W.image_grid(321, 481, 8, seed=3)
    a32, aref, _ = _full_scale_check(torch, g, 8, 3, 30, 3, fsc.F32, 1e-5)
    G = fsc.Graph.from_workload(g)
    emb = fsc.embed(G, 3, 30, 3, store=fsc.BF16, rescale=True).cpu().numpy()
    assert rel_fro(emb[:, :3], spectral.embed(g, 3, 30, 3)) <= 2e-2
    labels, _ = fsc.cluster(G, 8, 3, 30, 3, store=fsc.BF16, rescale=True)
    a16 = metrics.ari(labels.cpu().numpy(), g.labels)
    assert abs(a16 - a32) <= 0.01, (a16, a32)
