"""Rows longer than 1024 entries (hubs) in the sparse steps: split into segments by their own
kernels, summed in segment order.  An SBM with a star centre joined to every vertex and a few hubs
of 1,500 .. 5,000 neighbours, against the float64 oracle at the usual bars (one power step 2e-6,
embedding 1e-5 float32 / 2e-2 bfloat16, filter basis 1e-5, orthogonal iteration 1e-5, ARI within
0.01), and against the same graph without its hubs for the step time."""
import time

import numpy as np
import pytest

import workloads as W
from _helpers import rel_fro, require_cuda
from oracle import cluster as ocluster
from oracle import filter as ofl
from oracle import metrics, spectral
from oracle.rng import gaussian_block

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def _hub_graph(n=20000, k=8, seed=3, weighted=False):
    base = W.sbm_by_degree(n, k, 20.0, 2.0, seed=seed)
    rows = np.repeat(np.arange(n), np.diff(base.row_ptr))
    keep = rows < base.col
    u, v = list(rows[keep]), list(base.col[keep])
    have = set(zip(u, v))
    rng = np.random.default_rng(seed)
    hubs = {0: np.arange(1, n)}                               # a star centre: degree n - 1
    for h, d in ((11, 1500), (222, 3000), (3333, 5000)):
        hubs[h] = rng.choice(np.setdiff1d(np.arange(n), [h]), d, replace=False)
    for h, nb in hubs.items():
        for j in nb:
            a, b = (h, int(j)) if h < j else (int(j), h)
            if (a, b) not in have:
                have.add((a, b))
                u.append(a)
                v.append(b)
    w = rng.uniform(0.5, 1.5, len(u)) if weighted else None
    return W.from_edges(n, np.array(u), np.array(v), w, labels=base.labels, name="sbm+hubs")


@pytest.mark.parametrize("weighted", [False, True])
def test_power_step_and_embedding_with_hubs(torch, weighted):
    import paper_2310_10939_gb300 as fsc
    g = _hub_graph(weighted=weighted)
    assert np.diff(g.row_ptr).max() == g.n - 1
    G = fsc.Graph.from_workload(g)
    lp = 4
    x0 = gaussian_block(g.n, 3, 5)
    dm = spectral.inv_sqrt_degrees(spectral.degrees(g))[:, None]
    z = np.zeros((g.n, lp), dtype=np.float32)
    z[:, :3] = dm * x0
    zin = torch.as_tensor(z, device="cuda")
    zout = torch.empty_like(zin)
    fsc.power_step(G, 3, zin, zout)
    ref = dm * (spectral.signless_laplacian(g) @ x0)
    assert rel_fro(zout.cpu().numpy()[:, :3], ref) <= 2e-6
    emb = fsc.embed(G, 3, 12, 7).cpu().numpy()[:, :3]
    assert rel_fro(emb, spectral.embed(g, 3, 12, 7)) <= 1e-5
    embb = fsc.embed(G, 3, 12, 7, store=fsc.BF16, rescale=True).cpu().numpy()[:, :3]
    assert rel_fro(embb, spectral.embed(g, 3, 12, 7)) <= 2e-2


def test_filter_and_orthogonal_iteration_with_hubs(torch):
    import paper_2310_10939_gb300 as fsc
    g = _hub_graph()
    G = fsc.Graph.from_workload(g)
    coeffs = torch.as_tensor(np.array([0.3, -0.2, 0.5, 0.1, -0.4, 0.2, 0.05, -0.1, 0.25], np.float32), device="cuda")
    emb, feats, _ = fsc.filter_embed(G, 4, 8, 9, coeffs=coeffs, store=fsc.F32)
    K = ofl.cheb_basis(g, gaussian_block(g.n, 4, 9))
    dm = spectral.inv_sqrt_degrees(spectral.degrees(g))[:, None]
    ref = dm * sum(float(c) * Kj for c, Kj in zip(coeffs.cpu().numpy(), K))
    assert rel_fro(emb.cpu().numpy()[:, :4], ref) <= 1e-5
    f_ref = ofl.features(g, 8, 4, gaussian_block(g.n, 4, 9))
    assert np.allclose(feats.cpu().numpy()[8:], f_ref[8:], rtol=1e-5, atol=1e-6)   # the moments
    orth = fsc.embed_orthogonal(G, 4, 10, 11, every=2).cpu().numpy()[:, :4].astype(np.float64)
    assert rel_fro(orth, spectral.orthogonal_iteration(g, 4, 10, 2, 11)) <= 1e-5


def test_cluster_with_hubs_matches_oracle_ari(torch):
    import paper_2310_10939_gb300 as fsc
    g = _hub_graph(seed=4)
    G = fsc.Graph.from_workload(g)
    labels, _ = fsc.cluster(G, 8, 3, 15, 4)
    ref = ocluster.fast_spectral_cluster(g, 8, 3, 15, 4)
    assert abs(metrics.ari(labels.cpu().numpy(), g.labels) - metrics.ari(ref["labels"], g.labels)) <= 0.01


def test_hubs_do_not_stall_the_step(torch):
    """A row of n - 1 entries walked by one lane group would take n / 16 dependent passes; split into
    segments the step stays within a few times the hub-free graph's."""
    import paper_2310_10939_gb300 as fsc
    n = 200_000
    base = W.sbm_by_degree(n, 8, 20.0, 2.0, seed=5)
    rows = np.repeat(np.arange(n), np.diff(base.row_ptr))
    keep = (rows < base.col) & (rows != 0)
    u = np.concatenate([rows[keep], np.zeros(n - 1, dtype=np.int64)])
    v = np.concatenate([base.col[keep], np.arange(1, n)])
    star = W.from_edges(n, u, v, labels=base.labels)

    def step_ms(g):
        G = fsc.Graph.from_workload(g)
        z = torch.randn((n, 4), device="cuda")
        out = torch.empty_like(z)
        for _ in range(3):
            fsc.power_step(G, 4, z, out)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(10):
            fsc.power_step(G, 4, z, out)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 100.0

    t_star, t_base = step_ms(star), step_ms(base)
    assert t_star <= 5.0 * t_base + 0.05, (t_star, t_base)
