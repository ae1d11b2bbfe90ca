"""GPU parity of k-means++ seeding and Lloyd iterations (Sec. 2.2).

Both sides take the same float32 point set (produced by the oracle or a seeded
mixture, never by the CUDA path).  k-means++ picks must be identical (the
float64 prefix sums differ only by summation order, far below the gap between
consecutive prefixes in these cases; a pick within 1e-12 relative of a
boundary would be reported by the check below).  Lloyd labels must be
identical except for points whose oracle nearest/second-nearest margin is
below 1e-6 relative; inertia agrees to 1e-6 relative.
"""
import numpy as np
import pytest

import workloads as W
from _helpers import fixed_point_scales as _fixed_point_scales
from _helpers import near_boundary as _near_boundary
from _helpers import oracle_embedding_f32, require_cuda
from oracle import kmeans as km
from oracle import metrics
from oracle.rng import kmeanspp_uniform

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def _mixture(n, k, l, seed, spread=0.4, lp=None):
    rng = np.random.default_rng(seed)
    centres = rng.normal(0, 3, size=(k, l))
    lab = rng.integers(0, k, n)
    X = (centres[lab] + rng.normal(0, spread, size=(n, l))).astype(np.float32)
    lp = lp or l
    out = np.zeros((n, lp), dtype=np.float32)
    out[:, :l] = X
    return out, lab


def _compare(torch, X, l, k, seed, max_iter=100):
    import paper_2310_10939_gb300 as fsc
    n, lp = X.shape
    Xt = torch.as_tensor(X, device="cuda")
    labels, st, cen, sd = fsc.kmeans(Xt, l, k, seed, max_iter, want_centroids=True, want_seeds=True)
    labels = labels.cpu().numpy()
    sd = sd.cpu().numpy()
    ref = km.kmeans(X[:, :l], k, seed, max_iter)
    if not np.array_equal(sd, ref["seeds"]):
        assert _near_boundary(X[:, :l], k, seed, ref["seeds"]), (sd, ref["seeds"])
        return None
    margin = km.relative_margin(ref["best"], ref["second"])
    diff = labels != ref["labels"]
    assert not (diff & (margin >= 1e-6)).any(), int((diff & (margin >= 1e-6)).sum())
    if not diff.any():
        assert st["iterations"] == ref["iters"]
        assert np.isclose(st["inertia"], ref["inertia"], rtol=1e-6)
        Sx, _ = _fixed_point_scales(X[:, :l], n, l)   # means of values truncated to 2^-Sx
        assert np.allclose(cen.cpu().numpy(), ref["centroids"][:, :l], rtol=1e-12, atol=2.0 ** -Sx + 1e-15)
    assert st["device_status"] == 0
    return labels, st, ref


@pytest.mark.parametrize("n,k,l,lp", [
    (1, 1, 1, 1), (2, 2, 1, 1), (7, 3, 2, 2), (511, 4, 3, 4), (513, 5, 4, 4), (1000, 4, 2, 2),
    (4099, 16, 4, 4), (20000, 10, 7, 8), (65537, 32, 5, 8), (3000, 100, 8, 8), (100000, 3, 1, 1),
    (2000, 1024, 2, 2),
])
def test_kmeans_matches_oracle_on_mixtures(torch, n, k, l, lp):
    X, _ = _mixture(n, max(1, min(k, 50)), l, seed=n + k, lp=lp)
    _compare(torch, X, l, k, seed=31 + k)


@pytest.mark.parametrize("seed", [3, 4])
def test_kmeans_several_tiles_per_block(torch, seed):
    """650,000 points: some blocks take three tiles of 2048 points, so Lloyd's per-warp queues fill
    and are worked in the middle of a pass (in the first iteration every point is queued).  With
    max_iter = 12 the run converges (seed 3) or stops with labels still changing (seed 4, where
    the inertia is that of the last assignment, taken with the centroids it used)."""
    X, _ = _mixture(650_000, 12, 4, seed=650_000 + seed, spread=0.3)
    _compare(torch, X, 4, 12, seed=43 + seed, max_iter=12)


@pytest.mark.parametrize("seed", range(1, 6))
def test_kmeans_on_oracle_embedding_of_sbm(torch, seed):
    g = W.sbm([250] * 4, 0.1, 0.002, seed)
    _, X = oracle_embedding_f32(g, 2, 20, seed, 2)
    out = _compare(torch, X, 2, 4, seed)
    if out is not None:
        labels, st, ref = out
        assert abs(metrics.ari(labels, g.labels) - metrics.ari(ref["labels"], g.labels)) <= 0.01


def test_kmeans_pad_columns_are_ignored(torch):
    import paper_2310_10939_gb300 as fsc
    X, _ = _mixture(3000, 6, 3, seed=4, lp=4)
    Y = X.copy()
    Y[:, 3] = np.random.default_rng(0).normal(size=3000)     # garbage in the pad column
    a = fsc.kmeans(torch.as_tensor(X, device="cuda"), 3, 6, 9)[0]
    b = fsc.kmeans(torch.as_tensor(Y, device="cuda"), 3, 6, 9)[0]
    assert torch.equal(a, b)


def test_kmeans_degenerate_identical_points(torch):
    import paper_2310_10939_gb300 as fsc
    X = np.zeros((600, 2), dtype=np.float32)
    labels, st, cen, sd = fsc.kmeans(torch.as_tensor(X, device="cuda"), 2, 5, 3, want_seeds=True)
    first = int(np.floor(kmeanspp_uniform(3, 0) * 600))
    assert sd.cpu().tolist() == [first] + [i for i in range(600) if i != first][:4]
    assert (labels.cpu().numpy() == 0).all()
    assert st["empty_events"] >= 4
    ref = km.kmeans(X, 5, 3)
    assert np.array_equal(labels.cpu().numpy(), ref["labels"])


def test_kmeans_duplicates_and_ties(torch):
    """Many exact ties: points equidistant from two centroids go to the lower index on both sides."""
    rng = np.random.default_rng(5)
    base = rng.integers(-3, 4, size=(40, 2)).astype(np.float32)
    X = base[rng.integers(0, 40, 5000)]
    _compare(torch, X, 2, 7, seed=12)


def test_kmeans_max_iter_respected(torch):
    import paper_2310_10939_gb300 as fsc
    X, _ = _mixture(20000, 12, 4, seed=8, spread=2.5)
    labels, st, _, _ = fsc.kmeans(torch.as_tensor(X, device="cuda"), 4, 12, 2, max_iter=2)
    assert st["iterations"] == 2
    ref = km.kmeans(X, 12, 2, max_iter=2)
    margin = km.relative_margin(ref["best"], ref["second"])
    diff = labels.cpu().numpy() != ref["labels"]
    assert not (diff & (margin >= 1e-6)).any()


def test_kmeans_invalid_arguments(torch):
    import paper_2310_10939_gb300 as fsc
    X = torch.zeros((10, 4), dtype=torch.float32, device="cuda")
    for l, k in [(0, 2), (5, 2), (2, 0), (2, 11)]:
        with pytest.raises(fsc.FscError):
            fsc.kmeans(X, l, k, 0)


def test_wait_limit_timeout_is_reported_and_recoverable(torch):
    """A grid-barrier wait that runs out (a barrier nothing releases) returns FSC_ERR_TIMEOUT,
    with no trap; the context stays usable and the next call succeeds."""
    import paper_2310_10939_gb300 as fsc
    X, _ = _mixture(400000, 8, 4, seed=9)
    Xt = torch.as_tensor(X, device="cuda")
    fsc.set_wait_limit_ns(5_000_000)
    fsc.inject_barrier_stall(True)
    try:
        with pytest.raises(fsc.FscError) as e:
            fsc.kmeans(Xt, 4, 8, 1)
        assert e.value.name == "FSC_ERR_TIMEOUT"
        # asynchronous form: the error reaches the per-device status word
        fsc.kmeans(Xt, 4, 8, 1, sync=False)
        with pytest.raises(fsc.FscError) as e:
            fsc.sync_status()
        assert e.value.name == "FSC_ERR_TIMEOUT"
    finally:
        fsc.inject_barrier_stall(False)
        fsc.set_wait_limit_ns(2_000_000_000)
    labels, st, _, _ = fsc.kmeans(Xt, 4, 8, 1)
    assert st["device_status"] == 0
    fsc.sync_status()
    ref = km.kmeans(X, 8, 1)
    margin = km.relative_margin(ref["best"], ref["second"])
    assert not ((labels.cpu().numpy() != ref["labels"]) & (margin >= 1e-6)).any()
