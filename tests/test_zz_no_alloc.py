"""fsc_kmeans_static: k-means without device allocation, checked against fsc_kmeans.

Some callers cannot allocate device memory once they are running (a runtime that
reserves a fixed memory budget up front, or a latency-critical loop where an
allocation could block or fail).  fsc_kmeans_static serves them from one fixed
scratch array compiled into the library.  These tests call both entry points
through the C ABI on the same inputs, two problems in a row (the shared array
keeps the previous call's contents), and expect the same labels, k-means++ picks
and centroids; the labels must also match the float64 oracle up to near-ties.
This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from _helpers import require_cuda
from oracle import kmeans as km

pytestmark = pytest.mark.gpu


def _mixture(n, k, l, seed, lp):
    rng = np.random.default_rng(seed)
    centres = rng.normal(0, 3, size=(k, l))
    X = np.zeros((n, lp), dtype=np.float32)
    X[:, :l] = centres[rng.integers(0, k, n)] + rng.normal(0, 0.4, size=(n, l))
    return X


def _call(fn, torch, Xt, l, k, seed):
    import paper_2310_10939_gb300 as fsc
    n, ld = Xt.shape
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    cen = torch.empty((k, l), dtype=torch.float64, device="cuda")
    seeds = torch.empty(k, dtype=torch.int64, device="cuda")
    st = fsc.KmeansStats()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(C.c_void_p(Xt.data_ptr()), n, l, ld, k, seed, 100, C.c_void_p(labels.data_ptr()),
            C.c_void_p(cen.data_ptr()), C.c_void_p(seeds.data_ptr()), C.byref(st), stream)
    torch.cuda.synchronize()
    return rc, labels.cpu().numpy(), cen.cpu().numpy(), seeds.cpu().numpy(), st


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def test_static_kmeans_matches_allocating_kmeans_twice(torch):
    import paper_2310_10939_gb300 as fsc
    L = fsc.lib()
    problems = [(200_000, 12, 4, 4, 5), (70_001, 5, 3, 4, 9)]   # (n, k, l, ld, seed); the second is smaller
    for n, k, l, ld, seed in problems:
        X = _mixture(n, k, l, seed, ld)
        Xt = torch.as_tensor(X, device="cuda")
        rc_a, lab_a, cen_a, sd_a, st_a = _call(L.fsc_kmeans, torch, Xt, l, k, seed)
        rc_s, lab_s, cen_s, sd_s, st_s = _call(L.fsc_kmeans_static, torch, Xt, l, k, seed)
        assert rc_a == 0 and rc_s == 0
        assert np.array_equal(sd_s, sd_a)
        assert np.array_equal(lab_s, lab_a)
        assert np.allclose(cen_s, cen_a, rtol=1e-12, atol=1e-12)
        assert st_s.iterations == st_a.iterations and st_s.device_status == 0
        ref = km.kmeans(X[:, :l], k, seed)
        margin = km.relative_margin(ref["best"], ref["second"])
        assert not ((lab_s != ref["labels"]) & (margin >= 1e-6)).any()


def test_static_kmeans_allocates_nothing_and_rejects_oversized_problems(torch):
    import paper_2310_10939_gb300 as fsc
    L = fsc.lib()
    X = _mixture(100_000, 6, 2, 3, 2)
    Xt = torch.as_tensor(X, device="cuda")
    rc, lab1, _, _, _ = _call(L.fsc_kmeans_static, torch, Xt, 2, 6, 3)      # first call: set-up
    assert rc == 0
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    rc, lab2, _, _, _ = _call(L.fsc_kmeans_static, torch, Xt, 2, 6, 3)
    free_after = torch.cuda.mem_get_info()[0]
    assert rc == 0 and np.array_equal(lab1, lab2)
    assert free_after == free_before
    big = torch.zeros((2 ** 21, 8), dtype=torch.float32, device="cuda")   # 2 x 8 MiB of D^2 alone
    rc, *_ = _call(L.fsc_kmeans_static, torch, big, 8, 64, 1)
    assert rc == 10 and fsc.status_string(rc).startswith("problem exceeds")


def test_static_kmeans_size_limit_edge(torch):
    """The limit depends on n, k and ld only: with k = 64 and ld = 8 about 16 bytes per point plus
    the per-cluster tables fit in the 16 MiB array up to about 1.04 million points."""
    import paper_2310_10939_gb300 as fsc
    L = fsc.lib()
    fits = torch.zeros((1_000_000, 8), dtype=torch.float32, device="cuda")
    rc, lab, *_ = _call(L.fsc_kmeans_static, torch, fits, 8, 64, 2)
    assert rc == 0 and (lab == 0).all()          # identical points: every label is the first centre's
    del fits
    over = torch.zeros((1_100_000, 8), dtype=torch.float32, device="cuda")
    rc, *_ = _call(L.fsc_kmeans_static, torch, over, 8, 64, 2)
    assert rc == 10


def test_static_kmeans_refuses_a_capturing_stream(torch):
    """The call waits for its stream and copies results to the host, which a capture cannot hold:
    on a capturing stream it returns FSC_ERR_INVALID_ARG and leaves the capture intact."""
    import paper_2310_10939_gb300 as fsc
    L = fsc.lib()
    Xt = torch.as_tensor(_mixture(10_000, 3, 2, 1, 2), device="cuda")
    labels = torch.empty(10_000, dtype=torch.int32, device="cuda")
    y = torch.zeros(16, device="cuda")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        y.add_(1.0)
        stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = L.fsc_kmeans_static(C.c_void_p(Xt.data_ptr()), 10_000, 2, 2, 3, 1, 100, C.c_void_p(labels.data_ptr()),
                                 None, None, None, stream)
    assert rc == 1
    graph.replay()
    torch.cuda.synchronize()
    assert float(y[0]) == 1.0
