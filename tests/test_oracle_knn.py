"""Pins of the oracle's kNN-graph construction (the Sec. 4.2 pre-processing)."""
import numpy as np
import pytest

from oracle import knn as ok


def _points(n, dim, seed):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=(n, dim)) * 3 + rng.normal(size=(1, dim))).astype(np.float32)


def test_neighbours_match_a_library_search():
    nb = pytest.importorskip("sklearn.neighbors")
    X = _points(400, 6, 1)
    idx, dd = ok.neighbours(X, 10)
    ref = nb.NearestNeighbors(n_neighbors=11, algorithm="brute").fit(X.astype(np.float64))
    d_ref, i_ref = ref.kneighbors(X.astype(np.float64))
    # drop self (distance 0) from the library's lists
    i_ref = np.array([[j for j in row if j != i][:10] for i, row in enumerate(i_ref)])
    assert np.array_equal(np.sort(idx, 1), np.sort(i_ref, 1))
    assert np.allclose(np.sqrt(dd), d_ref[:, 1:], rtol=1e-5)


def test_ties_go_to_the_lower_index_and_self_is_excluded():
    X = np.array([[0, 0], [1, 0], [-1, 0], [0, 1], [0, -1], [5, 5]], dtype=np.float32)
    idx, dd = ok.neighbours(X, 3)
    assert list(idx[0]) == [1, 2, 3]               # four points at distance 1: the three lowest ids
    assert all(i not in idx[i] for i in range(len(X)))


def test_graph_is_the_symmetric_union_with_median_sigma():
    nb = pytest.importorskip("sklearn.neighbors")
    X = _points(300, 5, 2)
    row_ptr, col, w, sigma, idx, dd = ok.knn_graph(X, 7)
    n = X.shape[0]
    edges = {(i, int(j)) for i in range(n) for j in col[row_ptr[i]:row_ptr[i + 1]]}
    assert all((j, i) in edges for (i, j) in edges)                       # symmetric
    assert all((i, int(j)) in edges for i in range(n) for j in idx[i])    # contains every list
    assert len(edges) == len({(i, int(j)) for i in range(n) for j in idx[i]} |
                             {(int(j), i) for i in range(n) for j in idx[i]})
    assert all(np.all(np.diff(col[row_ptr[i]:row_ptr[i + 1]]) > 0) for i in range(n))
    d_ref = nb.NearestNeighbors(n_neighbors=7, algorithm="brute").fit(X.astype(np.float64)).kneighbors()[0]
    assert abs(sigma - float(np.median(d_ref))) <= 1e-5 * sigma
    W = {(i, int(j)): w[p] for i in range(n) for p, j in zip(range(row_ptr[i], row_ptr[i + 1]),
                                                              col[row_ptr[i]:row_ptr[i + 1]])}
    assert all(abs(W[(i, j)] - W[(j, i)]) <= 1e-12 for (i, j) in edges)
    assert all(0.0 < v <= 1.0 for v in w)


def test_weights_on_a_hand_worked_line():
    """Points 0, 1, 3, 7 on a line, one neighbour each: directed distances 1, 1, 2, 4, so
    sigma = (1 + 2) / 2 = 1.5 (median of an even count); edges {0,1}, {1,2}, {2,3} at distances
    1, 2, 4 weigh exp(-1/2.25), exp(-4/2.25), exp(-16/2.25).  A slip such as exp(-d^2/sigma),
    exp(-d^2/(2 sigma^2)) or exp(-d/sigma^2) fails here."""
    X = np.array([[0.0], [1.0], [3.0], [7.0]], dtype=np.float32)
    row_ptr, col, w, sigma, idx, _ = ok.knn_graph(X, 1)
    assert list(idx[:, 0]) == [1, 0, 1, 2]
    assert sigma == 1.5
    assert list(row_ptr) == [0, 1, 3, 5, 6]
    assert list(col) == [1, 0, 2, 1, 3, 2]
    e1, e2, e3 = np.exp(-1 / 2.25), np.exp(-4 / 2.25), np.exp(-16 / 2.25)
    assert np.allclose(w, [e1, e1, e2, e2, e3, e3], rtol=1e-15, atol=0)


def test_weights_follow_library_distances():
    """Every stored weight equals exp(-d^2 / sigma^2) with d the library's float64 distance of the
    pair and sigma the median of its directed neighbour distances; the weights are unchanged when
    all points are scaled by 2.5 (d and sigma scale alike)."""
    nb = pytest.importorskip("sklearn.neighbors")
    pw = pytest.importorskip("sklearn.metrics")
    X = _points(300, 5, 2)
    row_ptr, col, w, sigma, _, _ = ok.knn_graph(X, 7)
    X64 = X.astype(np.float64)
    d_dir = nb.NearestNeighbors(n_neighbors=7, algorithm="brute").fit(X64).kneighbors()[0]
    s_ref = float(np.median(d_dir))
    rows = np.repeat(np.arange(X.shape[0]), np.diff(row_ptr))
    d = pw.pairwise_distances(X64)[rows, col]
    # float32 squared distances of 5 columns: relative error a few 2^-24, carried into the exponent
    a = d * d / s_ref ** 2
    assert np.all(np.abs(w - np.exp(-a)) <= np.exp(-a) * (1e-5 + 1e-5 * a))
    _, _, w2, sigma2, _, _ = ok.knn_graph((X * np.float32(2.5)).astype(np.float32), 7)
    assert abs(sigma2 - 2.5 * sigma) <= 1e-6 * sigma2
    assert np.allclose(w2, w, rtol=1e-5, atol=0)
