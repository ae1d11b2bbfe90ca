"""GPU parity of graph ingest, the power step and the embedding (Sec. 2, Algorithms 1-2).

Every case compares the CUDA path (through the C ABI) with the float64 oracle on
the same seeded inputs.  Tolerances: degrees exact (unit weights: counts; weights:
float64 sums in entry order, the oracle's order); one power step 2e-6 relative
Frobenius (float32 accumulation of ~30 terms); the embedding 1e-5 relative
Frobenius in float32 storage and 2e-2 in bfloat16 storage.
"""
import numpy as np
import pytest

import workloads as W
from _helpers import rel_fro, require_cuda
from oracle import spectral

pytestmark = pytest.mark.gpu

GRAPHS = {
    "sbm_1000_k4": lambda: W.sbm([250] * 4, 0.1, 0.002, 1),
    "sbm_ragged": lambda: W.sbm([131, 77, 260], 0.08, 0.004, 2),
    "knn_weighted": lambda: W.knn_mixture(3000, 16, 6, 10, seed=3),
    "image_weighted": lambda: W.image_grid(40, 57, 5, seed=4),
    "cycle": lambda: W.cycle(1001),
    "cliques": lambda: W.disjoint_cliques(7, 23),
    "isolated": lambda: W.with_isolated(W.sbm([200, 300], 0.05, 0.003, 5), 37),
    "permuted_sbm": lambda: W.permuted(W.sbm([500] * 3, 0.04, 0.002, 6), 7),
}


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def _graph(torch, g):
    import paper_2310_10939_gb300 as fsc
    return fsc.Graph.from_workload(g)


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_degrees_and_isolated_count(torch, name):
    g = GRAPHS[name]()
    G = _graph(torch, g)
    d = G.degrees().cpu().numpy()
    ref = spectral.degrees(g)
    # unit weights: exact counts; weights: float64 sums in entry order, the oracle's order too
    assert np.array_equal(d, ref)
    info = G.info()
    assert info["n_isolated"] == int((ref == 0).sum())
    assert np.isclose(info["volume"], ref.sum(), rtol=1e-12)
    dinv = G.dinv().cpu().numpy()
    # float32 1/sqrt(float32(d)): two correctly rounded operations, within 2 ulp of d^-1/2
    assert np.allclose(dinv, spectral.inv_sqrt_degrees(ref), rtol=2.5e-7, atol=0)
    assert np.array_equal(dinv == 0, ref == 0)


@pytest.mark.parametrize("name", ["sbm_1000_k4", "knn_weighted", "image_weighted", "isolated"])
@pytest.mark.parametrize("l", [1, 2, 3, 8])
@pytest.mark.parametrize("tpr", [4, 8, 16, 32])
def test_power_step_matches_oracle(torch, name, l, tpr):
    import paper_2310_10939_gb300 as fsc
    g = GRAPHS[name]()
    G = _graph(torch, g)
    lp = fsc.pad_l(l)
    rng = np.random.default_rng(l * 100 + tpr)
    z = np.zeros((g.n, lp), dtype=np.float32)
    z[:, :l] = rng.normal(size=(g.n, l)).astype(np.float32)
    zin = torch.as_tensor(z, device="cuda")
    zout = torch.full_like(zin, float("nan"))
    fsc.power_step(G, l, zin, zout, threads_per_row=tpr)
    got = zout.cpu().numpy()
    d = spectral.degrees(g)
    dh = np.sqrt(d)
    dm = spectral.inv_sqrt_degrees(d)
    M = spectral.signless_laplacian(g)
    ref = dm[:, None] * (M @ (dh[:, None] * z[:, :l].astype(np.float64)))
    # isolated vertices: z = D^-1/2 x is 0 there; the step keeps z/2 (D^-1 A z = 0)
    iso = d == 0
    ref[iso] = 0.5 * z[iso, :l]
    assert rel_fro(got[:, :l], ref) <= 2e-6
    assert np.array_equal(got[:, l:], np.zeros((g.n, lp - l), dtype=np.float32))


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("l,t", [(2, 20), (3, 7), (1, 5), (5, 12), (8, 3)])
def test_embed_f32_matches_oracle(torch, name, l, t):
    import paper_2310_10939_gb300 as fsc
    g = GRAPHS[name]()
    G = _graph(torch, g)
    seed = 1000 + 7 * l + t
    emb = fsc.embed(G, l, t, seed).cpu().numpy()
    ref = spectral.embed(g, l, t, seed)
    assert rel_fro(emb[:, :l], ref) <= 1e-5
    assert np.array_equal(emb[:, l:], np.zeros((g.n, emb.shape[1] - l), dtype=np.float32))


@pytest.mark.parametrize("t", [0, 1, 2, 3])
def test_embed_small_t_including_zero(torch, t):
    import paper_2310_10939_gb300 as fsc
    g = GRAPHS["isolated"]()
    G = _graph(torch, g)
    for store in (fsc.F32, fsc.BF16):
        emb = fsc.embed(G, 3, t, 77, store=store, rescale=True).cpu().numpy()
        ref = spectral.embed(g, 3, t, 77)
        assert rel_fro(emb[:, :3], ref) <= (1e-5 if store == fsc.F32 or t == 0 else 2e-2)
        assert np.array_equal(emb[-37:], np.zeros_like(emb[-37:]))   # isolated rows are zero


@pytest.mark.parametrize("name", ["sbm_1000_k4", "knn_weighted", "image_weighted", "cliques"])
@pytest.mark.parametrize("tpr", [4, 8, 16, 32])
def test_rescale_is_exact_and_threads_per_row_agree(torch, name, tpr):
    import paper_2310_10939_gb300 as fsc
    g = GRAPHS[name]()
    G = _graph(torch, g)
    for store in (fsc.F32, fsc.BF16):
        a = fsc.embed(G, 4, 25, 5, store=store, rescale=False, threads_per_row=tpr)
        b = fsc.embed(G, 4, 25, 5, store=store, rescale=True, threads_per_row=tpr)
        assert torch.equal(a, b), "power-of-two rescale must not change the result"


@pytest.mark.parametrize("name", ["sbm_1000_k4", "knn_weighted", "image_weighted", "cycle", "isolated"])
def test_embed_bf16_within_tolerance(torch, name):
    import paper_2310_10939_gb300 as fsc
    g = GRAPHS[name]()
    G = _graph(torch, g)
    l, t = 3, 30
    emb = fsc.embed(G, l, t, 11, store=fsc.BF16, rescale=True).cpu().numpy()
    ref = spectral.embed(g, l, t, 11)
    err = rel_fro(emb[:, :l], ref)
    assert err <= 2e-2
    emb32 = fsc.embed(G, l, t, 11).cpu().numpy()
    assert rel_fro(emb32[:, :l], ref) <= 1e-5


def test_embed_eigenvalue_one_direction(torch):
    """P-a through the GPU: x = D^1/2 1 is fixed by M, so z = D^-1/2 x = 1 is fixed by the step."""
    import paper_2310_10939_gb300 as fsc
    g = GRAPHS["knn_weighted"]()
    G = _graph(torch, g)
    z = torch.zeros((g.n, 4), dtype=torch.float32, device="cuda")
    z[:, 0] = 1.0
    out = torch.empty_like(z)
    fsc.power_step(G, 4, z, out)
    assert torch.allclose(out[:, 0], torch.ones_like(out[:, 0]), rtol=0, atol=1e-6)


def test_graph_validation_errors(torch):
    import paper_2310_10939_gb300 as fsc
    g = W.sbm([30, 30], 0.2, 0.05, 9)

    def make(rp, col, w=None, **kw):
        return fsc.Graph(torch.as_tensor(rp, device="cuda"), torch.as_tensor(col, device="cuda"),
                         None if w is None else torch.as_tensor(w, device="cuda"), **kw)

    col = g.col.copy()
    col[5] = g.n + 3
    with pytest.raises(fsc.FscError) as e:
        make(g.row_ptr, col)
    assert e.value.name == "FSC_ERR_INDEX_RANGE"
    col = g.col.copy()
    r0 = np.searchsorted(g.row_ptr, 10, side="right") - 1
    col[g.row_ptr[10]] = 10
    with pytest.raises(fsc.FscError) as e:
        make(g.row_ptr, col)
    assert e.value.name == "FSC_ERR_SELF_LOOP"
    w = np.ones(g.nnz, dtype=np.float32)
    w[3] = np.nan
    with pytest.raises(fsc.FscError) as e:
        make(g.row_ptr, g.col, w)
    assert e.value.name == "FSC_ERR_BAD_WEIGHT"
    w[3] = -1.0
    with pytest.raises(fsc.FscError) as e:
        make(g.row_ptr, g.col, w)
    assert e.value.name == "FSC_ERR_BAD_WEIGHT"
    w = np.ones(g.nnz, dtype=np.float32)
    w[7] = 2.0                                   # mirror entry keeps weight 1
    make(g.row_ptr, g.col, w)                    # accepted without the symmetry check
    with pytest.raises(fsc.FscError) as e:
        make(g.row_ptr, g.col, w, validate_symmetry=True)
    assert e.value.name == "FSC_ERR_NOT_SYMMETRIC"
    rp = g.row_ptr.copy()
    rp[-1] += 1
    with pytest.raises(fsc.FscError) as e:
        make(rp, np.concatenate([g.col, [0]]).astype(np.int32)[:g.nnz])
    assert e.value.name == "FSC_ERR_INDEX_RANGE"
    make(g.row_ptr, g.col, validate_symmetry=True)   # the valid graph passes
    del r0


def _unit_csr(torch, row_ptr, col, offset=0):
    """row_ptr and col on the device, col starting ``offset`` int32 elements into a larger buffer
    (offset 0: a 16-byte aligned start; 1-3: the unaligned starts a caller's view can have)."""
    rp = torch.as_tensor(row_ptr, device="cuda")
    buf = torch.zeros(col.size + offset, dtype=torch.int32, device="cuda")
    buf[offset:] = torch.as_tensor(col, device="cuda")
    return rp, buf[offset:]


@pytest.mark.parametrize("offset", [0, 1, 2, 3])
def test_unit_degrees_many_tiles_any_alignment(torch, offset):
    """Unit-weight degrees and header statistics (Sec. 2: d(v) is the row length) on a graph of
    hundreds of row tiles with isolated vertices scattered through it, for a col array at each
    4-byte offset from a 16-byte boundary (the vector scan and the scalar scan)."""
    import paper_2310_10939_gb300 as fsc
    g = W.permuted(W.with_isolated(W.sbm([20000, 13001, 7000], 0.0008, 0.00005, 11), 311), 12)
    rp, col = _unit_csr(torch, g.row_ptr, g.col, offset)
    assert (col.data_ptr() % 16 == 0) == (offset == 0)
    G = fsc.Graph(rp, col)
    ref = spectral.degrees(g)
    assert np.array_equal(G.degrees().cpu().numpy(), ref)
    info = G.info()
    assert info["n_isolated"] == int((ref == 0).sum()) >= 311
    assert info["volume"] == float(ref.sum())
    assert info["deg_max"] == float(ref.max())
    assert info["deg_sumsq"] == float((ref * ref).sum())
    assert np.array_equal(G.dinv().cpu().numpy() == 0, ref == 0)
    # the same power step as from the aligned copy (the SpMM reads col one entry at a time)
    if offset:
        G0 = fsc.Graph(*_unit_csr(torch, g.row_ptr, g.col, 0))
        z = torch.as_tensor(np.random.default_rng(3).normal(size=(g.n, 4)).astype(np.float32), device="cuda")
        a, b = torch.empty_like(z), torch.empty_like(z)
        fsc.power_step(G, 4, z, a)
        fsc.power_step(G0, 4, z, b)
        assert torch.equal(a, b)


def _graph_with_nnz_mod4(want: int):
    for seed in range(40, 200):
        g = W.sbm([300, 301], 0.05, 0.005, seed)
        if g.nnz % 4 == want:
            return g
    raise AssertionError("no seed gives the wanted nnz mod 4")


@pytest.mark.parametrize("lane", [0, 1, 2, 3])
@pytest.mark.parametrize("offset", [0, 1])
def test_validation_at_each_vector_position(torch, lane, offset):
    """A self-loop, an out-of-range index and an unsorted pair (with the symmetry check) are each
    found wherever they sit in a 4-entry vector, for aligned and unaligned col."""
    import paper_2310_10939_gb300 as fsc
    g = _graph_with_nnz_mod4(2)
    rp = g.row_ptr

    def entry_in_middle_row(need_next=False):
        for i in range(g.n // 2, g.n):
            for p in range(rp[i], rp[i + 1] - (1 if need_next else 0)):
                if (p - offset) % 4 == lane and (not need_next or p > rp[i]):
                    return i, p
        raise AssertionError

    def status(col, sym=False):
        with pytest.raises(fsc.FscError) as e:
            fsc.Graph(*_unit_csr(torch, rp, col, offset), validate_symmetry=sym)
        return e.value.name

    i, p = entry_in_middle_row()
    col = g.col.copy()
    col[p] = i
    assert status(col) == "FSC_ERR_SELF_LOOP"
    for bad in (g.n, -1, 2**31 - 1):
        col = g.col.copy()
        col[p] = bad
        assert status(col) == "FSC_ERR_INDEX_RANGE"
    # unsorted: the pair (p - 1, p) inverted, found at p, whose predecessor is in the same vector
    # (lane > 0) or in the previous one (lane 0)
    i, p = entry_in_middle_row(need_next=True)
    col = g.col.copy()
    col[p - 1], col[p] = col[p], col[p - 1]
    assert status(col, sym=True) == "FSC_ERR_UNSORTED"
    fsc.Graph(*_unit_csr(torch, rp, col, offset))   # accepted when sortedness is not asked for


def test_validation_tail_and_middle_row_ptr(torch):
    """The last entry of a col array whose length is not a multiple of 4 (the scalar tail), and a
    row_ptr that decreases in a middle tile, are both reported."""
    import paper_2310_10939_gb300 as fsc
    g = _graph_with_nnz_mod4(2)
    col = g.col.copy()
    col[-1] = g.n
    with pytest.raises(fsc.FscError) as e:
        fsc.Graph(*_unit_csr(torch, g.row_ptr, col))
    assert e.value.name == "FSC_ERR_INDEX_RANGE"
    big = W.sbm([20000, 20000], 0.0006, 0.00004, 13)
    rp = big.row_ptr.copy()
    mid = big.n // 2 + 17
    rp[mid] = rp[mid + 1] + 1
    with pytest.raises(fsc.FscError) as e:
        fsc.Graph(*_unit_csr(torch, rp, big.col))
    assert e.value.name == "FSC_ERR_INDEX_RANGE"


def _star(leaves: int, seed: int):
    """Vertex 0 joined to every other vertex, random positive weights (symmetric)."""
    rng = np.random.default_rng(seed)
    n = leaves + 1
    wl = rng.uniform(0.1, 2.0, size=leaves).astype(np.float32)
    row_ptr = np.concatenate([[0, leaves], leaves + np.arange(1, leaves + 1)]).astype(np.int64)
    col = np.concatenate([np.arange(1, n), np.zeros(leaves)]).astype(np.int32)
    w = np.concatenate([wl, wl]).astype(np.float32)
    return W.Graph(n, row_ptr, col, w, None, "star")


@pytest.mark.parametrize("which", ["knn_many_tiles", "star_long_row"])
def test_weighted_degrees_exact(torch, which):
    """Weighted degrees (Sec. 2: d(v) = sum of w(u, v)) equal the oracle's float64 sums bit for
    bit on a kNN graph of many row tiles, and on a star whose centre row (12,000 entries) does
    not fit one tile's staging buffer, so that tile sums from global memory."""
    import paper_2310_10939_gb300 as fsc
    g = W.knn_mixture(20000, 16, 8, 10, seed=21) if which == "knn_many_tiles" else _star(12000, 22)
    G = fsc.Graph.from_workload(g)
    ref = spectral.degrees(g)
    assert np.array_equal(G.degrees().cpu().numpy(), ref)
    info = G.info()
    assert info["n_isolated"] == 0
    assert info["deg_max"] == float(ref.max())
    assert np.isclose(info["volume"], ref.sum(), rtol=1e-13)
    assert np.array_equal(G.dinv().cpu().numpy() == 0, ref == 0)


@pytest.mark.parametrize("weighted", [False, True])
def test_copy_flag_graph_owns_its_csr(torch, weighted):
    """With FSC_COPY the graph keeps its own CSR: the caller's arrays are overwritten and freed after
    creation, and the degrees, a power step and the embedding equal those of a graph that borrows an
    intact copy (the same kernels on the same values: bit for bit)."""
    import paper_2310_10939_gb300 as fsc
    g = W.knn_mixture(5000, 8, 5, 10, seed=31) if weighted else W.sbm([700] * 6, 0.03, 0.002, 31)
    rp, col = torch.as_tensor(g.row_ptr, device="cuda"), torch.as_tensor(g.col, device="cuda")
    w = None if g.w is None else torch.as_tensor(g.w, device="cuda")
    Gc = fsc.Graph(rp, col, w, copy=True, validate_symmetry=True)
    assert Gc.row_ptr is None and Gc.col is None
    rp.fill_(0)
    col.fill_(-1)
    if w is not None:
        w.fill_(float("nan"))
    del rp, col, w
    torch.cuda.synchronize()
    Gb = fsc.Graph.from_workload(g)
    assert torch.equal(Gc.degrees(), Gb.degrees())
    assert np.array_equal(Gc.degrees().cpu().numpy(), spectral.degrees(g))
    z = torch.randn((g.n, 4), device="cuda")
    oc, ob = torch.empty_like(z), torch.empty_like(z)
    fsc.power_step(Gc, 4, z, oc)
    fsc.power_step(Gb, 4, z, ob)
    assert torch.equal(oc, ob)
    assert torch.equal(fsc.embed(Gc, 3, 9, 4), fsc.embed(Gb, 3, 9, 4))
    assert rel_fro(fsc.embed(Gc, 3, 9, 4).cpu().numpy()[:, :3], spectral.embed(g, 3, 9, 4)) <= 1e-5
    Gc.close()


@pytest.mark.parametrize("n", [3, 5, 6, 7, 10, 1025, 1026, 1027, 4099])
def test_start_block_every_row_alignment(torch, n):
    """The start block (t = 0) on cycles whose n leaves every remainder mod 4 (a row group of four
    then takes its draws from one Philox block or from two), for every l up to 8, in float32 and
    bfloat16: against the oracle's D^-1/2 X0, and the padding columns zero."""
    import paper_2310_10939_gb300 as fsc
    g = W.cycle(n)
    G = _graph(torch, g)
    for l in range(1, 9):
        ref = spectral.embed(g, l, 0, 100 + l)
        for store, bar in ((fsc.F32, 1e-6), (fsc.BF16, 4e-3)):
            emb = fsc.embed(G, l, 0, 100 + l, store=store, rescale=store == fsc.BF16).cpu().numpy()
            assert rel_fro(emb[:, :l], ref) <= bar, (l, store)
            assert np.all(emb[:, l:] == 0)
