"""GPU parity: the CUDA search kernel against the CPU oracle, element by element,
on the same seeded inputs (graphs and PQ codebooks built by the oracle).

uint8 data is exact on both sides, so ids, distances and per-query step counts
must be identical.  float32 data: distances within 1e-5 relative, ids may
differ only where the distance gap is below that, recall@10 within 0.002.
"""
import numpy as np
import pytest

import datagen
import oracle
import paper_2507_10070_b300 as ann

pytestmark = pytest.mark.gpu

REL = 1e-5


@pytest.fixture(scope="module")
def pq_index(u8_pq):
    w = u8_pq
    ix = ann.Index(w["base"], w["adj"], w["entry"], w["cb"], w["codes"],
                   tier=ann.ANN_TIER_HOST_PINNED)
    yield ix
    ix.close()


def _oracle_pq(w, k, L, depth, q=None):
    return oracle.search(w["base"], w["adj"], w["entry"], w["q"] if q is None else q, k, L, depth,
                         codebook=w["cb"], codes=w["codes"])


@pytest.mark.parametrize("L", [16, 64, 256])
@pytest.mark.parametrize("depth", [0, 1, 2, 4])
def test_pq_search_bit_exact(u8_pq, pq_index, L, depth):
    k = 10
    ids, dists, stats, tr = pq_index.search(u8_pq["q"], k, L, depth, trace=True)
    oi, od, osteps = _oracle_pq(u8_pq, k, L, depth)
    assert np.array_equal(ids, oi)
    assert np.array_equal(dists.astype(np.float64), od)
    assert np.array_equal(tr["steps"], osteps)
    assert np.all(tr["status"] == 0) and stats.n_failed == 0
    assert stats.expansions == int(osteps.sum())


@pytest.mark.parametrize("L", [2048, 4096, 5120, 8192])
@pytest.mark.parametrize("depth", [0, 1, 2, 4])
def test_pq_search_long_lists_bit_exact(u8_pq, pq_index, L, depth):
    """From L = 2048 on, each step's candidates go to a short sorted pending
    buffer merged into the list only when full; selection and the entry bound
    work on the union.  The list, and so every step, must stay the oracle's
    (up to L = 8192, the longest list the benchmarks use)."""
    q = u8_pq["q"][:48]
    ids, dists, stats, tr = pq_index.search(q, 10, L, depth, trace=True)
    oi, od, osteps = _oracle_pq(u8_pq, 10, L, depth, q=q)
    assert np.array_equal(ids, oi)
    assert np.array_equal(dists.astype(np.float64), od)
    assert np.array_equal(tr["steps"], osteps)


@pytest.mark.parametrize("k,L", [(1, 1), (1, 8), (33, 40), (100, 128), (256, 512), (10, 1536)])
def test_pq_search_k_and_L_extremes(u8_pq, pq_index, k, L):
    ids, dists, _ = pq_index.search(u8_pq["q"][:97], k, L, 1)
    oi, od, _ = _oracle_pq(u8_pq, k, L, 1, q=u8_pq["q"][:97])
    assert np.array_equal(ids, oi)
    assert np.array_equal(dists.astype(np.float64), od)


def test_pq_hbm_tier_matches_host_tier(u8_pq, pq_index):
    w = u8_pq
    ix = ann.Index(w["base"], w["adj"], w["entry"], w["cb"], w["codes"], tier=ann.ANN_TIER_HBM)
    try:
        a = ix.search(w["q"], 10, 64, 1)
        b = pq_index.search(w["q"], 10, 64, 1)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    finally:
        ix.close()


def test_exact_u8_navigation_bit_exact(u8_pq):
    w = u8_pq
    ix = ann.Index(w["base"], w["adj"], w["entry"], tier=ann.ANN_TIER_HBM)
    try:
        for depth in (0, 1, 4):
            ids, dists, _, tr = ix.search(w["q"], 10, 48, depth, trace=True)
            oi, od, os_ = oracle.search(w["base"], w["adj"], w["entry"], w["q"], 10, 48, depth)
            assert np.array_equal(ids, oi)
            assert np.array_equal(dists.astype(np.float64), od)
            assert np.array_equal(tr["steps"], os_)
    finally:
        ix.close()


@pytest.fixture(scope="module")
def f32_inmem():
    """In-memory float workload: 10k float32 vectors, d=128, 32 clusters, 200
    queries, Vamana R=32 alpha=1.2 L_build=64 built by the oracle."""
    mx = datagen.inmemory_f32()
    base, q = mx.base(10_000), mx.queries(200)
    entry = oracle.medoid(base)
    adj = oracle.vamana(base, 32, 1.2, 64, entry, datagen.build_order(mx.seed, 10_000),
                        datagen.random_out_neighbours(mx.seed, 10_000, 32))
    gi, gd = oracle.knn(base, q, 10)
    return dict(base=base, q=q, entry=entry, adj=adj, gi=gi, gd=gd)


def _check_f32(ids, dists, oi, od):
    # distances agree within REL where the ids agree ...
    same = ids == oi
    assert np.all(np.abs(dists[same] - od[same]) <= REL * np.maximum(od[same], 1e-30))
    # ... and a differing id is only a near-tie swap at that rank
    diff = ~same
    if diff.any():
        assert np.all(np.abs(dists[diff] - od[diff]) <= REL * od[diff])
    return float(same.mean())


@pytest.mark.parametrize("depth", [0, 1, 2, 4])
def test_exact_f32_inmemory_parity(f32_inmem, depth):
    w = f32_inmem
    ix = ann.Index(w["base"], w["adj"], w["entry"], tier=ann.ANN_TIER_HBM)
    try:
        ids, dists, _ = ix.search(w["q"], 10, 64, depth)
        oi, od, _ = oracle.search(w["base"], w["adj"], w["entry"], w["q"], 10, 64, depth)
        _check_f32(ids, dists, oi, od)
        r_gpu = ann.recall_at_k(ids, w["gi"], w["gd"], dists)
        r_orc = oracle.recall_at_k(oi, w["gi"], w["gd"], od)
        assert abs(r_gpu - r_orc) <= 0.002
        if depth == 0:
            assert r_gpu >= 0.95
    finally:
        ix.close()


def test_search_dev_matches_host_and_sync_reports(u8_pq, pq_index):
    import torch
    q = torch.from_numpy(u8_pq["q"]).cuda()
    nq, k = q.shape[0], 10
    ids = torch.empty((nq, k), dtype=torch.int32, device="cuda")
    dists = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    steps = torch.empty(nq, dtype=torch.int32, device="cuda")
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        for _ in range(2):   # two calls before one sync accumulate
            pq_index.search_dev(q, k, 64, 1, ids, dists, stream=st, trace={"steps": steps})
    stats = pq_index.sync(st)
    hi, hd, _, tr = pq_index.search(u8_pq["q"], k, 64, 1, trace=True)
    assert np.array_equal(ids.cpu().numpy(), hi)
    assert np.array_equal(dists.cpu().numpy(), hd)
    assert np.array_equal(steps.cpu().numpy(), tr["steps"])
    assert stats.queries == 2 * nq and stats.expansions == 2 * int(tr["steps"].sum())
    assert stats.n_failed == 0 and stats.first_failed == -1
    # timestamps: every query has a begin <= end
    assert np.all(tr["t_end"] >= tr["t_begin"]) and np.all(tr["t_begin"] > 0)


def test_edge_cases(u8_pq, pq_index):
    # empty batch
    ids, dists, stats = pq_index.search(u8_pq["q"][:0], 10, 32, 1)
    assert ids.shape == (0, 10) and stats.queries == 0
    # single query, deepest pipeline
    ids, dists, _ = pq_index.search(u8_pq["q"][:1], 5, 5, 4)
    oi, od, _ = _oracle_pq(u8_pq, 5, 5, 4, q=u8_pq["q"][:1])
    assert np.array_equal(ids, oi)
    # argument errors
    for k, L, depth in [(0, 10, 0), (11, 10, 0), (10, 16385, 0), (10, 32, 5), (10, 32, -1)]:
        with pytest.raises(ann.AnnError):
            pq_index.search(u8_pq["q"][:4], k, L, depth)


def test_degenerate_graphs():
    # a single node, and an entry with no out-edges: results are padded
    base = np.array([[1, 2, 3, 4], [9, 9, 9, 9]], np.uint8)
    adj = np.array([[-1], [0]], np.int32)
    ix = ann.Index(base, adj, 0, tier=ann.ANN_TIER_HBM)
    try:
        ids, dists, _ = ix.search(np.array([[9, 9, 9, 9]], np.uint8), 2, 4, 2)
        assert ids.tolist() == [[0, -1]]
        assert dists[0, 0] == 8 * 8 + 7 * 7 + 6 * 6 + 5 * 5 and np.isinf(dists[0, 1])
    finally:
        ix.close()
    one = ann.Index(base[:1], np.array([[-1]], np.int32), 0, tier=ann.ANN_TIER_HBM)
    try:
        ids, dists, _ = one.search(base[:1], 1, 1, 0)
        assert ids.tolist() == [[0]] and dists[0, 0] == 0
    finally:
        one.close()


@pytest.mark.parametrize("L,depth", [(16, 0), (128, 2)])
def test_repeated_ids_and_self_links(u8_pq, L, depth):
    """Rows with repeated neighbour ids and self links (a random-link graph
    folded onto 400 ids): a repeat is seen as visited, as in the oracle."""
    w = u8_pq
    n = 3000
    base = w["base"][:n]
    adj = datagen.random_links(1, n, 64) % 400
    codes = np.ascontiguousarray(w["codes"][:n])
    assert any(len(set(r.tolist())) < 64 for r in adj) and any(i in adj[i] for i in range(400))
    ix = ann.Index(base, adj, 7, w["cb"], codes, tier=ann.ANN_TIER_HOST_PINNED)
    try:
        ids, d, _, tr = ix.search(w["q"], 10, L, depth, trace=True)
    finally:
        ix.close()
    oi, od, os_ = oracle.search(base, adj, 7, w["q"], 10, L, depth, codebook=w["cb"], codes=codes)
    assert np.array_equal(ids, oi) and np.array_equal(d.astype(np.float64), od)
    assert np.array_equal(tr["steps"], os_)


def _relabel(ids, labels):
    return np.where(ids >= 0, labels[np.maximum(ids, 0)], -1)


def test_id_map_relabels_results(u8_pq, pq_index, tmp_path):
    """An index loaded with an id map reports id_map[node] and searches as
    before: batch call, index file, exact-navigation index."""
    w = u8_pq
    n = w["base"].shape[0]
    labels = (np.arange(n, dtype=np.int64) * 3 + 11).astype(np.int32)
    ref_i, ref_d, _ = pq_index.search(w["q"], 10, 64, 1)
    ixm = ann.Index(w["base"], w["adj"], w["entry"], w["cb"], w["codes"],
                    tier=ann.ANN_TIER_HOST_PINNED, id_map=labels)
    try:
        i1, d1, _ = ixm.search(w["q"], 10, 64, 1)
    finally:
        ixm.close()
    assert np.array_equal(i1, _relabel(ref_i, labels)) and np.array_equal(d1, ref_d)
    path = str(tmp_path / "mapped.idx")
    ann.save_index(path, w["base"], w["adj"], w["entry"], w["cb"], w["codes"], id_map=labels)
    ixf = ann.Index(path=path, tier=ann.ANN_TIER_HOST_PINNED)
    try:
        i2, d2, _ = ixf.search(w["q"], 10, 64, 1)
    finally:
        ixf.close()
    assert np.array_equal(i2, i1) and np.array_equal(d2, ref_d)
    e0 = ann.Index(w["base"], w["adj"], w["entry"], tier=ann.ANN_TIER_HBM)
    e1 = ann.Index(w["base"], w["adj"], w["entry"], tier=ann.ANN_TIER_HBM, id_map=labels)
    try:
        a_i, a_d, _ = e0.search(w["q"], 10, 32, 2)
        b_i, b_d, _ = e1.search(w["q"], 10, 32, 2)
    finally:
        e0.close()
        e1.close()
    assert np.array_equal(b_i, _relabel(a_i, labels)) and np.array_equal(b_d, a_d)


@pytest.mark.parametrize("order", ["bfs", "spatial"])
@pytest.mark.parametrize("L,depth", [(64, 1), (256, 0)])
def test_reordered_layout_matches_oracle(u8_pq, order, L, depth):
    """The kernel on the reordered index (breadth-first or spatial) reports
    original ids (through the id map) and equals the oracle searching the
    same reordered index, mapped back the same way."""
    w = u8_pq
    b2, a2, e2, c2, old = ann.reorder_graph(w["base"], w["adj"], w["entry"], w["codes"], order=order)
    ix = ann.Index(b2, a2, e2, w["cb"], c2, tier=ann.ANN_TIER_HOST_PINNED, id_map=old)
    try:
        ids, d, _, tr = ix.search(w["q"], 10, L, depth, trace=True)
    finally:
        ix.close()
    oi, od, os_ = oracle.search(b2, a2, e2, w["q"], 10, L, depth, codebook=w["cb"], codes=c2)
    assert np.array_equal(ids, _relabel(oi, old)) and np.array_equal(d.astype(np.float64), od)
    assert np.array_equal(tr["steps"], os_)


@pytest.mark.parametrize("depth", [0, 1])
def test_kernel_grained_ablation_matches_query_grained(u8_pq, pq_index, depth):
    """The kernel-grained I/O ablation (grid barrier after every fetch wait)
    changes only timing: results and step counts equal the query-grained
    search, for a full grid and for fewer queries than resident warps."""
    import torch
    w = u8_pq
    st = torch.cuda.Stream()

    def run(fn, qh):
        q = torch.from_numpy(qh).cuda()
        nq = q.shape[0]
        ids = torch.empty((nq, 10), dtype=torch.int32, device="cuda")
        d = torch.empty((nq, 10), dtype=torch.float32, device="cuda")
        steps = torch.empty(nq, dtype=torch.int32, device="cuda")
        fn(q, 10, 64, depth, ids, d, stream=st, trace={"steps": steps})
        stats = pq_index.sync(st)
        return ids.cpu().numpy(), d.cpu().numpy(), steps.cpu().numpy(), stats

    for qh in (w["q"], w["q"][:5]):
        a = run(pq_index.search_dev, qh)
        b = run(pq_index.search_dev_kernel_grained, qh)
        assert b[3].n_failed == 0 and b[3].expansions == a[3].expansions
        for x, y in zip(a[:3], b[:3]):
            assert np.array_equal(x, y)


def test_kernel_grained_bounded_wait_reports_timeout(u8_pq, pq_index, monkeypatch):
    """The ablation's barrier waits are bounded.  A host-side hook presets its
    arrival count so that no round can ever complete: every warp must give
    up after its bounded spin, the call must report ANN_ETIMEOUT, and the
    index must keep working afterwards."""
    import torch
    w = u8_pq
    q = torch.from_numpy(w["q"][:64]).cuda()
    ids = torch.empty((64, 10), dtype=torch.int32, device="cuda")
    d = torch.empty((64, 10), dtype=torch.float32, device="cuda")
    st = torch.cuda.Stream()
    monkeypatch.setenv("ANN_TEST_STALL_ROUNDS", "1")
    pq_index.search_dev_kernel_grained(q, 10, 64, 0, ids, d, stream=st)
    with pytest.raises(ann.AnnError) as e:
        pq_index.sync(st)
    assert e.value.status == ann._abi.ANN_ETIMEOUT
    monkeypatch.delenv("ANN_TEST_STALL_ROUNDS")
    pq_index.search_dev_kernel_grained(q, 10, 64, 0, ids, d, stream=st)
    assert pq_index.sync(st).n_failed == 0
    ref_i, ref_d, _ = pq_index.search(w["q"][:64], 10, 64, 0)
    assert np.array_equal(ids.cpu().numpy(), ref_i) and np.array_equal(d.cpu().numpy(), ref_d)


def test_visited_set_holds_every_node():
    """On a ring lattice (node i -> i+1..i+R, positions on a line) a query at
    the far end makes the search march through every one of 60,000 nodes.
    The visited set is one bit per node, so the query completes and matches
    the oracle (integer coordinates: FP32 distances are exact), and a second
    batch on the same index, which needs its bits cleared, does too."""
    n, R = 60_000, 128
    base = np.zeros((n, 4), np.float32)
    base[:, 0] = np.arange(n, dtype=np.float32)
    adj = ((np.arange(n)[:, None] + 1 + np.arange(R)[None, :]) % n).astype(np.int32)
    ix = ann.Index(base, adj, 0, tier=ann.ANN_TIER_HBM)
    try:
        q = np.zeros((3, 4), np.float32)
        q[:, 0] = n - 1
        ids, dists, stats, tr = ix.search(q, 10, 32, 1, trace=True)
        assert np.all(tr["status"] == 0) and stats.n_failed == 0
        oi, od, os_ = oracle.search(base, adj, 0, q, 10, 32, 1)
        assert np.array_equal(ids, oi) and np.array_equal(dists.astype(np.float64), od)
        assert np.array_equal(tr["steps"], os_) and os_.min() > n // R
        ids2, _, _, tr2 = ix.search(q, 10, 32, 1, trace=True)
        assert np.array_equal(ids2, ids) and np.array_equal(tr2["steps"], tr["steps"])
        ok, okd, _ = ix.search(np.zeros((1, 4), np.float32), 3, 32, 1)
        assert ok.tolist() == [[0, 1, 2]]
    finally:
        ix.close()


@pytest.mark.parametrize("dtype", ["u8", "f32"])
def test_knn_exact_matches_oracle(dtype):
    mx = datagen.sift_like() if dtype == "u8" else datagen.inmemory_f32()
    base, q = mx.base(7000), mx.queries(150)
    ids, d = ann.knn_exact(base, q, 10)
    oi, od = oracle.knn(base, q, 10)
    if dtype == "u8":
        assert np.array_equal(ids, oi) and np.array_equal(d.astype(np.float64), od)
    else:
        _check_f32(ids, d, oi, od)


def test_read_probe_runs():
    g_host = ann.probe_read_bandwidth(64 << 20, 512, ann.ANN_TIER_HOST_PINNED, 16)
    g_hbm = ann.probe_read_bandwidth(256 << 20, 512, ann.ANN_TIER_HBM, 16)
    assert g_host > 1.0 and g_hbm > g_host
