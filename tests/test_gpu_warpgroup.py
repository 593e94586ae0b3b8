"""A warp group per query (ann_set_warps_per_query): 2 or 4 warps share one
query's lookup table, list, fetch ring and visited set; warp 0 keeps the
relaxed pipeline and the warps split each expansion's neighbours and the list
merge (for long lists, the merge of a pending buffer).  The schedule is the
single warp's, so ids, distances and per-query step counts must equal the
oracle's bit for bit, at every depth."""
import numpy as np
import pytest

import datagen
import oracle
import paper_2507_10070_b300 as ann

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pq_index(u8_pq):
    w = u8_pq
    ix = ann.Index(w["base"], w["adj"], w["entry"], w["cb"], w["codes"],
                   tier=ann.ANN_TIER_HOST_PINNED)
    yield ix
    ix.close()


def _oracle(w, k, L, depth, q=None, adj=None, base=None, codes=None, entry=None):
    return oracle.search(w["base"] if base is None else base, w["adj"] if adj is None else adj,
                         w["entry"] if entry is None else entry, w["q"] if q is None else q, k, L, depth,
                         codebook=w["cb"], codes=w["codes"] if codes is None else codes)


@pytest.mark.parametrize("W", [2, 4])
@pytest.mark.parametrize("L", [16, 64, 256])
@pytest.mark.parametrize("depth", [0, 1, 2, 4])
def test_warp_group_bit_exact(u8_pq, pq_index, W, L, depth):
    pq_index.set_warps_per_query(W)
    try:
        ids, dists, stats, tr = pq_index.search(u8_pq["q"], 10, L, depth, trace=True)
    finally:
        pq_index.set_warps_per_query(1)
    oi, od, osteps = _oracle(u8_pq, 10, L, depth)
    assert np.array_equal(ids, oi)
    assert np.array_equal(dists.astype(np.float64), od)
    assert np.array_equal(tr["steps"], osteps)
    assert np.all(tr["status"] == 0) and stats.expansions == int(osteps.sum())


@pytest.mark.parametrize("W", [2, 4])
@pytest.mark.parametrize("k,L", [(1, 1), (33, 40), (256, 512), (10, 2048)])
def test_warp_group_k_and_L_extremes(u8_pq, pq_index, W, k, L):
    q = u8_pq["q"][:41]
    pq_index.set_warps_per_query(W)
    try:
        ids, dists, _, tr = pq_index.search(q, k, L, 1, trace=True)
    finally:
        pq_index.set_warps_per_query(1)
    oi, od, os_ = _oracle(u8_pq, k, L, 1, q=q)
    assert np.array_equal(ids, oi) and np.array_equal(dists.astype(np.float64), od)
    assert np.array_equal(tr["steps"], os_)


@pytest.mark.parametrize("W", [2, 4])
@pytest.mark.parametrize("L", [2048, 4096, 8192])
@pytest.mark.parametrize("depth", [0, 1, 2, 4])
def test_warp_group_long_lists_bit_exact(u8_pq, pq_index, W, L, depth):
    """From L = 2048 on the group keeps a pending buffer in front of the list
    (warp 0 merges each step's candidates into it, all warps merge it into
    the list when full); selection and the entry bound work on the union."""
    q = u8_pq["q"][:40]
    pq_index.set_warps_per_query(W)
    try:
        ids, dists, _, tr = pq_index.search(q, 10, L, depth, trace=True)
    finally:
        pq_index.set_warps_per_query(1)
    oi, od, os_ = _oracle(u8_pq, 10, L, depth, q=q)
    assert np.array_equal(ids, oi) and np.array_equal(dists.astype(np.float64), od)
    assert np.array_equal(tr["steps"], os_)


@pytest.mark.parametrize("R", [128])
@pytest.mark.parametrize("W", [2, 4])
def test_warp_group_long_lists_degree_128(u8_pq, R, W):
    """Degree 128 (up to 128 entering candidates a step, the pending buffer's
    size) with a long list."""
    w = u8_pq
    n = 6000
    base = w["base"][:n]
    codes = np.ascontiguousarray(w["codes"][:n])
    adj = datagen.random_links(3, n, R)
    ix = ann.Index(base, adj, 11, w["cb"], codes, tier=ann.ANN_TIER_HOST_PINNED)
    try:
        ix.set_warps_per_query(W)
        ids, d, _, tr = ix.search(w["q"][:32], 10, 2560, 2, trace=True)
    finally:
        ix.close()
    oi, od, os_ = _oracle(w, 10, 2560, 2, q=w["q"][:32], adj=adj, base=base, codes=codes, entry=11)
    assert np.array_equal(ids, oi) and np.array_equal(d.astype(np.float64), od)
    assert np.array_equal(tr["steps"], os_)


@pytest.mark.parametrize("R", [32, 128])
@pytest.mark.parametrize("W", [2, 4])
def test_warp_group_degrees_and_repeated_ids(u8_pq, R, W):
    """Random-link rows of 32 and 128 ids (one and four neighbour slots per
    lane in the single-warp kernel), folded onto 500 ids so rows repeat ids
    and link to themselves."""
    w = u8_pq
    n = 3000
    base = w["base"][:n]
    codes = np.ascontiguousarray(w["codes"][:n])
    adj = datagen.random_links(2, n, R) % 500
    ix = ann.Index(base, adj, 7, w["cb"], codes, tier=ann.ANN_TIER_HOST_PINNED)
    try:
        ix.set_warps_per_query(W)
        ids, d, _, tr = ix.search(w["q"][:100], 10, 128, 1, trace=True)
    finally:
        ix.close()
    oi, od, os_ = _oracle(w, 10, 128, 1, q=w["q"][:100], adj=adj, base=base, codes=codes, entry=7)
    assert np.array_equal(ids, oi) and np.array_equal(d.astype(np.float64), od)
    assert np.array_equal(tr["steps"], os_)


def test_warp_group_device_call_matches_host_call(u8_pq, pq_index):
    import torch
    q = torch.from_numpy(u8_pq["q"]).cuda()
    nq = q.shape[0]
    ids = torch.empty((nq, 10), dtype=torch.int32, device="cuda")
    d = torch.empty((nq, 10), dtype=torch.float32, device="cuda")
    st = torch.cuda.Stream()
    pq_index.set_warps_per_query(4)
    try:
        pq_index.search_dev(q, 10, 128, 1, ids, d, stream=st)
        stats = pq_index.sync(st)
    finally:
        pq_index.set_warps_per_query(1)
    ref = pq_index.search(u8_pq["q"], 10, 128, 1)
    assert np.array_equal(ids.cpu().numpy(), ref[0]) and np.array_equal(d.cpu().numpy(), ref[1])
    assert stats.expansions == ref[2].expansions


def test_warp_group_large_visited_sets(u8_pq):
    """A random-link graph of 60,000 nodes and R = 128 (random vectors and
    codes) at L = 1024: each query visits most of the graph, far more nodes
    than a log of the set bits keeps, so the bitset is cleared in full
    after the query.  Every group size matches the oracle bit for bit, twice
    in a row (the second batch needs the first one's bits cleared)."""
    w = u8_pq
    n = 60_000
    rng_base = datagen.random_bytes(3, n, 128)
    cb = w["cb"]
    codes = datagen.random_bytes(5, n, 32)
    adj = datagen.random_links(4, n, 128)
    ix = ann.Index(rng_base, adj, 0, cb, codes, tier=ann.ANN_TIER_HOST_PINNED)
    try:
        q = w["q"][:4]
        oi, od, os_ = oracle.search(rng_base, adj, 0, q, 10, 1024, 1, codebook=cb, codes=codes,
                                    return_visited=True)[:3]
        for W in (1, 2, 4):
            ix.set_warps_per_query(W)
            for _ in range(2):
                ids, d, stats, tr = ix.search(q, 10, 1024, 1, trace=True)
                assert np.all(tr["status"] == 0) and stats.n_failed == 0, W
                assert np.array_equal(ids, oi) and np.array_equal(d.astype(np.float64), od), W
                assert np.array_equal(tr["steps"], os_), W
        nvis = oracle.search(rng_base, adj, 0, q, 10, 1024, 1, codebook=cb, codes=codes,
                             return_visited=True)[-1]
        assert nvis.min() > 8192      # beyond the clear log's 8,192 entries
    finally:
        ix.close()


def test_set_warps_per_query_validates(u8_pq, pq_index):
    with pytest.raises(ann.AnnError):
        pq_index.set_warps_per_query(3)
    base = np.zeros((8, 8), np.float32)
    adj = np.array([[1], [2], [3], [4], [5], [6], [7], [0]], np.int32)
    ix = ann.Index(base, adj, 0, tier=ann.ANN_TIER_HBM)
    try:
        with pytest.raises(ann.AnnError):
            ix.set_warps_per_query(2)       # exact navigation: one warp per query only
        ix.set_warps_per_query(1)
    finally:
        ix.close()
