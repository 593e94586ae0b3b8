"""Index-construction tooling of the library (host threads) against the oracle."""
import numpy as np
import pytest

import datagen
import oracle
import paper_2507_10070_b300 as ann


def test_build_pq_bit_exact_with_oracle_u8():
    """uint8 data: the same k-means++ draws and Lloyd steps give the same
    integer codebook and the same codes as the oracle, whatever the threads."""
    mx = datagen.sift_like()
    x = mx.base(2500)
    u = datagen.kmeanspp_uniforms(mx.seed, 32)
    cb_o = oracle.pq_train(x, 32, u, iters=4)
    cb, codes = ann.build_pq(x, 32, n_train=2500, iters=4, kpp_uniforms=u, threads=3)
    assert np.array_equal(cb, cb_o)
    assert np.array_equal(codes, oracle.pq_encode(x, cb_o))
    cb1, codes1 = ann.build_pq(x, 32, n_train=2500, iters=4, kpp_uniforms=u, threads=1)
    assert np.array_equal(cb1, cb) and np.array_equal(codes1, codes)


def test_build_graph_invariants_and_quality():
    mx = datagen.inmemory_f32()
    base, q = mx.base(6000), mx.queries(100)
    adj, entry = ann.build_graph(base, 32, 1.2, 64, seed=7, threads=4)
    assert entry == oracle.medoid(base)
    for i, row in enumerate(adj):
        nb = row[row >= 0]
        assert np.all(row[len(nb):] == -1)
        assert i not in nb and len(set(nb.tolist())) == len(nb)
    adj1, _ = ann.build_graph(base, 32, 1.2, 64, seed=7, threads=1)
    assert np.array_equal(adj, adj1)              # deterministic batches
    gi, gd = oracle.knn(base, q, 10)
    ids, d, _ = oracle.search(base, adj, entry, q, 10, 64, 0)
    assert oracle.recall_at_k(ids, gi, gd, d) >= 0.95


def _bfs(adj, entry):
    """Breadth-first order written out: neighbours in row order up to the
    first -1; when the queue runs dry, breadth-first again from the lowest
    id not yet placed."""
    import collections
    n = adj.shape[0]
    pos = np.full(n, -1)
    order = [entry]
    pos[entry] = 0
    dq = collections.deque([entry])
    nxt = 0
    while len(order) < n:
        if not dq:
            while pos[nxt] >= 0:
                nxt += 1
            pos[nxt] = len(order)
            order.append(nxt)
            dq.append(nxt)
        u = dq.popleft()
        for w in adj[u]:
            if w < 0:
                break
            if pos[w] < 0:
                pos[w] = len(order)
                order.append(w)
                dq.append(w)
    return np.array(order)


def test_reorder_graph_is_breadth_first_and_relabels():
    rng = np.random.default_rng(3)
    n, R = 3000, 12
    adj = rng.integers(0, n, (n, R)).astype(np.int32)          # repeats and self links
    adj[rng.random((n, R)) < 0.2] = -1                          # rows end at the first -1
    adj[:50] = -1                                               # nodes 0..49 have no out-edges
    adj[:, :1][adj[:, :1] < 50] = 100                           # ... and nobody links to them
    adj[(adj >= 0) & (adj < 50)] = 200
    base = rng.integers(0, 256, (n, 16)).astype(np.uint8)
    codes = rng.integers(0, 256, (n, 4)).astype(np.uint8)
    b2, a2, e2, c2, old = ann.reorder_graph(base, adj, 777, codes)
    assert np.array_equal(old, _bfs(adj, 777)) and e2 == 0
    pos = np.empty(n, np.int64)
    pos[old] = np.arange(n)
    assert np.all(np.diff(pos[:50]) > 0) and pos[0] > n // 2     # isolated nodes: late, in id order
    assert np.array_equal(b2, base[old]) and np.array_equal(c2, codes[old])
    assert np.array_equal(a2, np.where(adj[old] >= 0, pos[np.maximum(adj[old], 0)], -1))
    with pytest.raises(ann.AnnError):
        bad = adj.copy()
        bad[5, 0] = n
        ann.reorder_graph(base, bad, 0, codes)


@pytest.mark.parametrize("order", ["bfs", "spatial"])
def test_reordered_index_searches_the_same_graph(order):
    """The oracle on the reordered index, with ids mapped back, equals the
    oracle on the original (float32 data: no distance ties)."""
    mx = datagen.inmemory_f32()
    base, q = mx.base(4000), mx.queries(100)
    entry = oracle.medoid(base)
    adj = oracle.vamana(base, 32, 1.2, 64, entry, datagen.build_order(mx.seed, 4000),
                        datagen.random_out_neighbours(mx.seed, 4000, 32))
    b2, a2, e2, _, old = ann.reorder_graph(base, adj, entry, order=order)
    assert old[e2] == entry
    for depth in (0, 2):
        i0, d0, s0 = oracle.search(base, adj, entry, q, 10, 48, depth)
        i1, d1, s1 = oracle.search(b2, a2, e2, q, 10, 48, depth)
        assert np.array_equal(old[i1], i0) and np.array_equal(d1, d0) and np.array_equal(s1, s0)


def test_spatial_order_relabels_and_groups_neighbours_in_space():
    """The spatial order is a permutation that relabels rows, codes and ids
    consistently, is deterministic, and puts points that are close in space
    into the same 128-node leaves: within a leaf the mean squared distance is
    a fraction of that between random points, and a point's nearest
    neighbour shares its leaf far more often than chance."""
    rng = np.random.default_rng(7)
    n, R = 5000, 8
    centres = rng.integers(0, 256, (40, 16))
    base = np.clip(centres[rng.integers(0, 40, n)] + rng.normal(0, 12, (n, 16)), 0, 255).astype(np.uint8)
    adj = rng.integers(0, n, (n, R)).astype(np.int32)
    adj[rng.random((n, R)) < 0.2] = -1
    codes = rng.integers(0, 256, (n, 4)).astype(np.uint8)
    b2, a2, e2, c2, old = ann.reorder_graph(base, adj, 123, codes, order="spatial")
    assert np.array_equal(np.sort(old), np.arange(n))
    pos = np.empty(n, np.int64)
    pos[old] = np.arange(n)
    assert e2 == pos[123]
    assert np.array_equal(b2, base[old]) and np.array_equal(c2, codes[old])
    assert np.array_equal(a2, np.where(adj[old] >= 0, pos[np.maximum(adj[old], 0)], -1))
    again = ann.reorder_graph(base, adj, 123, codes, order="spatial")
    assert np.array_equal(again[4], old)
    x = b2.astype(np.float64)
    leaf = np.arange(n) // 128
    within = np.mean([((x[leaf == l] - x[leaf == l].mean(0)) ** 2).sum(1).mean() for l in range(leaf.max())])
    overall = ((x - x.mean(0)) ** 2).sum(1).mean()
    assert within < 0.25 * overall
    sample = rng.choice(n, 300, replace=False)
    dd = ((x[sample][:, None, :] - x[None, :, :]) ** 2).sum(-1)
    dd[np.arange(300), sample] = np.inf
    nn = dd.argmin(1)
    same_leaf = np.mean(leaf[sample] == leaf[nn])
    assert same_leaf > 0.3 and same_leaf > 10 * (128 / n)
    # an unknown order is rejected
    import ctypes
    e_out = ctypes.c_int32(0)
    rc = ann._lib().ann_reorder_graph_ex(ann._p(base), 0, n, 16, R, ann._p(adj), 0, None, 0, 7,
                                         ann._p(b2.copy()), ann._p(a2.copy()), None, ann._p(old.copy()),
                                         ctypes.byref(e_out))
    assert rc == ann._abi.ANN_EINVAL and b"unknown order" in ann._lib().ann_last_error()


def test_index_file_keeps_the_id_map(tmp_path):
    rng = np.random.default_rng(1)
    n = 500
    base = rng.integers(0, 256, (n, 64)).astype(np.uint8)
    adj = rng.integers(0, n, (n, 8)).astype(np.int32)
    cb = rng.integers(0, 256, (16, 256, 4)).astype(np.float32)
    codes = rng.integers(0, 256, (n, 16)).astype(np.uint8)
    labels = (np.arange(n) * 7 + 3).astype(np.int32)
    p0, p1 = str(tmp_path / "a.idx"), str(tmp_path / "b.idx")
    ann.save_index(p0, base, adj, 0, cb, codes)
    ann.save_index(p1, base, adj, 0, cb, codes, id_map=labels)
    h0, h1 = open(p0, "rb").read(), open(p1, "rb").read()
    assert len(h1) == len(h0) + 4 * n
    assert np.frombuffer(h0[36:40], np.int32)[0] == 0 and np.frombuffer(h1[36:40], np.int32)[0] == 1
    assert np.array_equal(np.frombuffer(h1[-4 * n:], np.int32), labels)
