"""GPU Vamana construction (ann_build_graph_gpu): graph invariants,
determinism, and search quality against the host builder."""
import collections

import numpy as np
import pytest

import datagen
import oracle
import paper_2507_10070_b300 as ann

pytestmark = pytest.mark.gpu


def _check_rows(adj, R):
    assert adj.shape[1] == R
    for i, row in enumerate(adj):
        nb = row[row >= 0]
        assert np.all(row[len(nb):] == -1)
        assert i not in nb and len(set(nb.tolist())) == len(nb)


def _reach(adj, s):
    seen = np.zeros(adj.shape[0], bool)
    seen[s] = True
    dq = collections.deque([s])
    while dq:
        u = dq.popleft()
        for w in adj[u]:
            if w >= 0 and not seen[w]:
                seen[w] = True
                dq.append(w)
    return int(seen.sum())


def test_gpu_build_u8_matches_host_quality():
    mx = datagen.sift_like()
    base, q = mx.base(30_000), mx.queries(300)
    g_adj, g_entry = ann.build_graph(base, 64, 1.2, 128, seed=5, device="gpu")
    h_adj, h_entry = ann.build_graph(base, 64, 1.2, 128, seed=5, device="cpu")
    assert g_entry == h_entry == oracle.medoid(base)
    _check_rows(g_adj, 64)
    assert _reach(g_adj, g_entry) >= 0.999 * base.shape[0]
    again, _ = ann.build_graph(base, 64, 1.2, 128, seed=5, device="gpu")
    assert np.array_equal(g_adj, again)                      # deterministic
    gi, gd = oracle.knn(base, q, 10)
    for L in (32, 64):
        ig, dg, _ = oracle.search(base, g_adj, g_entry, q, 10, L, 0)
        ih, dh, _ = oracle.search(base, h_adj, h_entry, q, 10, L, 0)
        rg = oracle.recall_at_k(ig, gi, gd, dg)
        rh = oracle.recall_at_k(ih, gi, gd, dh)
        assert rg >= rh - 0.01, (L, rg, rh)


def test_gpu_build_f32_inmemory_workload():
    mx = datagen.inmemory_f32()
    base, q = mx.base(10_000), mx.queries(200)
    adj, entry = ann.build_graph(base, 32, 1.2, 64, seed=1, device="gpu")
    _check_rows(adj, 32)
    gi, gd = oracle.knn(base, q, 10)
    ids, d, _ = oracle.search(base, adj, entry, q, 10, 64, 0)
    assert oracle.recall_at_k(ids, gi, gd, d) >= 0.95


def test_gpu_build_degree_96_matches_host_quality():
    """R = 96 (the degree selector's pick on some samples): rows of up to 96
    ids, reachability, and search quality within 0.01 of the host builder."""
    mx = datagen.sift_like()
    base, q = mx.base(20_000), mx.queries(200)
    g_adj, g_entry = ann.build_graph(base, 96, 1.2, 128, seed=7, device="gpu")
    h_adj, h_entry = ann.build_graph(base, 96, 1.2, 128, seed=7, device="cpu")
    _check_rows(g_adj, 96)
    assert (g_adj >= 0).sum(1).max() > 64                   # rows use the larger degree
    assert _reach(g_adj, g_entry) >= 0.999 * base.shape[0]
    gi, gd = oracle.knn(base, q, 10)
    ig, dg, _ = oracle.search(base, g_adj, g_entry, q, 10, 48, 0)
    ih, dh, _ = oracle.search(base, h_adj, h_entry, q, 10, 48, 0)
    assert oracle.recall_at_k(ig, gi, gd, dg) >= oracle.recall_at_k(ih, gi, gd, dh) - 0.01


def test_gpu_build_rejects_bad_sizes():
    x = np.zeros((100, 8), np.uint8)
    with pytest.raises(ann.AnnError):
        ann.build_graph(x, 16, device="gpu")                 # d % 16 != 0
    with pytest.raises(ann.AnnError):
        ann.build_graph(np.zeros((100, 16), np.uint8), 130, L_build=126, device="gpu")   # R > 128
    with pytest.raises(ann.AnnError):
        ann.build_graph(np.zeros((100, 16), np.uint8), 96, L_build=192, device="gpu")    # L_build > 256 - R


def test_gpu_pq_encoder_equals_host_encoder():
    mx = datagen.sift_like()
    base = mx.base(50_000)
    u = datagen.kmeanspp_uniforms(mx.seed, 32)
    cb, codes = ann.build_pq(base, 32, n_train=5000, iters=4, kpp_uniforms=u)
    cb2, codes2 = ann.build_pq(base, 32, n_train=5000, iters=4, kpp_uniforms=u, encode_device="gpu")
    assert np.array_equal(cb, cb2) and np.array_equal(codes, codes2)


@pytest.mark.parametrize("n,d,R,L_build", [(30_000, 128, 64, 128), (12_000, 128, 96, 128),
                                           (8_000, 64, 32, 96), (6_000, 48, 24, 64)])
def test_gpu_build_tensor_prune_equals_cuda_cores(n, d, R, L_build):
    """RobustPrune with the candidate distances from BF16 MMAs (exact for
    uint8) makes the same decisions as the CUDA-core prune: the graphs are
    identical, row for row.  d = 48 has an odd number of 16-coordinate MMA
    steps; R = 96 fills candidate sets up to 256."""
    if d == 128:
        base = datagen.sift_like().base(n)
    else:
        base = np.random.default_rng(d).integers(0, 256, size=(n, d)).astype(np.uint8)
    t_adj, t_entry = ann.build_graph(base, R, 1.2, L_build, seed=11, device="gpu", engine="tensor")
    c_adj, c_entry = ann.build_graph(base, R, 1.2, L_build, seed=11, device="gpu", engine="cuda")
    assert t_entry == c_entry
    assert np.array_equal(t_adj, c_adj)
    _check_rows(t_adj, R)


def test_gpu_build_tensor_engine_needs_small_uint8():
    x = np.zeros((100, 16), np.float32)
    with pytest.raises(ann.AnnError) as e:
        ann.build_graph(x, 8, 1.2, 16, device="gpu", engine="tensor")
    assert e.value.status == ann._abi.ANN_EINVAL
    y = np.zeros((100, 144), np.uint8)
    with pytest.raises(ann.AnnError) as e:
        ann.build_graph(y, 8, 1.2, 16, device="gpu", engine="tensor")
    assert e.value.status == ann._abi.ANN_EINVAL
