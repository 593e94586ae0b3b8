"""Index-construction tooling of the library (host threads) against the oracle."""
import numpy as np

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
