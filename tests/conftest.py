import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def u8_pq():
    """SIFT-like uint8 index, 20,000 nodes, R=64, PQ M=32, built by the
    oracle (graph, codebook, codes); 333 queries, a ragged tail over the
    grid.  Shared by the GPU parity tests."""
    import datagen
    import oracle
    mx = datagen.sift_like()
    n, nq = 20_000, 333
    base, q = mx.base(n), mx.queries(nq)
    cb = oracle.pq_train(base[:5000], 32, datagen.kmeanspp_uniforms(mx.seed, 32), iters=8)
    codes = oracle.pq_encode(base, cb)
    entry = oracle.medoid(base)
    adj = oracle.vamana(base, 64, 1.2, 96, entry, datagen.build_order(mx.seed, n),
                        datagen.random_out_neighbours(mx.seed, n, 64))
    return dict(base=base, q=q, cb=cb, codes=codes, entry=entry, adj=adj)
