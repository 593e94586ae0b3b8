"""Full-size parity: the out-of-core workload the benchmark times (1,000,000
SIFT-like uint8 vectors, 10,000 queries, Vamana R=64, PQ M=32, node blocks in
host pinned memory), searched by the CUDA kernel for the whole batch in the
benchmark's launch configuration; a sample of queries is recomputed one by one
by the oracle and must match bit-exactly (ids, distances, step counts).

The index (graph, codebook, codes) comes from the library's host-side
construction tooling (ann_build_graph / ann_build_pq, plain C++ threads, no
GPU); it is input data for both sides and is cached under _data/.  It is
the index the benchmark times (its default builder); L=1280 is the
benchmark's operating point on it, timed at depths 0, 1 and 2 with one or
more warps per query (the benchmark keeps the fastest).
"""
import numpy as np
import pytest

import oracle
import paper_2507_10070_b300 as ann

pytestmark = pytest.mark.gpu

SAMPLE = np.r_[0:40, 4990:5000, 9950:10000]   # head, middle and ragged tail of the batch


@pytest.fixture(scope="module")
def sift1m():
    import bench
    w = bench.prepare_sift_like(1_000_000, 10_000, builder="cpu")
    ix = ann.Index(w["base"], w["adj"], w["entry"], w["cb"], w["codes"],
                   tier=ann.ANN_TIER_HOST_PINNED)
    yield w, ix
    ix.close()


@pytest.mark.parametrize("L,depth,wpq", [(1280, 2, 1), (1280, 2, 4), (1280, 1, 1), (1280, 0, 1),
                                          (1536, 1, 1), (128, 4, 1)])
def test_full_batch_sampled_against_oracle(sift1m, L, depth, wpq):
    import torch
    w, ix = sift1m
    ix.set_warps_per_query(wpq)
    nq, k = w["q"].shape[0], 10
    q = torch.from_numpy(w["q"]).cuda()
    ids = torch.empty((nq, k), dtype=torch.int32, device="cuda")
    dists = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    steps = torch.empty(nq, dtype=torch.int32, device="cuda")
    st = torch.cuda.Stream()
    ix.search_dev(q, k, L, depth, ids, dists, stream=st, trace={"steps": steps})
    stats = ix.sync(st)
    ix.set_warps_per_query(1)
    assert stats.n_failed == 0
    ids, dists, steps = ids.cpu().numpy(), dists.cpu().numpy(), steps.cpu().numpy()
    oi, od, os_ = oracle.search(w["base"], w["adj"], w["entry"], w["q"][SAMPLE], k, L, depth,
                                codebook=w["cb"], codes=w["codes"])
    assert np.array_equal(ids[SAMPLE], oi)
    assert np.array_equal(dists[SAMPLE].astype(np.float64), od)
    assert np.array_equal(steps[SAMPLE], os_)
    # properties that hold for every query of the batch
    assert np.all(ids >= 0) and np.all(np.diff(dists, axis=1) >= 0)
    assert np.all(steps >= k) and stats.expansions == int(steps.sum())
