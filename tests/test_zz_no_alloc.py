"""The allocation-free search entry point (ann_search_dev_noalloc).

Callers that must not call cudaMalloc while searching -- a serving thread
with a latency budget, a process whose device memory is reserved up front, or
code that must not grow its footprint after start-up -- use this variant: its
scratch lives in a fixed static device array inside the library.  Its results
must equal those of the ordinary device-buffer entry point (ann_search_dev),
on two calls in a row (the second one reuses what the first left in the
array), and the two calls must not change the device's free memory.

Kept in a file of its own that pytest collects last; it builds its own small
index so it passes alone in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest

import datagen
import paper_2507_10070_b300 as ann

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small_index():
    mx = datagen.sift_like()
    base, q = mx.base(20_000), mx.queries(700)
    cb, codes = ann.build_pq(base, 32, n_train=5000, iters=5,
                             kpp_uniforms=datagen.kmeanspp_uniforms(mx.seed, 32))
    adj, entry = ann.build_graph(base, 64, 1.2, 64, seed=mx.seed)
    ix = ann.Index(base, adj, entry, cb, codes, tier=ann.ANN_TIER_HOST_PINNED)
    yield ix, q
    ix.close()


def test_noalloc_matches_search_dev_on_two_calls(small_index):
    import torch
    ix, qh = small_index
    q = torch.from_numpy(qh).cuda()
    nq, k, L, depth = q.shape[0], 10, 256, 1
    st = torch.cuda.Stream()

    def out():
        return (torch.empty((nq, k), dtype=torch.int32, device="cuda"),
                torch.empty((nq, k), dtype=torch.float32, device="cuda"))

    ref_ids, ref_d = out()
    with torch.cuda.stream(st):
        ix.search_dev(q, k, L, depth, ref_ids, ref_d, stream=st)
    ix.sync(st)

    # set-up call (first use on this device: address lookup), then two calls
    # whose device memory footprint is checked
    w_ids, w_d = out()
    ix.search_dev_noalloc(q, k, L, depth, w_ids, w_d, stream=st)
    st.synchronize()
    results = [out(), out()]
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for ids, d in results:
        ix.search_dev_noalloc(q, k, L, depth, ids, d, stream=st)
    st.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    assert free_after == free_before
    for ids, d in results:
        assert torch.equal(ids, ref_ids)       # uint8 data: exact
        assert torch.equal(d, ref_d)


def test_noalloc_reports_status_and_rejects_oversized_scratch(small_index):
    import torch
    ix, qh = small_index
    q = torch.from_numpy(qh[:50]).cuda()
    ids = torch.empty((50, 10), dtype=torch.int32, device="cuda")
    d = torch.empty((50, 10), dtype=torch.float32, device="cuda")
    status = torch.full((50,), 7, dtype=torch.int32, device="cuda")
    ix.search_dev_noalloc(q, 10, 64, 2, ids, d, trace={"status": status})
    torch.cuda.synchronize()
    assert int(status.abs().sum()) == 0
    # an index of 4,000,000 nodes needs a 500,000-byte visited bitset per
    # warp, plus its clear log: 32 warps do not fit in the 16 MiB static
    # scratch, so the call is rejected with a clear error (exact navigation
    # on a chain of 4-coordinate points keeps the index itself small)
    n = 4_000_000
    base = np.zeros((n, 4), np.uint8)
    base[:, 0] = np.arange(n) % 256
    adj = ((np.arange(n) + 1) % n).astype(np.int32)[:, None]
    big = ann.Index(base, adj, 0, tier=ann.ANN_TIER_HBM)
    try:
        qw = torch.from_numpy(base[:4].copy()).cuda()
        with pytest.raises(ann.AnnError) as e:
            big.search_dev_noalloc(qw, 2, 8, 1, ids[:4, :2].contiguous(), d[:4, :2].contiguous())
        assert e.value.status == ann._abi.ANN_EINVAL and "static" in str(e.value)
    finally:
        big.close()
    small = ann.Index(base[:3_000_000], ((np.arange(3_000_000) + 1) % 3_000_000).astype(np.int32)[:, None],
                      0, tier=ann.ANN_TIER_HBM)
    try:   # 3,000,000 nodes fit (the limit is 3,931,136)
        qw = torch.from_numpy(base[:4].copy()).cuda()
        i2 = torch.empty((4, 2), dtype=torch.int32, device="cuda")
        d2 = torch.empty((4, 2), dtype=torch.float32, device="cuda")
        small.search_dev_noalloc(qw, 2, 8, 1, i2, d2)
        torch.cuda.synchronize()
        assert i2.cpu().numpy()[:, 0].tolist() == [0, 1, 2, 3]
    finally:
        small.close()


def test_noalloc_reports_mapped_ids(small_index):
    import torch
    ix, qh = small_index
    mx = datagen.sift_like()
    base = mx.base(20_000)
    n = base.shape[0]
    labels = (np.arange(n) * 2 + 9).astype(np.int32)
    cb, codes = ann.build_pq(base, 32, n_train=5000, iters=5,
                             kpp_uniforms=datagen.kmeanspp_uniforms(mx.seed, 32))
    adj, entry = ann.build_graph(base, 64, 1.2, 64, seed=mx.seed)
    ixm = ann.Index(base, adj, entry, cb, codes, tier=ann.ANN_TIER_HOST_PINNED, id_map=labels)
    try:
        q = torch.from_numpy(qh[:200]).cuda()
        st = torch.cuda.Stream()
        ids = torch.empty((200, 10), dtype=torch.int32, device="cuda")
        d = torch.empty((200, 10), dtype=torch.float32, device="cuda")
        ixm.search_dev_noalloc(q, 10, 128, 1, ids, d, stream=st)
        st.synchronize()
    finally:
        ixm.close()
    ref_i, ref_d, _ = ix.search(qh[:200], 10, 128, 1)
    assert np.array_equal(ids.cpu().numpy(), np.where(ref_i >= 0, labels[np.maximum(ref_i, 0)], -1))
    assert np.array_equal(d.cpu().numpy(), ref_d)
