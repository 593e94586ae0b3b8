"""The continuous-batching request loop (ann_serve_*).

Requests of uneven size, k and L are admitted while others run; every
request's results must equal those of the same queries searched alone (the
batch call with the same k, L and depth), and a sample must equal the oracle.
"""
import threading
import time

import numpy as np
import pytest

import datagen
import oracle
import paper_2507_10070_b300 as ann

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served():
    mx = datagen.sift_like()
    base, q = mx.base(20_000), mx.queries(2000)
    cb, codes = ann.build_pq(base, 32, n_train=5000, iters=5,
                             kpp_uniforms=datagen.kmeanspp_uniforms(mx.seed, 32))
    adj, entry = ann.build_graph(base, 64, 1.2, 64, seed=mx.seed)
    ix = ann.Index(base, adj, entry, cb, codes, tier=ann.ANN_TIER_HOST_PINNED)
    yield dict(ix=ix, base=base, q=q, cb=cb, codes=codes, adj=adj, entry=entry)
    ix.close()


def _mixed_requests(q, seed):
    rng = np.random.default_rng(seed)
    reqs, pos = [], 0
    while pos < q.shape[0]:
        nq = int(min(q.shape[0] - pos, np.exp(rng.uniform(0, np.log(300)))))
        k = int(rng.choice([10, 100]))
        L = int(rng.choice([100, 128, 256]))
        reqs.append((pos, nq, k, L))
        pos += nq
    return reqs


def test_results_same_alone_and_in_the_mix(served):
    ix, q = served["ix"], served["q"]
    srv = ann.Server(ix, max_L=256, max_k=100, depth=1, slots=4096)
    try:
        reqs = _mixed_requests(q, 1)
        ids = [srv.submit(q[p:p + n], k, L) for p, n, k, L in reqs]   # all in flight at once
        out = {}
        deadline = time.time() + 60
        while len(out) < len(ids) and time.time() < deadline:
            for rid in srv.ready(100_000):          # completed, not yet collected
                assert rid in ids and rid not in out
                out[rid] = srv.poll(rid, 0)
        assert len(out) == len(ids)
        assert srv.ready(0) == []
        for rid, (p, n, k, L) in zip(ids, reqs):
            ref_ids, ref_d, _ = ix.search(q[p:p + n], k, L, 1)            # alone
            got_ids, got_d, info = out[rid]
            assert np.array_equal(got_ids, ref_ids) and np.array_equal(got_d, ref_d)
            assert info.queries == n and info.n_failed == 0
        # a sample against the oracle (uint8: bit-exact)
        p, n, k, L = reqs[0]
        oi, od, _ = oracle.search(served["base"], served["adj"], served["entry"], q[p:p + n], k, L, 1,
                                  codebook=served["cb"], codes=served["codes"])
        assert np.array_equal(out[ids[0]][0], oi)
        assert np.array_equal(out[ids[0]][1].astype(np.float64), od)
    finally:
        srv.close()


def test_admission_by_free_slots(served):
    ix, q = served["ix"], served["q"]
    srv = ann.Server(ix, max_L=128, max_k=10, depth=1, slots=64)
    try:
        a = srv.submit(q[:50], 10, 128)
        with pytest.raises(ann.AnnError) as e:
            srv.submit(q[50:70], 10, 128)                  # 20 > 14 free slots
        assert e.value.status == ann._abi.ANN_EBUSY
        assert srv.poll(a, 10_000_000) is not None         # frees the 50 slots
        b = srv.submit(q[50:70], 10, 128)
        assert srv.poll(b, 10_000_000) is not None
        with pytest.raises(ann.AnnError):
            srv.submit(q[:2], 11, 128)                     # k above max_k
        with pytest.raises(ann.AnnError):
            srv.submit(q[:2], 10, 129)                     # L above max_L
    finally:
        srv.close()


def test_idle_exit_and_relaunch(served):
    ix, q = served["ix"], served["q"]
    srv = ann.Server(ix, max_L=128, max_k=10, depth=1, slots=256, idle_exit_us=1000)
    try:
        r = srv.submit(q[:32], 10, 64)
        first = srv.poll(r, 10_000_000)
        time.sleep(0.1)                                     # the kernel returns when idle
        st = srv.stats()
        assert st.running == 0 and st.launches == 1
        r = srv.submit(q[:32], 10, 64)
        again = srv.poll(r, 10_000_000)
        assert srv.stats().launches == 2
        assert np.array_equal(first[0], again[0]) and np.array_equal(first[1], again[1])
    finally:
        srv.close()


def test_served_results_carry_the_id_map(served):
    ix, q = served["ix"], served["q"]
    n = served["base"].shape[0]
    labels = (n - 1 - np.arange(n)).astype(np.int32)
    ixm = ann.Index(served["base"], served["adj"], served["entry"], served["cb"], served["codes"],
                    tier=ann.ANN_TIER_HOST_PINNED, id_map=labels)
    srv = ann.Server(ixm, max_L=128, max_k=10, depth=1, slots=256)
    try:
        got_i, got_d, _ = srv.poll(srv.submit(q[:64], 10, 96), 10_000_000)
    finally:
        srv.close()
        ixm.close()
    ref_i, ref_d, _ = ix.search(q[:64], 10, 96, 1)
    assert np.array_equal(got_i, np.where(ref_i >= 0, labels[np.maximum(ref_i, 0)], -1))
    assert np.array_equal(got_d, ref_d)


def test_concurrent_submitters(served):
    ix, q = served["ix"], served["q"]
    srv = ann.Server(ix, max_L=256, max_k=10, depth=2, slots=2048)
    errors, results = [], {}

    def client(c):
        try:
            for j in range(6):
                lo = (c * 6 + j) * 40
                rid = srv.submit(q[lo:lo + 40], 10, 96 + 32 * (j % 3))
                results[(c, j)] = srv.poll(rid, 30_000_000)
        except Exception as ex:  # noqa: BLE001
            errors.append(ex)

    try:
        th = [threading.Thread(target=client, args=(c,)) for c in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        assert not errors
        for (c, j), (got, gd, _) in results.items():
            lo = (c * 6 + j) * 40
            ref, rd, _ = ix.search(q[lo:lo + 40], 10, 96 + 32 * (j % 3), 2)
            assert np.array_equal(got, ref) and np.array_equal(gd, rd)
    finally:
        srv.close()
