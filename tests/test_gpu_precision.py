"""Precision variants: navigation on BF16, FP8-E4M3 and 48-byte float-PQ
copies of float32 vectors (FP32 accumulation), then an exact FP32 rerank of
the top 4k expanded candidates -- against the oracle navigating on the same
decoded values in float64 and reranking the same way.

float32 arithmetic on the device against float64 in the oracle: distances of
matching ids within 1e-5 relative, a differing id only where the oracle's
distances at that rank agree within 1e-5, recall@10 within 0.002."""
import numpy as np
import pytest

import datagen
import oracle
import paper_2507_10070_b300 as ann

pytestmark = pytest.mark.gpu
REL = 1e-5


@pytest.fixture(scope="module")
def deep():
    mx = datagen.deep_like()
    base, q = mx.base(20_000), mx.queries(300)
    adj, entry = ann.build_graph(base, 48, 1.2, 96, seed=mx.seed, device="cpu")
    cb, codes = ann.build_pq(base, 48, n_train=8000, iters=8,
                             kpp_uniforms=datagen.kmeanspp_uniforms(mx.seed, 48))
    gi, gd = oracle.knn(base, q, 10)
    return dict(base=base, q=q, adj=adj, entry=entry, cb=cb, codes=codes, gi=gi, gd=gd)


def _compare(ids, d, oi, od, gi, gd):
    same = ids == oi
    assert np.all(np.abs(d[same] - od[same]) <= REL * np.maximum(od[same], 1e-30))
    diff = ~same
    if diff.any():
        assert np.all(np.abs(d[diff] - od[diff]) <= REL * od[diff])
    r_gpu = ann.recall_at_k(ids, gi, gd, d)
    r_orc = oracle.recall_at_k(oi, gi, gd, od)
    assert abs(r_gpu - r_orc) <= 0.002
    return r_gpu


@pytest.mark.parametrize("variant", ["bf16", "fp8", "pq48"])
@pytest.mark.parametrize("depth", [0, 1])
def test_precision_variant_matches_oracle(deep, variant, depth):
    w = deep
    k, L = 10, 64
    if variant == "bf16":
        ix = ann.Index(w["base"], w["adj"], w["entry"], tier=ann.ANN_TIER_HBM, nav=ann.ANN_NAV_BF16)
        nav = oracle.decode_bf16(ann.encode_bf16(w["base"]))
        kw = dict(nav_vectors=nav)
    elif variant == "fp8":
        ix = ann.Index(w["base"], w["adj"], w["entry"], tier=ann.ANN_TIER_HBM, nav=ann.ANN_NAV_FP8,
                       nav_scale=64.0)
        nav = oracle.decode_fp8e4m3(ann.encode_fp8e4m3(w["base"], 64.0), 64.0)
        kw = dict(nav_vectors=nav)
    else:
        ix = ann.Index(w["base"], w["adj"], w["entry"], w["cb"], w["codes"], tier=ann.ANN_TIER_HBM)
        kw = dict(codebook=w["cb"], codes=w["codes"])
    try:
        ids, d, _ = ix.search(w["q"], k, L, depth)
    finally:
        ix.close()
    oi, od, _ = oracle.search(w["base"], w["adj"], w["entry"], w["q"], k, L, depth, rerank=4 * k, **kw)
    r = _compare(ids, d, oi, od, w["gi"], w["gd"])
    assert r > 0.8
    # distances are exact FP32 L2 of the returned ids: against float64
    x = w["base"][np.maximum(ids, 0)].astype(np.float64)
    d64 = ((x - w["q"][:, None, :].astype(np.float64)) ** 2).sum(-1)
    assert np.all(np.abs(d - d64)[ids >= 0] <= 1e-5 * d64[ids >= 0] + 1e-7)


def test_rerank_reports_mapped_ids(deep):
    n = deep["base"].shape[0]
    labels = (np.arange(n) * 5 + 1).astype(np.int32)
    a = ann.Index(deep["base"], deep["adj"], deep["entry"], tier=ann.ANN_TIER_HBM, nav=ann.ANN_NAV_BF16)
    b = ann.Index(deep["base"], deep["adj"], deep["entry"], tier=ann.ANN_TIER_HBM, nav=ann.ANN_NAV_BF16,
                  id_map=labels)
    try:
        ai, ad, _ = a.search(deep["q"], 10, 64, 1)
        bi, bd, _ = b.search(deep["q"], 10, 64, 1)
    finally:
        a.close()
        b.close()
    assert np.array_equal(bi, np.where(ai >= 0, labels[np.maximum(ai, 0)], -1))
    assert np.array_equal(bd, ad)


def test_fp32_navigation_is_the_reference(deep):
    """The FP32 traversal (exact navigation) that the variants are compared with."""
    w = deep
    ix = ann.Index(w["base"], w["adj"], w["entry"], tier=ann.ANN_TIER_HBM)
    try:
        ids, d, _ = ix.search(w["q"], 10, 64, 1)
    finally:
        ix.close()
    oi, od, _ = oracle.search(w["base"], w["adj"], w["entry"], w["q"], 10, 64, 1)
    _compare(ids, d, oi, od, w["gi"], w["gd"])


def test_precision_modes_are_rejected_where_no_rerank_runs(deep):
    import torch
    w = deep
    ix = ann.Index(w["base"], w["adj"], w["entry"], tier=ann.ANN_TIER_HBM, nav=ann.ANN_NAV_BF16)
    try:
        with pytest.raises(ann.AnnError):
            ann.Server(ix, max_L=64, max_k=10)
        q = torch.from_numpy(w["q"][:4]).cuda()
        out = torch.empty((4, 10), dtype=torch.int32, device="cuda")
        dd = torch.empty((4, 10), dtype=torch.float32, device="cuda")
        with pytest.raises(ann.AnnError):
            ix.search_dev_noalloc(q, 10, 64, 1, out, dd)
    finally:
        ix.close()
