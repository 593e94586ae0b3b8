"""CPU-agent I/O (ann_search_cpu_agent): the paper's mapped request array
served by host threads, as an ablation of the warps reading node blocks
themselves.  Only the data path changes, so ids, distances and expansion
counts equal the oracle's (and so the direct search's), bit for bit.  The
bounded wait is tested with no agent thread at all: a completion word that
nothing writes."""
import numpy as np
import pytest

import oracle
import paper_2507_10070_b300 as ann

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def agent_index(u8_pq):
    w = u8_pq
    ix = ann.Index(w["base"], w["adj"], w["entry"], w["cb"], w["codes"], tier=ann.ANN_TIER_HOST_PINNED)
    yield ix
    ix.close()


@pytest.mark.parametrize("depth", [0, 1, 2, 4])
@pytest.mark.parametrize("threads", [1, 3])
def test_cpu_agent_bit_exact(u8_pq, agent_index, depth, threads):
    k, L = 10, 64
    ids, dists, stats, secs = agent_index.search_cpu_agent(u8_pq["q"], k, L, depth, agent_threads=threads)
    oi, od, osteps = oracle.search(u8_pq["base"], u8_pq["adj"], u8_pq["entry"], u8_pq["q"], k, L, depth,
                                   codebook=u8_pq["cb"], codes=u8_pq["codes"])
    assert np.array_equal(ids, oi)
    assert np.array_equal(dists.astype(np.float64), od)
    assert stats.expansions == int(osteps.sum()) and stats.n_failed == 0
    assert secs > 0
    # the same call through the warps' own reads
    di, dd, ds = agent_index.search(u8_pq["q"], k, L, depth)
    assert np.array_equal(ids, di) and np.array_equal(dists, dd) and ds.expansions == stats.expansions


def test_cpu_agent_wait_runs_out_without_an_agent(u8_pq, agent_index):
    q = u8_pq["q"][:6]
    with pytest.raises(ann.AnnError) as e:
        agent_index.search_cpu_agent(q, 10, 32, 1, agent_threads=0, wait_us=20_000)
    assert e.value.status == ann._abi.ANN_ETIMEOUT
    ids, dists, stats, _ = agent_index.search_cpu_agent(q, 10, 32, 1, agent_threads=0, wait_us=20_000,
                                                        check=False)
    assert stats.n_failed == len(q)
    # the index stays usable, on both paths
    ids, dists, stats, _ = agent_index.search_cpu_agent(q, 10, 32, 1, agent_threads=2)
    di, dd, _ = agent_index.search(q, 10, 32, 1)
    assert np.array_equal(ids, di) and np.array_equal(dists, dd)


def test_cpu_agent_rejects_other_tiers(u8_pq):
    w = u8_pq
    ix = ann.Index(w["base"], w["adj"], w["entry"], w["cb"], w["codes"], tier=ann.ANN_TIER_HBM)
    try:
        with pytest.raises(ann.AnnError) as e:
            ix.search_cpu_agent(w["q"][:4], 10, 32, 1)
        assert e.value.status == ann._abi.ANN_EINVAL
    finally:
        ix.close()
