"""The computation / I/O balanced degree selector (ann_autotune_degree)."""
import numpy as np
import pytest

import paper_2507_10070_b300 as ann

pytestmark = pytest.mark.gpu


def test_degree_selector_follows_its_rule():
    r = ann.autotune_degree(degrees=(32, 64, 96), n_sample=20_000, L=32, nq=512, seed=3)
    t = r["table"]
    assert [p["degree"] for p in t] == [32, 64, 96]
    for p in t:
        assert p["t_compute_us"] > 0 and p["t_fetch_us"] >= 0 and p["qps_sync"] > 0
        # the host-tier step is the HBM-tier step plus the fetch excess (clamped at 0)
        if p["t_fetch_us"] > 0:
            assert abs(p["step_us_sync"] - (p["t_compute_us"] + p["t_fetch_us"])) <= 1e-2 * p["step_us_sync"] + 1e-3
        else:
            assert p["step_us_sync"] <= p["t_compute_us"] * 1.01
    gaps = [abs(p["t_compute_us"] - p["t_fetch_us"]) for p in t]
    assert r["degree"] == t[int(np.argmin(gaps))]["degree"]          # d = argmin |T_c - T_f|
    assert r["depth"] == int(np.argmax(r["qps_by_depth"])) and all(q > 0 for q in r["qps_by_depth"])
    # more neighbours per step cost more computation per step
    assert t[2]["t_compute_us"] > t[0]["t_compute_us"]
    # warps per query: the fastest of 1, 2, 4 at the chosen degree and depth
    wq = r["qps_by_warps_per_query"]
    assert set(wq) == {"1", "2", "4"} and all(v > 0 for v in wq.values())
    assert r["warps_per_query"] == int(max(wq, key=wq.get))
