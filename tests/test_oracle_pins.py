"""Hand-worked pins for the oracle's remaining free steps, and proof that each
pin catches the mistake it is meant to catch.

* k-means++ seeding of the PQ trainer (Arthur & Vassilvitskii 2007: each new
  centre is drawn with probability proportional to D(x)^2): 1-d points whose
  squared distances sum to a power of two, so the boundary draws are exact.
* The empty-cluster rule of the Lloyd iterations (the cluster takes the point
  farthest from its own centroid, lowest id on ties, each point used once).
* The relaxed schedule at depth 2 and 4 (Section "Dependency Relaxed
  Strategy"), traced by hand in tests/golden/search_tree9.json.

The mutation tests compile copies of oracle.c with one planted mistake each
(on the CPU, in a temporary directory) and check that the pins above fail on
them while the committed oracle passes.
"""
import importlib.util
import json
import os
import shutil

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ORACLE_DIR = os.path.dirname(oracle.__file__)


def _load_tree9():
    with open(os.path.join(GOLDEN, "search_tree9.json")) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# k-means++ seeding, worked by hand
# --------------------------------------------------------------------------

KPP_X = [0, 1, 2, 7, 9, 11]


def kpp_case(orc):
    """Subspace 0: x = [0, 1, 2, 7, 9, 11], u = [0, 54/256, 0.1].
      centre 0: point floor(0 * 6) = 0 (x = 0).
      D^2 to {0}:     [0, 1, 4, 49, 81, 121], total 256, running sums
                      [0, 1, 5, 54, 135, 256].
      centre 1: target 54/256 * 256 = 54 exactly; the first running sum
                strictly above 54 is 135 -> point 4 (x = 9).  (A ">=" rule
                would stop at 54 -> x = 7; sampling on D instead of D^2
                has running sums [0, 1, 3, 10, 19, 30], target 6.33 -> x = 7.)
      D^2 to {0, 9}:  [0, 1, 4, 4, 0, 4], total 13, running [0, 1, 5, 9, 9, 13].
      centre 2: target 0.1 * 13 = 1.3 -> first sum above it is 5 -> point 2
                (x = 2).  (On D: [0, 1, 2, 2, 0, 2], target 0.7 -> x = 1.)
    Subspace 1: x = [7, 9, 11, 0, 1, 2], u = [0.5, 0.51, 0]:
      centre 0: point floor(0.5 * 6) = 3 (x = 0).
      D^2: [49, 81, 121, 0, 1, 4], total 256, running [49, 130, 251, ...];
      centre 1: target 0.51 * 256 = 130.56 -> point 2 (x = 11).
                (On D: [7, 9, 11, 0, 1, 2], running [7, 16, 27, ...],
                target 15.3 -> x = 9.)
      D^2 to {0, 11}: [16, 4, 0, 0, 1, 4]; centre 2: target 0 -> the first
                running sum above 0 is 16 -> point 0 (x = 7).
    Returns the seeds of K = 2 and K = 3 (no Lloyd iteration)."""
    x = np.array([[a, b] for a, b in zip(KPP_X, [7, 9, 11, 0, 1, 2])], np.uint8)
    u3 = np.array([[0.0, 54.0 / 256.0, 0.1], [0.5, 0.51, 0.0]])
    cb3 = orc.pq_train(x, 2, u3, iters=0, K=3)
    cb2 = orc.pq_train(x, 2, u3[:, :2], iters=0, K=2)
    return cb2[:, :, 0].tolist(), cb3[:, :, 0].tolist()


KPP_WANT = ([[0.0, 9.0], [0.0, 11.0]], [[0.0, 9.0, 2.0], [0.0, 11.0, 7.0]])


def test_kmeanspp_seeding_hand_worked():
    got2, got3 = kpp_case(oracle)
    assert got2 == KPP_WANT[0]
    assert got3 == KPP_WANT[1]


# --------------------------------------------------------------------------
# empty clusters, worked by hand
# --------------------------------------------------------------------------

def empty_after_update_case(orc):
    """x = [9, 10, 11, 18, 19, 27] (1-d), K = 3, u = [0, 0.5, 0], 2 iterations.
    Seeding: centre 0 = x[0] = 9; D^2 = [0, 1, 4, 81, 100, 324] (total 510,
    running [0, 1, 5, 86, 186, 510]); target 255 -> point 5 (27);
    D^2 = [0, 1, 4, 81, 64, 0] (running [0, 1, 5, 86, 150, 150]), target 0
    -> point 1 (10).  Centres [9, 27, 10].
    Iteration 0: 9 -> c0; 10, 11, 18 -> c2; 19, 27 -> c1.  Means [9, 23, 13].
    Iteration 1: 9, 10 -> c0; 11 is 2 from both c0 and c2 -> c0 (lower
    index); 18 is 5 from both c1 and c2 -> c1; 19, 27 -> c1.  Cluster 2 is
    empty.  Squared distances to the own centroid: [0, 1, 4, 25, 16, 16];
    the farthest point is x = 18 (25), so centre 2 becomes 18.  Means of the
    others: c0 = (9+10+11)/3 = 10, c1 = (18+19+27)/3 = 64/3.
    Returns the final centroids unrounded and rounded half to even."""
    x = np.array([[9], [10], [11], [18], [19], [27]], np.uint8)
    u = np.array([[0.0, 0.5, 0.0]])
    raw = orc.pq_train(x, 1, u, iters=2, K=3, round_int=False)
    rounded = orc.pq_train(x, 1, u, iters=2, K=3)
    return raw[0, :, 0].tolist(), rounded[0, :, 0].tolist()


def two_empty_clusters_case(orc):
    """x = [5, 6, 9, 9, 9] (1-d), K = 5, u = [0, 0.9, 0.5, 0.5, 0.7], 1 iteration.
    Seeding: centre 0 = 5; D^2 = [0, 1, 16, 16, 16] (total 49, running
    [0, 1, 17, 33, 49]), target 44.1 -> point 4 (9); D^2 = [0, 1, 0, 0, 0],
    target 0.5 -> point 1 (6); now every D^2 is 0, so centre 3 is point
    floor(0.5 * 5) = 2 (9) and centre 4 is point floor(0.7 * 5) = 3 (9).
    Centres [5, 9, 6, 9, 9].
    Iteration 0: 5 -> c0; 6 -> c2; each 9 ties between c1, c3, c4 -> c1.
    Clusters 3 and 4 are empty and every point sits on its centroid (all
    squared distances 0).  Centre 3 takes the lowest id of the farthest
    points, point 0 (5), which is then used; centre 4 takes the next, point 1
    (6).  Result [5, 9, 6, 5, 6]."""
    x = np.array([[5], [6], [9], [9], [9]], np.uint8)
    u = np.array([[0.0, 0.9, 0.5, 0.5, 0.7]])
    return oracle_cb(orc, x, u)


def oracle_cb(orc, x, u):
    return orc.pq_train(x, 1, u, iters=1, K=5)[0, :, 0].tolist()


def test_empty_cluster_takes_farthest_point_hand_worked():
    raw, rounded = empty_after_update_case(oracle)
    assert raw == [10.0, float(np.float32(64.0 / 3.0)), 18.0]
    assert rounded == [10.0, 21.0, 18.0]


def test_two_empty_clusters_lowest_id_each_point_once():
    assert two_empty_clusters_case(oracle) == [5.0, 9.0, 6.0, 5.0, 6.0]


# --------------------------------------------------------------------------
# relaxed schedule at depth 2 and 4, traced by hand
# --------------------------------------------------------------------------

def tree9_traces(orc):
    g = _load_tree9()
    base = np.array(g["vectors"], np.uint8)
    adj = np.array(g["adjacency"], np.int32)
    q = np.array([g["query"]], np.uint8)
    out = {}
    for c in g["cases"]:
        ids, d, steps, trace = orc.search(base, adj, g["entry"], q, g["k"], g["L"], c["depth"],
                                          trace_cap=16)
        out[c["depth"]] = (trace[0, :steps[0]].tolist(), int(steps[0]), ids[0].tolist(),
                           d[0].tolist())
    return out


@pytest.mark.parametrize("depth", [0, 1, 2, 4])
def test_search_hand_traced_tree(depth):
    g = _load_tree9()
    base = np.array(g["vectors"], np.uint8)
    q = np.array(g["query"], np.uint8)
    for i, v in g["distances_by_hand"].items():
        assert oracle.l2(base[int(i)], q) == v
    case = next(c for c in g["cases"] if c["depth"] == depth)
    expanded, steps, ids, dists = tree9_traces(oracle)[depth]
    assert expanded == case["expanded"]
    assert steps == case["steps"]
    assert ids == case["ids"] and dists == case["dists"]


def _tree9_matches(orc):
    g = _load_tree9()
    got = tree9_traces(orc)
    return all(got[c["depth"]][0] == c["expanded"] for c in g["cases"])


# --------------------------------------------------------------------------
# planted mistakes: each must break a pin above
# --------------------------------------------------------------------------

def _mutant(tmp_path, replacements):
    """A copy of the oracle package with `replacements` applied to oracle.c,
    compiled into tmp_path and loaded as a separate module."""
    with open(os.path.join(ORACLE_DIR, "oracle.c")) as f:
        src = f.read()
    for old, new in replacements:
        assert src.count(old) == 1, f"pattern not found once in oracle.c: {old!r}"
        src = src.replace(old, new)
    d = tmp_path / "oracle_mutant"
    d.mkdir()
    (d / "oracle.c").write_text(src)
    shutil.copy(os.path.join(ORACLE_DIR, "__init__.py"), d / "__init__.py")
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{abs(hash(str(d)))}",
                                                  d / "__init__.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


MUTATIONS = {
    "kpp_samples_on_D": [("total += D2[i];", "total += sqrt(D2[i]);"),
                         ("run += D2[i];", "run += sqrt(D2[i]);")],
    "kpp_greater_or_equal": [("if (run > target) {", "if (run >= target) {")],
    "empty_takes_nearest": [("if (adist[i] > fd) {", "if (adist[i] >= 0.0 && (fd < 0.0 || adist[i] < fd)) {")],
    "empty_ties_to_highest_id": [("if (adist[i] > fd) {", "if (adist[i] >= fd) {")],
    "empty_reuses_points": [("adist[far] = -2.0; /* used */", "/* not marked */")],
    "fetch_lifo": [("int32_t u = fifo[fhead];\n      fhead = (fhead + 1) % (D + 1);",
                    "int32_t u = fifo[(fhead + fcount - 1) % (D + 1)];")],
    "depth_off_by_one": [("if (fcount > D || (v < 0 && fcount > 0)) {",
                          "if (fcount > D + 1 || (v < 0 && fcount > 0)) {")],
    "ring_too_small": [("fifo[(fhead + fcount) % (D + 1)] = list[v].key.id;",
                        "fifo[(fhead + fcount) % (D > 1 ? D : 1)] = list[v].key.id;"),
                       ("fhead = (fhead + 1) % (D + 1);", "fhead = (fhead + 1) % (D > 1 ? D : 1);")],
}


def _pins_hold(orc):
    """Every hand-worked pin of this file, evaluated on `orc`."""
    got2, got3 = kpp_case(orc)
    kpp_ok = got2 == KPP_WANT[0] and got3 == KPP_WANT[1]
    raw, rounded = empty_after_update_case(orc)
    empty_ok = (raw == [10.0, float(np.float32(64.0 / 3.0)), 18.0] and rounded == [10.0, 21.0, 18.0]
                and two_empty_clusters_case(orc) == [5.0, 9.0, 6.0, 5.0, 6.0])
    return {"kpp": kpp_ok, "empty": empty_ok, "schedule": _tree9_matches(orc)}


EXPECTED_BREAK = {
    "kpp_samples_on_D": "kpp",
    "kpp_greater_or_equal": "kpp",
    "empty_takes_nearest": "empty",
    "empty_ties_to_highest_id": "empty",
    "empty_reuses_points": "empty",
    "fetch_lifo": "schedule",
    "depth_off_by_one": "schedule",
    "ring_too_small": "schedule",
}


def test_pins_hold_on_the_committed_oracle():
    assert _pins_hold(oracle) == {"kpp": True, "empty": True, "schedule": True}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_breaks_its_pin(tmp_path, name):
    mod = _mutant(tmp_path, MUTATIONS[name])
    held = _pins_hold(mod)
    assert not held[EXPECTED_BREAK[name]], f"mutation {name} is not caught by the {EXPECTED_BREAK[name]} pin"
