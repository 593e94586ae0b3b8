"""Brute-force ground truth on the tensor cores (ann_knn_exact_ex, engine
"tensor"): tcgen05 BF16 MMAs with FP32 accumulation, exact for uint8 data,
with the top-k chosen from the accumulator.  Every case is bit-exact against
the oracle's brute force (ids and distances, ties by id), on ragged sizes
(query and base counts that are not multiples of the 128 x 128 tile), padded
dimensions, duplicate points, the largest distances d = 128 allows, more than
one base chunk, and k beyond n."""
import numpy as np
import pytest

import datagen
import oracle
import paper_2507_10070_b300 as ann

pytestmark = pytest.mark.gpu


def _exact(ids, d, oi, od):
    assert np.array_equal(ids, oi)
    assert np.array_equal(d.astype(np.float64), od)


@pytest.mark.parametrize("k", [1, 10, 100, 128])
def test_tensor_knn_sift_like_ragged(k):
    mx = datagen.sift_like()
    base, q = mx.base(7000), mx.queries(150)      # 54 tiles + 88 rows; 1 query tile + 22
    ids, d = ann.knn_exact(base, q, k, engine="tensor")
    _exact(ids, d, *oracle.knn(base, q, k))


@pytest.mark.parametrize("dim", [32, 64, 100, 128])
def test_tensor_knn_padded_dimensions(dim):
    rng = np.random.default_rng(dim)
    base = rng.integers(0, 256, size=(3001, dim)).astype(np.uint8)
    q = rng.integers(0, 256, size=(129, dim)).astype(np.uint8)
    ids, d = ann.knn_exact(base, q, 16, engine="tensor")
    _exact(ids, d, *oracle.knn(base, q, 16))


def test_tensor_knn_ties_and_duplicates():
    rng = np.random.default_rng(5)
    base = rng.integers(0, 3, size=(5000, 128)).astype(np.uint8)   # many equal distances
    base[4000:4100] = base[7]                                         # exact duplicates of one row
    q = np.concatenate([base[[7, 11]], rng.integers(0, 3, size=(60, 128)).astype(np.uint8)])
    ids, d = ann.knn_exact(base, q, 50, engine="tensor")
    _exact(ids, d, *oracle.knn(base, q, 50))


def test_tensor_knn_largest_distances():
    """d = 128 at the ends of the range: every base row is all 255 but one,
    which has a single 254; the query is all 0.  Distances are 128 * 255^2 =
    8,323,200 (the largest d = 128 allows) and 8,323,200 - 509 for the one
    row, so the top-k is that row, then ids 0, 1, ... by the id tie-break."""
    base = np.full((1000, 128), 255, np.uint8)
    base[500, 0] = 254
    rng = np.random.default_rng(9)
    q = np.concatenate([np.zeros((1, 128), np.uint8),
                        (rng.integers(0, 2, size=(30, 128)) * 255).astype(np.uint8)])
    ids, d = ann.knn_exact(base, q, 10, engine="tensor")
    _exact(ids, d, *oracle.knn(base, q, 10))
    assert ids[0].tolist() == [500] + list(range(9))
    assert d[0, 0] == 128 * 255 ** 2 - 509 and np.all(d[0, 1:] == 128 * 255 ** 2)


def test_tensor_knn_k_beyond_n_pads():
    base = np.array([[0] * 8, [1] * 8, [3] * 8], np.uint8)
    q = np.array([[1] * 8], np.uint8)
    ids, d = ann.knn_exact(base, q, 5, engine="tensor")
    oi, od = oracle.knn(base, q, 5)
    assert ids.tolist() == oi.tolist() == [[1, 0, 2, -1, -1]]
    assert np.array_equal(d.astype(np.float64), od) and np.isinf(d[0, 3:]).all()


def test_tensor_knn_two_base_chunks():
    """4.5M base rows: two chunks of the base (2^22 rows, then a ragged rest);
    a sample of queries is recomputed by the oracle, and the engines agree on
    every query."""
    mx = datagen.sift_like()
    base, q = mx.base(4_500_000), mx.queries(130)
    ids, d, ms = ann.knn_exact(base, q, 10, engine="tensor", return_ms=True)
    s = np.r_[0:4, 126:130]
    _exact(ids[s], d[s], *oracle.knn(base, q[s], 10))
    ci, cd = ann.knn_exact(base, q, 10, engine="cuda")
    assert np.array_equal(ids, ci) and np.array_equal(d, cd)
    assert ms > 0


def test_tensor_engine_rejects_float_data():
    x = np.zeros((10, 8), np.float32)
    with pytest.raises(ann.AnnError) as e:
        ann.knn_exact(x, x[:2], 3, engine="tensor")
    assert e.value.status == ann._abi.ANN_EINVAL


@pytest.mark.parametrize("n", [131_072, 131_077])
def test_tensor_knn_seed_chunk_boundary(n):
    """The base is processed as a first chunk of 2^17 rows, then chunks of
    2^22: exactly the first chunk, and the first chunk plus a 5-row second
    chunk (one ragged tile), bit-exact against the oracle."""
    mx = datagen.sift_like()
    base, q = mx.base(n), mx.queries(70)
    ids, d = ann.knn_exact(base, q, 12, engine="tensor")
    _exact(ids, d, *oracle.knn(base, q, 12))
