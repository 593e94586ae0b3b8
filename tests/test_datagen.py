"""The shared seeded input generator: determinism and the distribution it claims."""
import numpy as np

import datagen


def test_deterministic_and_chunk_independent():
    mx = datagen.sift_like()
    a = mx.base(70_000)            # crosses a generation chunk boundary
    b = mx.base(1000)
    assert np.array_equal(a[:1000], b)
    assert np.array_equal(mx.base(1000), b)
    assert not np.array_equal(mx.queries(1000), b)   # queries use their own stream


def test_box_muller_moments():
    s = datagen.Stream(123, 7)
    z = datagen._box_muller(s.uniform((200_000, 2)))
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.01


def test_uniform_range():
    u = datagen.Stream(1, 0).uniform(100_000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005


def test_mixture_shapes_and_spread():
    mx = datagen.sift_like()
    x = mx.base(20_000).astype(np.float64)
    c = mx.centres()
    # nearest centre of each point; residual std ~ sigma (clipping shrinks it a little)
    d2 = ((x[:2000, None, :] - c[None, :, :]) ** 2).sum(-1)
    r = x[:2000] - c[d2.argmin(1)]
    assert 17.0 < r.std() < 21.0
    f = datagen.inmemory_f32().base(5000)
    assert f.dtype == np.float32 and f.shape == (5000, 128)
    u = datagen.deep_like().base(1000)
    assert np.allclose(np.linalg.norm(u, axis=1), 1.0, atol=1e-5)


def test_build_randomness():
    o = datagen.build_order(5, 1000)
    assert sorted(o.tolist()) == list(range(1000))
    g = datagen.random_out_neighbours(5, 300, 16)
    assert g.shape == (300, 16)
    for i in range(300):
        assert i not in g[i] and len(set(g[i].tolist())) == 16
    assert np.array_equal(g, datagen.random_out_neighbours(5, 300, 16))


def test_parallel_generation_equals_sequential():
    mx = datagen.sift_like()
    n = 4 * datagen._PAR_ROWS + 12345          # several worker tasks and a ragged tail
    par = mx.base(n, workers=4)
    # spot-check rows against independent sequential draws of their runs
    for lo in (0, datagen._PAR_ROWS - 3, 2 * datagen._PAR_ROWS + 7, n - 5):
        chunk = np.empty((5, mx.d), np.uint8)
        mx._draw_rows(datagen.STREAM_BASE, lo, lo + 5, chunk)
        assert np.array_equal(par[lo:lo + 5], chunk)
    assert np.array_equal(par[:70_000], mx.base(70_000, workers=1))


def test_random_links_and_bytes():
    n = 4 * datagen._PAR_ROWS + 77
    g = datagen.random_links(9, n, 4, workers=4)                # parallel path
    assert g.shape == (n, 4) and g.dtype == np.int32
    assert g.min() >= 0 and g.max() < n
    assert np.array_equal(g[:50_000], datagen.random_links(9, n, 4, workers=1)[:50_000])
    tail = np.empty((77, 4), np.int32)
    datagen._link_rows(9, n, 4, n - 77, n, tail)                 # counter jump to the tail
    assert np.array_equal(g[-77:], tail)
    # roughly uniform: each quarter of the id range gets a quarter of the links
    frac = np.bincount(g.ravel() // (n // 4 + 1), minlength=4) / g.size
    assert np.all(np.abs(frac - 0.25) < 0.001)
    small = datagen.random_links(9, 1000, 64)
    assert any(len(set(r.tolist())) < 64 for r in small)          # repeats are kept
    b = datagen.random_bytes(3, 1000, 16)
    assert b.shape == (1000, 16) and b.dtype == np.uint8
    part = np.empty((10, 16), np.uint8)
    datagen._byte_rows(3, 16, 500, 510, part)
    assert np.array_equal(b[500:510], part)
    assert abs(b.mean() - 127.5) < 2.0
