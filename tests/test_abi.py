"""The C-ABI library loads and exports every symbol include/ann.h declares;
argument validation that runs before any device work.  No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2507_10070_b300 as ann
from paper_2507_10070_b300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "ann.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"^\S[^\n(]*?\b(ann_\w+)\(", src, re.M)))


def test_header_and_binding_agree():
    assert declared_symbols() == sorted(_abi.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = _abi.lib()
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert lib.ann_version().decode().startswith("libann")


def _desc(**kw):
    base = np.zeros((4, 8), np.uint8)
    adj = np.array([[1, 2], [0, -1], [3, -1], [-1, -1]], np.int32)
    d = dict(n=4, d=8, dtype=0, R=2, entry=0, vectors=base.ctypes.data, adj=adj.ctypes.data,
             M=0, codebook=None, codes=None, tier=ann.ANN_TIER_HBM)
    d.update(kw)
    return _abi.GraphDesc(**d), (base, adj)


@pytest.mark.parametrize("field,value", [("n", 0), ("d", 6), ("d", 1024), ("R", 0), ("R", 129),
                                         ("entry", 4), ("entry", -1), ("dtype", 7), ("tier", 3),
                                         ("M", 3)])
def test_load_graph_rejects_bad_descriptors(field, value):
    lib = _abi.lib()
    desc, keep = _desc(**{field: value})
    h = ctypes.c_void_p()
    assert lib.ann_load_graph(ctypes.byref(h), ctypes.byref(desc)) == _abi.ANN_EINVAL
    assert lib.ann_last_error().decode() != ""


def test_load_graph_rejects_bad_adjacency_and_codebook():
    lib = _abi.lib()
    base = np.zeros((4, 8), np.uint8)
    bad = np.array([[1, 4], [0, -1], [3, -1], [-1, -1]], np.int32)   # id 4 >= n
    desc = _abi.GraphDesc(n=4, d=8, dtype=0, R=2, entry=0, vectors=base.ctypes.data,
                          adj=bad.ctypes.data, M=0, tier=ann.ANN_TIER_HBM)
    h = ctypes.c_void_p()
    assert lib.ann_load_graph(ctypes.byref(h), ctypes.byref(desc)) == _abi.ANN_EINVAL
    # PQ: the codebook must hold integers in [0, 255] (exact integer distances)
    base = np.zeros((4, 32), np.uint8)
    adj = np.array([[1], [0], [0], [0]], np.int32)
    cb = np.full((16, 256, 2), 1.5, np.float32)
    codes = np.zeros((4, 16), np.uint8)
    desc = _abi.GraphDesc(n=4, d=32, dtype=0, R=1, entry=0, vectors=base.ctypes.data,
                          adj=adj.ctypes.data, M=16, codebook=cb.ctypes.data,
                          codes=codes.ctypes.data, tier=ann.ANN_TIER_HOST_PINNED)
    assert lib.ann_load_graph(ctypes.byref(h), ctypes.byref(desc)) == _abi.ANN_EINVAL  # dsub=2
    assert "(d/M) % 4" in lib.ann_last_error().decode()
    # exact navigation needs the vectors in HBM
    desc, keep = _desc(tier=ann.ANN_TIER_HOST_PINNED)
    assert lib.ann_load_graph(ctypes.byref(h), ctypes.byref(desc)) == _abi.ANN_EINVAL


def test_search_rejects_null_index():
    lib = _abi.lib()
    q = np.zeros((1, 8), np.uint8)
    out = np.zeros(1, np.int32)
    assert lib.ann_search(None, q.ctypes.data, 1, 1, 1, 0, out.ctypes.data, out.ctypes.data,
                          None, None) == _abi.ANN_EINVAL


def test_index_file_round_trip_and_corruption(tmp_path):
    lib = _abi.lib()
    base = np.arange(32, dtype=np.uint8).reshape(4, 8)
    adj = np.array([[1, 2], [0, -1], [3, -1], [-1, -1]], np.int32)
    path = str(tmp_path / "g.idx")
    ann.save_index(path, base, adj, 0)
    raw = open(path, "rb").read()
    assert raw[:8] == b"ANNIDX01" and len(raw) == 40 + 32 + 32
    h = ctypes.c_void_p()
    # truncated file -> EIO before any device work
    open(str(tmp_path / "t.idx"), "wb").write(raw[:-5])
    assert lib.ann_load_graph_file(ctypes.byref(h), str(tmp_path / "t.idx").encode(), 1) == _abi.ANN_EIO
    open(str(tmp_path / "c.idx"), "wb").write(b"NOTANIDX" + raw[8:])
    assert lib.ann_load_graph_file(ctypes.byref(h), str(tmp_path / "c.idx").encode(), 1) == _abi.ANN_EIO
    assert lib.ann_load_graph_file(ctypes.byref(h), b"/nonexistent/x.idx", 1) == _abi.ANN_EIO


def test_tooling_rejects_bad_sizes():
    x = np.zeros((100, 8), np.uint8)
    with pytest.raises(ann.AnnError):
        ann.build_pq(x, 3)            # d % M != 0
    with pytest.raises(ann.AnnError):
        ann.build_pq(x, 2)            # fewer than 256 training vectors
    with pytest.raises(ann.AnnError):
        ann.build_graph(x[:1], 4)     # n < 2


def test_autotune_rejects_bad_configuration():
    with pytest.raises(ann.AnnError):
        ann.autotune_degree(degrees=(0, 64), n_sample=20_000)
    with pytest.raises(ann.AnnError):
        ann.autotune_degree(degrees=(64,), n_sample=100)
    with pytest.raises(ann.AnnError):
        ann.autotune_degree(degrees=(64,), d=100)
