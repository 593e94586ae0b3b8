"""Python binding of libann, the B300 relaxed-pipeline graph search library.

Argument marshalling only: every step of index search runs in the CUDA
kernels of libann.so (built in-tree by `paper_2507_10070_b300.build`).  There
is no CPU fallback; importing the binding without the built library, or
searching without a GPU, raises.

Host arrays are numpy; device buffers are torch CUDA tensors (PyTorch is used
only for device memory and streams).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _abi
from ._abi import (ANN_F32, ANN_NAV_AUTO, ANN_NAV_BF16, ANN_NAV_FP8, ANN_TIER_HBM,
                   ANN_TIER_HOST_PINNED, ANN_U8, AnnError, GraphDesc, SearchStats, Trace)

__all__ = ["Index", "Server", "AnnError", "build_pq", "build_graph", "knn_exact", "probe_read_bandwidth",
           "autotune_degree",
           "recall_at_k", "library_path", "ANN_U8", "ANN_F32", "ANN_TIER_HOST_PINNED",
           "ANN_TIER_HBM", "save_index"]


def library_path() -> str:
    return _abi.LIB_PATH


def _lib():
    return _abi.lib()


def _check(rc: int):
    if rc != 0:
        raise AnnError(rc, _lib().ann_last_error().decode())


def _dtype_code(a: np.ndarray) -> int:
    if a.dtype == np.uint8:
        return ANN_U8
    if a.dtype == np.float32:
        return ANN_F32
    raise TypeError(f"vectors must be uint8 or float32, not {a.dtype}")


def _c(a, dtype=None):
    return np.ascontiguousarray(a if dtype is None else np.asarray(a).astype(dtype, copy=False))


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _desc(vectors, adj, entry, codebook, codes, tier, nav=0, nav_scale=0.0, rerank_mult=0,
          id_map=None):
    vectors = _c(vectors)
    adj = _c(adj, np.int32)
    n, d = vectors.shape
    assert adj.shape[0] == n
    M = 0
    if codebook is not None:
        codebook = _c(codebook, np.float32)
        codes = _c(codes, np.uint8)
        M = codebook.shape[0]
    if id_map is not None:
        id_map = _c(id_map, np.int32)
        assert id_map.shape == (n,)
    keep = (vectors, adj, codebook, codes, id_map)
    desc = GraphDesc(n=n, d=d, dtype=_dtype_code(vectors), R=adj.shape[1], entry=int(entry),
                     vectors=_p(vectors), adj=_p(adj), M=M, codebook=_p(codebook),
                     codes=_p(codes), tier=tier, nav=nav, nav_scale=nav_scale,
                     rerank_mult=rerank_mult, id_map=_p(id_map))
    return desc, keep


def save_index(path: str, vectors, adj, entry, codebook=None, codes=None, id_map=None):
    desc, keep = _desc(vectors, adj, entry, codebook, codes, ANN_TIER_HBM, id_map=id_map)
    _check(_lib().ann_save_graph_file(path.encode(), ctypes.byref(desc)))


class Index:
    """A loaded index: node blocks in `tier`, PQ codes / vectors in HBM."""

    def __init__(self, vectors=None, adj=None, entry=0, codebook=None, codes=None,
                 tier: int = ANN_TIER_HOST_PINNED, path: str | None = None, nav: int = 0,
                 nav_scale: float = 0.0, rerank_mult: int = 0, id_map=None):
        """`id_map` (n int32, optional): the caller's id of each stored node;
        results report it instead of the node's position (see reorder_graph)."""
        self._h = ctypes.c_void_p()
        if path is not None:
            _check(_lib().ann_load_graph_file(ctypes.byref(self._h), path.encode(), tier))
            with open(path, "rb") as f:
                hdr = np.frombuffer(f.read(40), dtype=np.uint8)
            fields = hdr[16:40].view(np.int32)
            self.d, self.dtype = int(fields[0]), int(fields[1])
        else:
            desc, _ = _desc(vectors, adj, entry, codebook, codes, tier, nav, nav_scale, rerank_mult,
                            id_map)
            _check(_lib().ann_load_graph(ctypes.byref(self._h), ctypes.byref(desc)))
            self.d, self.dtype = desc.d, desc.dtype
        self.n = int(_lib().ann_index_size(self._h))
        self.block_bytes = int(_lib().ann_index_block_bytes(self._h))

    def close(self):
        if self._h:
            _lib().ann_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_warps_per_query(self, w: int):
        """Warps per query of later searches (1, 2 or 4; see ann_set_warps_per_query)."""
        _check(_lib().ann_set_warps_per_query(self._h, int(w)))

    def _np_dtype(self):
        return np.uint8 if self.dtype == ANN_U8 else np.float32

    def search(self, queries, k: int, L: int, depth: int = 1, trace: bool = False, out=None):
        """Host-buffer search.  Returns (ids int32 (nq,k), dists float32 (nq,k), stats)
        plus a dict of per-query arrays (steps, status, t_begin, t_end) if trace.
        `out` = (ids, dists) preallocated C-contiguous arrays (e.g. views of
        pinned host memory) to write the results into."""
        q = _c(queries, self._np_dtype())
        nq = q.shape[0] if q.ndim == 2 else 0
        if out is not None:
            ids, dists = out
            assert ids.dtype == np.int32 and dists.dtype == np.float32
            assert ids.shape == (nq, k) and dists.shape == (nq, k)
            assert ids.flags.c_contiguous and dists.flags.c_contiguous
        else:
            ids = np.empty((nq, k), np.int32)
            dists = np.empty((nq, k), np.float32)
        stats = SearchStats()
        tr = tr_arrays = None
        if trace:
            tr_arrays = {"steps": np.empty(nq, np.int32), "status": np.empty(nq, np.int32),
                         "t_begin": np.empty(nq, np.int64), "t_end": np.empty(nq, np.int64)}
            tr = Trace(**{key: _p(v) for key, v in tr_arrays.items()})
        rc = _lib().ann_search(self._h, _p(q), nq, k, L, depth, _p(ids), _p(dists),
                               ctypes.byref(tr) if tr else None, ctypes.byref(stats))
        if rc != 0 and not (rc == _abi.ANN_ENOMEM and trace):
            _check(rc)
        out = (ids, dists, stats)
        return out + (tr_arrays,) if trace else out

    def search_dev(self, queries, k: int, L: int, depth: int, ids, dists, stream=None,
                   trace: dict | None = None):
        """Device-buffer search on a torch stream (asynchronous).  queries, ids,
        dists (and trace tensors) are contiguous CUDA tensors."""
        tr = None
        if trace:
            tr = Trace(**{key: ctypes.c_void_p(t.data_ptr()) for key, t in trace.items()})
        st = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
        nq = queries.shape[0]
        _check(_lib().ann_search_dev(self._h, ctypes.c_void_p(queries.data_ptr()), nq, k, L, depth,
                                     ctypes.c_void_p(ids.data_ptr()),
                                     ctypes.c_void_p(dists.data_ptr()),
                                     ctypes.byref(tr) if tr else None, st))

    def search_cpu_agent(self, queries, k: int, L: int, depth: int = 1, agent_threads: int = 4,
                         wait_us: int = 2_000_000, check: bool = True):
        """Host-buffer search with CPU-agent I/O (the ablation of the paper's
        mapped request array; see ann_search_cpu_agent).  Returns (ids, dists,
        stats, seconds); with check=False an ANN_ETIMEOUT does not raise."""
        q = _c(queries, self._np_dtype())
        nq = q.shape[0] if q.ndim == 2 else 0
        ids = np.empty((nq, k), np.int32)
        dists = np.empty((nq, k), np.float32)
        stats = SearchStats()
        secs = ctypes.c_double(0.0)
        rc = _lib().ann_search_cpu_agent(self._h, _p(q), nq, k, L, depth, agent_threads, wait_us,
                                         _p(ids), _p(dists), ctypes.byref(stats), ctypes.byref(secs))
        if check or rc != _abi.ANN_ETIMEOUT:
            _check(rc)
        return ids, dists, stats, secs.value

    def search_dev_kernel_grained(self, queries, k: int, L: int, depth: int, ids, dists,
                                  stream=None, trace: dict | None = None):
        """search_dev with kernel-grained I/O (the ablation: a grid-wide
        barrier after every fetch wait; see ann_search_dev_kernel_grained)."""
        tr = None
        if trace:
            tr = Trace(**{key: ctypes.c_void_p(t.data_ptr()) for key, t in trace.items()})
        st = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
        _check(_lib().ann_search_dev_kernel_grained(self._h, ctypes.c_void_p(queries.data_ptr()),
                                                    queries.shape[0], k, L, depth,
                                                    ctypes.c_void_p(ids.data_ptr()),
                                                    ctypes.c_void_p(dists.data_ptr()),
                                                    ctypes.byref(tr) if tr else None, st))

    def search_dev_noalloc(self, queries, k: int, L: int, depth: int, ids, dists, stream=None,
                           trace: dict | None = None):
        """search_dev with its scratch in the library's fixed static device
        array: no allocation at call time (see ann_search_dev_noalloc)."""
        tr = None
        if trace:
            tr = Trace(**{key: ctypes.c_void_p(t.data_ptr()) for key, t in trace.items()})
        st = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
        _check(_lib().ann_search_dev_noalloc(self._h, ctypes.c_void_p(queries.data_ptr()),
                                             queries.shape[0], k, L, depth,
                                             ctypes.c_void_p(ids.data_ptr()),
                                             ctypes.c_void_p(dists.data_ptr()),
                                             ctypes.byref(tr) if tr else None, st))

    def sync(self, stream=None, check: bool = True) -> SearchStats:
        """Wait for the stream; totals of the device calls since the last sync.
        With check=False a visited-set overflow (ANN_ENOMEM) does not raise:
        stats.n_failed says how many queries it stopped."""
        stats = SearchStats()
        st = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
        rc = _lib().ann_sync(self._h, st, ctypes.byref(stats))
        if rc != 0 and not (rc == _abi.ANN_ENOMEM and not check):
            _check(rc)
        return stats


class Server:
    """Continuous-batching request loop over an Index (see ann_serve_*)."""

    def __init__(self, index: Index, max_L: int = 256, max_k: int = 100, depth: int = 1,
                 slots: int = 16384, idle_exit_us: int = 2000):
        self.index = index
        self.max_k = max_k
        self._h = ctypes.c_void_p()
        cfg = _abi.ServeCfg(max_L=max_L, max_k=max_k, depth=depth, slots=slots,
                            idle_exit_us=idle_exit_us)
        _check(_lib().ann_serve_create(index._h, ctypes.byref(cfg), ctypes.byref(self._h)))
        self._k = {}

    def submit(self, queries, k: int, L: int) -> int:
        """Admit a request; returns its id (raises AnnError ANN_EBUSY when full)."""
        q = _c(queries, self.index._np_dtype())
        rid = ctypes.c_uint64(0)
        _check(_lib().ann_serve_submit(self._h, _p(q), q.shape[0], k, L, ctypes.byref(rid)))
        self._k[rid.value] = (q.shape[0], k)
        return rid.value

    def poll(self, req_id: int, timeout_us: int = 0, check: bool = True):
        """(ids, dists, info) once the request is done, or None if not yet.
        With check=False a visited-set overflow (ANN_ENOMEM) does not raise:
        info.n_failed counts the queries it stopped."""
        nq, k = self._k[req_id]
        ids = np.empty((nq, k), np.int32)
        dists = np.empty((nq, k), np.float32)
        info = _abi.ServeResult()
        rc = _lib().ann_serve_poll(self._h, req_id, _p(ids), _p(dists), timeout_us,
                                   ctypes.byref(info))
        if rc == _abi.ANN_ETIMEOUT:
            return None
        del self._k[req_id]
        if not (rc == _abi.ANN_ENOMEM and not check):
            _check(rc)
        return ids, dists, info

    def ready(self, timeout_us: int = 0, max_n: int = 4096):
        """Ids of admitted requests that are complete (not yet collected)."""
        buf = (ctypes.c_uint64 * max_n)()
        n = ctypes.c_int32(0)
        _check(_lib().ann_serve_poll_any(self._h, buf, max_n, timeout_us, ctypes.byref(n)))
        return [buf[i] for i in range(n.value)]

    def stats(self):
        st = _abi.ServeStats()
        _check(_lib().ann_serve_stats(self._h, ctypes.byref(st)))
        return st

    def close(self):
        if self._h:
            _lib().ann_serve_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_pq(base, M: int, n_train: int = 100_000, iters: int = 25, kpp_uniforms=None,
             seed: int = 0, threads: int = 0, encode_device: str = "cpu"):
    """Train a PQ codebook on the first n_train rows and encode every row
    (host threads, or the GPU for uint8 data with encode_device="gpu").
    Returns (codebook float32 (M,256,d/M), codes uint8 (n,M))."""
    base = _c(base)
    n, d = base.shape
    cb = np.empty((M, 256, d // M), np.float32)
    u = None if kpp_uniforms is None else _c(kpp_uniforms, np.float64)
    if encode_device == "gpu":
        ns = min(n, n_train)
        sample = np.ascontiguousarray(base[:ns])
        scratch = np.empty((ns, M), np.uint8)
        _check(_lib().ann_build_pq(_p(sample), _dtype_code(base), ns, d, M, n_train, iters, _p(u),
                                   ctypes.c_uint64(seed), _p(cb), _p(scratch), threads))
        codes = np.empty((n, M), np.uint8)
        _check(_lib().ann_pq_encode_gpu(_p(base), _dtype_code(base), n, d, M, _p(cb), _p(codes)))
        return cb, codes
    codes = np.empty((n, M), np.uint8)
    _check(_lib().ann_build_pq(_p(base), _dtype_code(base), n, d, M, n_train, iters, _p(u),
                               ctypes.c_uint64(seed), _p(cb), _p(codes), threads))
    return cb, codes


def build_graph(base, R: int, alpha: float = 1.2, L_build: int = 128, seed: int = 0,
                threads: int = 0, device: str = "cpu", engine: str = "auto"):
    """Vamana graph on host threads (device="cpu") or on the GPU
    (device="gpu").  On the GPU, engine chooses where RobustPrune's candidate
    distances run: "auto" (tensor cores for uint8 data with d <= 128, else
    CUDA cores), "tensor" or "cuda"; the graph is the same.  Returns
    (adj int32 (n,R), entry)."""
    base = _c(base)
    n, d = base.shape
    adj = np.empty((n, R), np.int32)
    entry = ctypes.c_int32(0)
    if device == "gpu":
        eng = {"auto": _abi.ANN_BUILD_AUTO, "tensor": _abi.ANN_BUILD_TENSOR_CORES,
               "cuda": _abi.ANN_BUILD_CUDA_CORES}[engine]
        _check(_lib().ann_build_graph_gpu_ex(_p(base), _dtype_code(base), n, d, R,
                                             ctypes.c_float(alpha), L_build, ctypes.c_uint64(seed), eng,
                                             _p(adj), ctypes.byref(entry)))
    else:
        _check(_lib().ann_build_graph(_p(base), _dtype_code(base), n, d, R, ctypes.c_float(alpha),
                                      L_build, ctypes.c_uint64(seed), threads, _p(adj),
                                      ctypes.byref(entry)))
    return adj, int(entry.value)


def autotune_degree(degrees=(32, 48, 64, 96), n_sample: int = 100_000, d: int = 128,
                    M: int = 32, L: int = 32, nq: int = 4096, seed: int = 1):
    """The paper's computation / I/O balanced degree selector on random-link
    sample indices.  Returns a dict with the per-degree table, the chosen
    degree (argmin |T_c - T_f|), the fastest depth at that degree and the
    fastest warps per query (1, 2 or 4) at that degree and depth."""
    deg = np.ascontiguousarray(np.asarray(degrees, np.int32))
    cfg = _abi.AutotuneCfg(n_sample=n_sample, d=d, M=M, degrees=deg.ctypes.data,
                           n_degrees=len(deg), L=L, nq=nq, seed=seed)
    pts = (_abi.AutotunePoint * len(deg))()
    best_d, best_depth, best_w = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    qps = np.zeros(5, np.float32)
    wqps = np.zeros(3, np.float32)
    _check(_lib().ann_autotune_degree(ctypes.byref(cfg), pts, ctypes.byref(best_d),
                                      ctypes.byref(best_depth), _p(qps), ctypes.byref(best_w),
                                      _p(wqps)))
    table = [{"degree": p.degree, "t_compute_us": round(p.t_compute_us, 3),
              "t_fetch_us": round(p.t_fetch_us, 3), "step_us_sync": round(p.step_us_sync, 3),
              "qps_sync": round(p.qps_sync, 1)} for p in pts]
    return {"table": table, "degree": best_d.value, "depth": best_depth.value,
            "qps_by_depth": [round(float(x), 1) for x in qps], "warps_per_query": best_w.value,
            "qps_by_warps_per_query": {str(w): round(float(x), 1) for w, x in zip((1, 2, 4), wqps)},
            "L": L}


def encode_bf16(x):
    """float32 -> BF16 bit patterns (uint16), round to nearest even."""
    x = _c(x, np.float32)
    out = np.empty(x.shape, np.uint16)
    _check(_lib().ann_encode_bf16(_p(x), x.size, _p(out)))
    return out


def encode_fp8e4m3(x, scale: float = 1.0):
    """float32 * scale -> FP8-E4M3 bytes (uint8), round to nearest even, saturating."""
    x = _c(x, np.float32)
    out = np.empty(x.shape, np.uint8)
    _check(_lib().ann_encode_fp8e4m3(_p(x), x.size, ctypes.c_float(scale), _p(out)))
    return out


def reorder_graph(base, adj, entry: int, codes=None, order: str = "bfs"):
    """Storage order of the node blocks (ann_reorder_graph_ex): "bfs", breadth
    first from the entry node, or "spatial", the leaves (128 nodes each) of a
    2-means bisection tree of the vectors.  Returns (base, adj, entry, codes,
    old_of_new) in the new order; load them with id_map=old_of_new so that
    searches report the original ids."""
    base = _c(base)
    adj = _c(adj, np.int32)
    n, d = base.shape
    R = adj.shape[1]
    M = 0 if codes is None else codes.shape[1]
    codes = None if codes is None else _c(codes, np.uint8)
    base_out = np.empty_like(base)
    adj_out = np.empty_like(adj)
    codes_out = None if codes is None else np.empty_like(codes)
    old_of_new = np.empty(n, np.int32)
    entry_out = ctypes.c_int32(0)
    od = {"bfs": _abi.ANN_ORDER_BFS, "spatial": _abi.ANN_ORDER_SPATIAL}[order]
    _check(_lib().ann_reorder_graph_ex(_p(base), _dtype_code(base), n, d, R, _p(adj), int(entry),
                                       _p(codes), M, od, _p(base_out), _p(adj_out), _p(codes_out),
                                       _p(old_of_new), ctypes.byref(entry_out)))
    return base_out, adj_out, int(entry_out.value), codes_out, old_of_new


def knn_exact(base, queries, k: int, engine: str = "auto", return_ms: bool = False):
    """Brute-force exact kNN on the GPU: (ids int32 (nq,k), dists float32 (nq,k)).
    engine: "auto" (tensor cores for uint8 data with d <= 128, else CUDA
    cores), "tensor" or "cuda".  With return_ms, also the device time of the
    search itself in ms."""
    base = _c(base)
    queries = _c(queries, base.dtype)
    nq = queries.shape[0]
    ids = np.empty((nq, k), np.int32)
    dists = np.empty((nq, k), np.float32)
    eng = {"auto": _abi.ANN_KNN_AUTO, "tensor": _abi.ANN_KNN_TENSOR_CORES,
           "cuda": _abi.ANN_KNN_CUDA_CORES}[engine]
    ms = ctypes.c_float(0.0)
    _check(_lib().ann_knn_exact_ex(_p(base), _dtype_code(base), base.shape[0], base.shape[1],
                                   _p(queries), nq, k, eng, _p(ids), _p(dists), ctypes.byref(ms)))
    return (ids, dists, ms.value) if return_ms else (ids, dists)


def probe_read_bandwidth(nbytes: int, block_bytes: int = 512, tier: int = ANN_TIER_HOST_PINNED,
                         iters: int = 64) -> float:
    """GB/s of random block reads from the storage tier (the search's access pattern)."""
    out = ctypes.c_double(0.0)
    _check(_lib().ann_probe_read_bandwidth(nbytes, block_bytes, tier, iters, ctypes.byref(out)))
    return out.value


def recall_at_k(ids, gt_ids, gt_dists, res_dists, k: int = 10) -> float:
    """Tie-aware recall@k, mean over queries: a returned id counts if it is one
    of the k true nearest neighbours, or if its distance is <= the k-th true
    distance (another point tied with a true neighbour).  Capped at k."""
    ids, gt_ids = np.asarray(ids)[:, :k], np.asarray(gt_ids)[:, :k]
    kth = np.asarray(gt_dists)[:, k - 1:k]
    member = (ids[:, :, None] == gt_ids[:, None, :]).any(-1)
    ok = (member | (np.asarray(res_dists)[:, :k] <= kth)) & (ids >= 0)
    return float(np.minimum(ok.sum(axis=1), k).mean() / k)
