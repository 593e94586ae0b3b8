"""ctypes declarations mirroring include/ann.h (same names, same layouts)."""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libann.so")

ANN_OK, ANN_EINVAL, ANN_ENOMEM, ANN_ECUDA, ANN_ETIMEOUT, ANN_EBUSY, ANN_EIO = 0, -1, -2, -3, -4, -5, -6
ANN_U8, ANN_F32 = 0, 1
ANN_TIER_HOST_PINNED, ANN_TIER_HBM = 0, 1
ANN_NAV_AUTO, ANN_NAV_BF16, ANN_NAV_FP8 = 0, 1, 2

ANN_KNN_AUTO, ANN_KNN_TENSOR_CORES, ANN_KNN_CUDA_CORES = 0, 1, 2
ANN_BUILD_AUTO, ANN_BUILD_TENSOR_CORES, ANN_BUILD_CUDA_CORES = 0, 1, 2
ANN_ORDER_BFS, ANN_ORDER_SPATIAL = 0, 1

STATUS_NAMES = {0: "ANN_OK", -1: "ANN_EINVAL", -2: "ANN_ENOMEM", -3: "ANN_ECUDA",
                -4: "ANN_ETIMEOUT", -5: "ANN_EBUSY", -6: "ANN_EIO"}

# Every symbol include/ann.h declares.
EXPORTS = ["ann_last_error", "ann_version", "ann_load_graph", "ann_save_graph_file",
           "ann_load_graph_file", "ann_free", "ann_index_block_bytes", "ann_index_size",
           "ann_set_warps_per_query",
           "ann_search", "ann_search_dev", "ann_sync", "ann_search_dev_noalloc",
           "ann_search_dev_kernel_grained", "ann_search_cpu_agent",
           "ann_build_pq", "ann_build_graph",
           "ann_knn_exact", "ann_knn_exact_ex", "ann_probe_read_bandwidth", "ann_serve_create", "ann_serve_submit",
           "ann_serve_poll", "ann_serve_poll_any", "ann_serve_stats", "ann_serve_destroy",
           "ann_autotune_degree", "ann_build_graph_gpu", "ann_build_graph_gpu_ex", "ann_encode_bf16",
           "ann_encode_fp8e4m3",
           "ann_pq_encode_gpu", "ann_reorder_graph", "ann_reorder_graph_ex"]


class AnnError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class GraphDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("R", ctypes.c_int32), ("entry", ctypes.c_int32), ("vectors", ctypes.c_void_p),
                ("adj", ctypes.c_void_p), ("M", ctypes.c_int32), ("codebook", ctypes.c_void_p),
                ("codes", ctypes.c_void_p), ("tier", ctypes.c_int32), ("nav", ctypes.c_int32),
                ("nav_scale", ctypes.c_float), ("rerank_mult", ctypes.c_int32),
                ("id_map", ctypes.c_void_p)]


class Trace(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_void_p), ("status", ctypes.c_void_p),
                ("t_begin", ctypes.c_void_p), ("t_end", ctypes.c_void_p)]


class SearchStats(ctypes.Structure):
    _fields_ = [("queries", ctypes.c_int64), ("expansions", ctypes.c_int64),
                ("bytes_per_expansion", ctypes.c_int64), ("n_failed", ctypes.c_int32),
                ("first_failed", ctypes.c_int32), ("kernel_ms", ctypes.c_float)]


class ServeCfg(ctypes.Structure):
    _fields_ = [("max_L", ctypes.c_int32), ("max_k", ctypes.c_int32), ("depth", ctypes.c_int32),
                ("slots", ctypes.c_int32), ("idle_exit_us", ctypes.c_int32)]


class ServeResult(ctypes.Structure):
    _fields_ = [("queries", ctypes.c_int64), ("expansions", ctypes.c_int64),
                ("n_failed", ctypes.c_int32), ("device_ns", ctypes.c_int64)]


class ServeStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("published", ctypes.c_int64),
                ("retired", ctypes.c_int64), ("resident_warps", ctypes.c_int64),
                ("running", ctypes.c_int32)]


class AutotuneCfg(ctypes.Structure):
    _fields_ = [("n_sample", ctypes.c_int32), ("d", ctypes.c_int32), ("M", ctypes.c_int32),
                ("degrees", ctypes.c_void_p), ("n_degrees", ctypes.c_int32),
                ("L", ctypes.c_int32), ("nq", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class AutotunePoint(ctypes.Structure):
    _fields_ = [("degree", ctypes.c_int32), ("t_compute_us", ctypes.c_float),
                ("t_fetch_us", ctypes.c_float), ("step_us_sync", ctypes.c_float),
                ("qps_sync", ctypes.c_float)]


_lib = None


def lib():
    """Load libann.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_2507_10070_b300.build` (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, I64, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        L.ann_last_error.restype = ctypes.c_char_p
        L.ann_last_error.argtypes = []
        L.ann_version.restype = ctypes.c_char_p
        L.ann_version.argtypes = []
        L.ann_load_graph.restype = ctypes.c_int
        L.ann_load_graph.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(GraphDesc)]
        L.ann_save_graph_file.restype = ctypes.c_int
        L.ann_save_graph_file.argtypes = [ctypes.c_char_p, ctypes.POINTER(GraphDesc)]
        L.ann_load_graph_file.restype = ctypes.c_int
        L.ann_load_graph_file.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_char_p, I32]
        L.ann_free.restype = None
        L.ann_free.argtypes = [P]
        L.ann_index_block_bytes.restype = I64
        L.ann_index_block_bytes.argtypes = [P]
        L.ann_index_size.restype = I64
        L.ann_index_size.argtypes = [P]
        L.ann_search.restype = ctypes.c_int
        L.ann_search.argtypes = [P, P, I64, I32, I32, I32, P, P, ctypes.POINTER(Trace),
                                 ctypes.POINTER(SearchStats)]
        L.ann_search_dev.restype = ctypes.c_int
        L.ann_search_dev.argtypes = [P, P, I64, I32, I32, I32, P, P, ctypes.POINTER(Trace), P]
        L.ann_search_cpu_agent.restype = ctypes.c_int
        L.ann_search_cpu_agent.argtypes = [P, P, I64, I32, I32, I32, I32, I64, P, P,
                                           ctypes.POINTER(SearchStats), ctypes.POINTER(ctypes.c_double)]
        L.ann_search_dev_kernel_grained.restype = ctypes.c_int
        L.ann_search_dev_kernel_grained.argtypes = [P, P, I64, I32, I32, I32, P, P,
                                                    ctypes.POINTER(Trace), P]
        L.ann_search_dev_noalloc.restype = ctypes.c_int
        L.ann_search_dev_noalloc.argtypes = [P, P, I64, I32, I32, I32, P, P,
                                             ctypes.POINTER(Trace), P]
        L.ann_sync.restype = ctypes.c_int
        L.ann_sync.argtypes = [P, P, ctypes.POINTER(SearchStats)]
        L.ann_build_pq.restype = ctypes.c_int
        L.ann_build_pq.argtypes = [P, I32, I64, I32, I32, I64, I32, P, U64, P, P, I32]
        L.ann_build_graph.restype = ctypes.c_int
        L.ann_build_graph.argtypes = [P, I32, I64, I32, I32, ctypes.c_float, I32, U64, I32, P,
                                      ctypes.POINTER(ctypes.c_int32)]
        L.ann_build_graph_gpu.restype = ctypes.c_int
        L.ann_build_graph_gpu.argtypes = [P, I32, I64, I32, I32, ctypes.c_float, I32, U64, P,
                                          ctypes.POINTER(ctypes.c_int32)]
        L.ann_build_graph_gpu_ex.restype = ctypes.c_int
        L.ann_build_graph_gpu_ex.argtypes = [P, I32, I64, I32, I32, ctypes.c_float, I32, U64, I32, P,
                                             ctypes.POINTER(ctypes.c_int32)]
        L.ann_encode_bf16.restype = ctypes.c_int
        L.ann_encode_bf16.argtypes = [P, I64, P]
        L.ann_encode_fp8e4m3.restype = ctypes.c_int
        L.ann_encode_fp8e4m3.argtypes = [P, I64, ctypes.c_float, P]
        L.ann_reorder_graph.restype = ctypes.c_int
        L.ann_reorder_graph.argtypes = [P, I32, I64, I32, I32, P, I32, P, I32, P, P, P, P, P]
        L.ann_reorder_graph_ex.restype = ctypes.c_int
        L.ann_reorder_graph_ex.argtypes = [P, I32, I64, I32, I32, P, I32, P, I32, I32, P, P, P, P,
                                           ctypes.POINTER(ctypes.c_int32)]
        L.ann_pq_encode_gpu.restype = ctypes.c_int
        L.ann_pq_encode_gpu.argtypes = [P, I32, I64, I32, I32, P, P]
        L.ann_set_warps_per_query.restype = ctypes.c_int
        L.ann_set_warps_per_query.argtypes = [P, I32]
        L.ann_knn_exact.restype = ctypes.c_int
        L.ann_knn_exact.argtypes = [P, I32, I64, I32, P, I64, I32, P, P]
        L.ann_knn_exact_ex.restype = ctypes.c_int
        L.ann_knn_exact_ex.argtypes = [P, I32, I64, I32, P, I64, I32, I32, P, P,
                                       ctypes.POINTER(ctypes.c_float)]
        L.ann_probe_read_bandwidth.restype = ctypes.c_int
        L.ann_probe_read_bandwidth.argtypes = [I64, I32, I32, I32, ctypes.POINTER(ctypes.c_double)]
        L.ann_serve_create.restype = ctypes.c_int
        L.ann_serve_create.argtypes = [P, ctypes.POINTER(ServeCfg), ctypes.POINTER(ctypes.c_void_p)]
        L.ann_serve_submit.restype = ctypes.c_int
        L.ann_serve_submit.argtypes = [P, P, I64, I32, I32, ctypes.POINTER(ctypes.c_uint64)]
        L.ann_serve_poll.restype = ctypes.c_int
        L.ann_serve_poll.argtypes = [P, U64, P, P, I64, ctypes.POINTER(ServeResult)]
        L.ann_serve_poll_any.restype = ctypes.c_int
        L.ann_serve_poll_any.argtypes = [P, ctypes.POINTER(ctypes.c_uint64), I32, I64,
                                         ctypes.POINTER(ctypes.c_int32)]
        L.ann_autotune_degree.restype = ctypes.c_int
        L.ann_autotune_degree.argtypes = [ctypes.POINTER(AutotuneCfg), ctypes.POINTER(AutotunePoint),
                                          ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32), P,
                                          ctypes.POINTER(ctypes.c_int32), P]
        L.ann_serve_stats.restype = ctypes.c_int
        L.ann_serve_stats.argtypes = [P, ctypes.POINTER(ServeStats)]
        L.ann_serve_destroy.restype = None
        L.ann_serve_destroy.argtypes = [P]
        _lib = L
    return _lib
