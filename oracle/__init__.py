"""CPU oracle for the relaxed-pipeline graph search -- TEST INFRASTRUCTURE.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  The product library never loads it and
it never loads the product library: the two share no code.

`oracle.c` holds the plain C definitions (see its header for what each
function follows in the paper); this module compiles it with gcc and exposes
numpy-facing wrappers.  Parity status per function:

* knn, l2, medoid, search (every depth): pinned by closed forms, brute force
  on tiny inputs and hand-traced graphs at depths 0, 1, 2 and 4
  (tests/test_oracle*.py, tests/golden/).
* pq_train: K=1 closed forms (the k-means++ pick, the mean, the mean
  rounded half to even for uint8 data), hand-worked k-means++ seeding at
  K=2 and K=3 (D^2 weighting, strict comparison), hand-worked empty-cluster
  cases (farthest point, lowest id on ties, each point used once), and
  Lloyd's iterations against scipy's kmeans2 from the same start (float
  data).  tests/test_oracle_pins.py also plants each of these mistakes in a
  copy of oracle.c and checks that a pin fails.
* vamana: closed forms on a line with complete candidate sets (alpha = 1
  gives the path graph; alpha > 1 gives the ladder of kept distances that
  alpha on squared distances implies) and graph invariants (degree bound, no
  self loops, connectivity, recall).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

U8, F32 = 0, 1


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain -O2, no FP contraction)."""
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lpthread", "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.orc_l2_u8.restype = I64
        lib.orc_l2_u8.argtypes = [P, P, I]
        lib.orc_l2_f32.restype = D
        lib.orc_l2_f32.argtypes = [P, P, I]
        lib.orc_knn.restype = None
        lib.orc_knn.argtypes = [I, P, I64, I, P, I64, I, P, P, I]
        lib.orc_medoid.restype = ctypes.c_int32
        lib.orc_medoid.argtypes = [I, P, I64, I]
        lib.orc_pq_train.restype = None
        lib.orc_pq_train.argtypes = [I, P, I64, I, I, I, I, P, I, P, P]
        lib.orc_pq_encode.restype = None
        lib.orc_pq_encode.argtypes = [I, P, I64, I, I, I, P, P]
        lib.orc_search.restype = I
        lib.orc_search.argtypes = [I, P, I64, I, I, P, I, P, P, ctypes.c_int32, P, I64,
                                   I, I, I, P, P, P, P, I, P, P, I, I]
        lib.orc_vamana.restype = I
        lib.orc_vamana.argtypes = [I, P, I64, I, I, D, I, ctypes.c_int32, P, P, I, P]
        _lib = lib
    return _lib


def _dtype_code(x: np.ndarray) -> int:
    if x.dtype == np.uint8:
        return U8
    if x.dtype == np.float32:
        return F32
    raise TypeError(f"unsupported element type {x.dtype}")


def _c(x: np.ndarray, dtype=None) -> np.ndarray:
    return np.ascontiguousarray(x if dtype is None else x.astype(dtype, copy=False))


def _ptr(x):
    return None if x is None else x.ctypes.data


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def l2(a: np.ndarray, b: np.ndarray) -> float:
    a, b = _c(a), _c(b)
    if a.dtype == np.uint8:
        return int(_load().orc_l2_u8(_ptr(a), _ptr(b), a.size))
    return float(_load().orc_l2_f32(_ptr(a), _ptr(b), a.size))


def knn(base: np.ndarray, queries: np.ndarray, k: int, threads: int | None = None):
    """Brute-force exact kNN by (squared L2, id); returns (ids int32, dists float64)."""
    base, queries = _c(base), _c(queries, base.dtype)
    nq = queries.shape[0]
    ids = np.empty((nq, k), np.int32)
    dists = np.empty((nq, k), np.float64)
    _load().orc_knn(_dtype_code(base), _ptr(base), base.shape[0], base.shape[1],
                    _ptr(queries), nq, k, _ptr(ids), _ptr(dists), threads or default_threads())
    return ids, dists


def medoid(base: np.ndarray) -> int:
    base = _c(base)
    return int(_load().orc_medoid(_dtype_code(base), _ptr(base), base.shape[0], base.shape[1]))


def pq_train(sample: np.ndarray, M: int, kpp_u: np.ndarray, iters: int = 25, K: int = 256,
             round_int: bool | None = None, return_distortion: bool = False):
    """k-means++ + Lloyd per subspace; returns codebook (M, K, d/M) float32."""
    sample = _c(sample)
    ns, d = sample.shape
    assert d % M == 0 and ns >= K
    if round_int is None:
        round_int = sample.dtype == np.uint8
    kpp_u = _c(kpp_u, np.float64).reshape(M, K)
    cb = np.empty((M, K, d // M), np.float32)
    dist = np.empty((M, iters + 1), np.float64)
    _load().orc_pq_train(_dtype_code(sample), _ptr(sample), ns, d, M, K, iters, _ptr(kpp_u),
                         int(round_int), _ptr(cb), _ptr(dist))
    return (cb, dist) if return_distortion else cb


def pq_encode(base: np.ndarray, codebook: np.ndarray) -> np.ndarray:
    base = _c(base)
    codebook = _c(codebook, np.float32)
    M, K, _ = codebook.shape
    codes = np.empty((base.shape[0], M), np.uint8)
    _load().orc_pq_encode(_dtype_code(base), _ptr(base), base.shape[0], base.shape[1], M, K,
                          _ptr(codebook), _ptr(codes))
    return codes


def search(base: np.ndarray, adj: np.ndarray, entry: int, queries: np.ndarray, k: int,
           L: int, depth: int, codebook: np.ndarray | None = None,
           codes: np.ndarray | None = None, threads: int | None = None,
           trace_cap: int = 0, return_visited: bool = False,
           nav_vectors: np.ndarray | None = None, rerank: int = 0):
    """Best-first search with relaxed fetch depth `depth` (0 = synchronous).

    Navigation uses PQ codes when `codebook`/`codes` are given, exact
    distances otherwise.  Returns (ids int32 (nq,k), dists float64 (nq,k),
    steps int32 (nq,)) and, with trace_cap > 0, the expansion sequences
    (nq, trace_cap) padded with -1; with return_visited, also the number of
    distinct nodes each query inserted into its visited set (last element).
    `nav_vectors` (n x d, float64): navigate on these instead of the base or
    the codes.  `rerank` > 0: the result is the exact rerank of the `rerank`
    expanded nodes nearest by navigation distance (instead of all expanded
    nodes ranked exactly).
    """
    base = _c(base)
    adj = _c(adj, np.int32)
    queries = _c(queries, base.dtype)
    n, d = base.shape
    nq = queries.shape[0]
    M = 0
    if codebook is not None:
        codebook = _c(codebook, np.float32)
        codes = _c(codes, np.uint8)
        M = codebook.shape[0]
        assert codebook.shape[1] == 256 and codes.shape == (n, M)
    ids = np.empty((nq, k), np.int32)
    dists = np.empty((nq, k), np.float64)
    steps = np.empty(nq, np.int32)
    trace = np.full((nq, trace_cap), -1, np.int32) if trace_cap else None
    nvis = np.empty(nq, np.int32) if return_visited else None
    navv = None if nav_vectors is None else _c(nav_vectors, np.float64)
    if navv is not None:
        assert navv.shape == (n, d)
    rc = _load().orc_search(_dtype_code(base), _ptr(base), n, d, adj.shape[1], _ptr(adj), M,
                            _ptr(codebook), _ptr(codes), entry, _ptr(queries), nq, k, L, depth,
                            _ptr(ids), _ptr(dists), _ptr(steps), _ptr(trace), trace_cap,
                            _ptr(nvis), _ptr(navv), int(rerank), threads or default_threads())
    if rc != 0:
        raise ValueError("oracle search: invalid arguments")
    out = (ids, dists, steps) + ((trace,) if trace_cap else ())
    return out + (nvis,) if return_visited else out


def vamana(base: np.ndarray, R: int, alpha: float, L_build: int, entry: int,
           order: np.ndarray, init_adj: np.ndarray) -> np.ndarray:
    """Sequential two-pass Vamana; returns (n, R) int32 adjacency, -1 padded."""
    base = _c(base)
    order = _c(order, np.int32)
    init_adj = _c(init_adj, np.int32)
    n, d = base.shape
    adj = np.empty((n, R), np.int32)
    rc = _load().orc_vamana(_dtype_code(base), _ptr(base), n, d, R, float(alpha), L_build, entry,
                            _ptr(order), _ptr(init_adj), init_adj.shape[1], _ptr(adj))
    if rc != 0:
        raise ValueError("oracle vamana: invalid arguments")
    return adj


def decode_bf16(bits: np.ndarray) -> np.ndarray:
    """BF16 bit patterns -> float64 (the value is the float32 with these upper 16 bits)."""
    b = np.asarray(bits, np.uint16).astype(np.uint32) << np.uint32(16)
    return b.view(np.float32).astype(np.float64)


def decode_fp8e4m3(b: np.ndarray, scale: float = 1.0) -> np.ndarray:
    """FP8-E4M3 bytes -> float64 values / scale, from the format's definition:
    sign bit, 4-bit exponent with bias 7, 3-bit mantissa; exponent field 0 is
    subnormal (m * 2^-9); S.1111.111 is NaN; no infinities."""
    b = np.asarray(b, np.uint8).astype(np.int64)
    s = np.where(b & 0x80, -1.0, 1.0)
    e = (b >> 3) & 0xF
    m = b & 0x7
    val = np.where(e == 0, m * 2.0 ** -9, (1.0 + m / 8.0) * np.exp2(e - 7.0))
    val = np.where((e == 15) & (m == 7), np.nan, val)
    return s * val / scale


def recall_at_k(ids, gt_ids, gt_dists, res_dists, k: int = 10) -> float:
    """Tie-aware recall@k, mean over queries: a returned id counts if it is one
    of the k true nearest neighbours, or if its distance is <= the k-th true
    distance (another point tied with a true neighbour).  Capped at k."""
    ids, gt_ids = np.asarray(ids)[:, :k], np.asarray(gt_ids)[:, :k]
    kth = np.asarray(gt_dists)[:, k - 1:k]
    member = (ids[:, :, None] == gt_ids[:, None, :]).any(-1)
    ok = (member | (np.asarray(res_dists)[:, :k] <= kth)) & (ids >= 0)
    return float(np.minimum(ok.sum(axis=1), k).mean() / k)
