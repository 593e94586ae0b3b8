"""Seeded synthetic workloads shaped like the paper's evaluation datasets.

The paper evaluates on SIFT1B (uint8, d=128), DEEP1B (float32, d=96) and
SPACEV1B (Section "Experimental Setting").  Those datasets are not available
here, so every input is drawn from a seeded Gaussian mixture with the same
element type and dimensionality.  This module is the ONE place both the CPU
oracle and the CUDA path get their inputs from; it holds random numbers only,
none of the search method's arithmetic.

Generator: numpy's counter-based Philox bit generator (Philox-4x64, 10 rounds,
Salmon et al., SC'11), keyed by (seed, stream).  Uniforms are the top 53 bits
of each 64-bit output scaled by 2^-53; normals come from the Box-Muller
transform in float64.  Each vector consumes exactly d+1 uniforms (one for its
mixture component, d for its d normals), so the output does not depend on the
chunk size used to generate it.

Streams: 0 centres, 1 base vectors, 2 queries, 3 PQ training randomness,
4 graph-build randomness, 5 random-link graphs, 6 random bytes.  Workload seeds are 2507_10070 + workload number.

Because the generator is counter-based, any run of vectors can be drawn on
its own (the stream jumps to draw i*(d+1)); large bases are generated in
parallel worker processes into shared memory, with the same result as a
sequential pass.
"""
from __future__ import annotations

import dataclasses
import math
import os

import numpy as np

SEED_BASE = 2507_10070
STREAM_CENTRES = 0
STREAM_BASE = 1
STREAM_QUERIES = 2
STREAM_PQ = 3
STREAM_BUILD = 4
STREAM_LINKS = 5
STREAM_BYTES = 6

_CHUNK = 1 << 16


class Stream:
    """Sequential uniform/normal source on one (seed, stream) Philox key."""

    def __init__(self, seed: int, stream: int, position: int = 0):
        key = np.array([seed & 0xFFFFFFFFFFFFFFFF, stream], dtype=np.uint64)
        self._bg = np.random.Philox(key=key)
        if position:
            # Philox produces 4 outputs per counter step
            self._bg.advance(position // 4)
            if position % 4:
                self._bg.random_raw(position % 4)

    def raw(self, count: int) -> np.ndarray:
        return self._bg.random_raw(int(count)).astype(np.uint64)

    def uniform(self, shape) -> np.ndarray:
        count = int(np.prod(shape)) if np.ndim(shape) else int(shape)
        u = (self.raw(count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return u.reshape(shape)


def _box_muller(u: np.ndarray) -> np.ndarray:
    """Map pairs of uniforms (last axis, even length) to standard normals."""
    u1 = u[..., 0::2]
    u2 = u[..., 1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))
    t = 2.0 * math.pi * u2
    z = np.empty_like(u)
    z[..., 0::2] = r * np.cos(t)
    z[..., 1::2] = r * np.sin(t)
    return z


@dataclasses.dataclass(frozen=True)
class Mixture:
    """Isotropic Gaussian mixture: centres uniform in [lo, hi]^d, std sigma."""

    seed: int
    d: int
    n_centres: int
    lo: float
    hi: float
    sigma: float
    kind: str  # "u8" (clip to [0,255], round half to even), "f32", "f32_unit"

    def centres(self) -> np.ndarray:
        s = Stream(self.seed, STREAM_CENTRES)
        return self.lo + (self.hi - self.lo) * s.uniform((self.n_centres, self.d))

    def _draw_rows(self, stream: int, lo: int, hi: int, out: np.ndarray) -> None:
        """Rows [lo, hi) of the stream into out[0:hi-lo]."""
        assert self.d % 2 == 0, "Box-Muller pairs need an even dimension"
        c = self.centres()
        s = Stream(self.seed, stream, position=lo * (self.d + 1))
        for a in range(lo, hi, _CHUNK):
            m = min(_CHUNK, hi - a)
            u = s.uniform((m, self.d + 1))
            comp = np.minimum((u[:, 0] * self.n_centres).astype(np.int64),
                              self.n_centres - 1)
            x = c[comp] + self.sigma * _box_muller(u[:, 1:])
            dst = out[a - lo:a - lo + m]
            if self.kind == "u8":
                dst[:] = np.clip(np.rint(x), 0, 255).astype(np.uint8)
            elif self.kind == "f32_unit":
                x /= np.linalg.norm(x, axis=1, keepdims=True)
                dst[:] = x.astype(np.float32)
            else:
                dst[:] = x.astype(np.float32)

    def _draw(self, stream: int, n: int, workers: int | None = None) -> np.ndarray:
        assert self.d % 2 == 0, "Box-Muller pairs need an even dimension"
        dtype = np.uint8 if self.kind == "u8" else np.float32
        return _rows(_mixture_rows, (self, stream), n, self.d, dtype, workers)

    def base(self, n: int, workers: int | None = None) -> np.ndarray:
        return self._draw(STREAM_BASE, n, workers)

    def queries(self, nq: int) -> np.ndarray:
        return self._draw(STREAM_QUERIES, nq, 1)


_PAR_ROWS = 1 << 20  # rows per worker task


def _mixture_rows(mixture, stream, lo, hi, out):
    mixture._draw_rows(stream, lo, hi, out)


def _link_rows(seed, n, R, lo, hi, out):
    """Rows [lo, hi) of a random-link graph: R ids uniform in [0, n) per row
    (draw i*R + j is row i's j-th id); repeats and self links are kept."""
    s = Stream(seed, STREAM_LINKS, position=lo * R)
    for a in range(lo, hi, _CHUNK):
        m = min(_CHUNK, hi - a)
        out[a - lo:a - lo + m] = (s.uniform((m, R)) * n).astype(np.int32)


def _byte_rows(seed, width, lo, hi, out):
    """Rows [lo, hi) of uniform random bytes, width/8 raw 64-bit draws per row
    (little-endian byte order)."""
    s = Stream(seed, STREAM_BYTES, position=lo * (width // 8))
    for a in range(lo, hi, _CHUNK):
        m = min(_CHUNK, hi - a)
        out[a - lo:a - lo + m] = s.raw(m * width // 8).view(np.uint8).reshape(m, width)


def _fill_task(args):
    from multiprocessing import shared_memory
    fn, fn_args, lo, hi, name, n, width, dtype = args
    shm = shared_memory.SharedMemory(name=name)
    try:
        arr = np.ndarray((n, width), dtype=dtype, buffer=shm.buf)
        fn(*fn_args, lo, hi, arr[lo:hi])
    finally:
        shm.close()
    return hi - lo


def _shm_free() -> int:
    """Free bytes of the shared-memory file system (0 if unknown): a slice
    that does not fit is drawn sequentially instead."""
    try:
        st = os.statvfs("/dev/shm")
        return st.f_bavail * st.f_frsize
    except OSError:
        return 0


def _rows(fn, fn_args, n, width, dtype, workers=None):
    """An (n, width) array whose rows [lo, hi) are fn(*fn_args, lo, hi, out).
    From 4M rows up, worker processes (spawned, so safe after CUDA is up) fill
    1M-row slices of shared memory; the result equals the sequential fill
    because every generator here jumps its counter to the slice's first row."""
    workers = workers if workers is not None else (os.cpu_count() or 1)
    nbytes = n * width * np.dtype(dtype).itemsize
    if n < 4 * _PAR_ROWS or workers <= 1 or _shm_free() < nbytes + (1 << 30):
        out = np.empty((n, width), dtype=dtype)
        fn(*fn_args, 0, n, out)
        return out
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(create=True, size=max(nbytes, 1))
    try:
        tasks = [(fn, fn_args, lo, min(n, lo + _PAR_ROWS), shm.name, n, width, dtype)
                 for lo in range(0, n, _PAR_ROWS)]
        # an executor (not a Pool) so that a worker that dies -- e.g. a script
        # without a __main__ guard re-running itself under spawn -- fails the
        # call at once instead of being respawned forever
        with ProcessPoolExecutor(min(workers, len(tasks)), mp_context=mp.get_context("spawn")) as ex:
            assert sum(ex.map(_fill_task, tasks)) == n
        out = np.ndarray((n, width), dtype=dtype, buffer=shm.buf).copy()
    finally:
        shm.close()
        shm.unlink()
    return out


def random_links(seed: int, n: int, R: int, workers: int | None = None) -> np.ndarray:
    """n x R int32 random-link graph (uniform ids with repeats and self links),
    as used for sample indices whose I/O pattern, not quality, matters."""
    return _rows(_link_rows, (seed, n, R), n, R, np.int32, workers)


def random_bytes(seed: int, n: int, width: int, workers: int | None = None) -> np.ndarray:
    """n x width uint8 of uniform random bytes (width a multiple of 8)."""
    assert width % 8 == 0
    return _rows(_byte_rows, (seed, width), n, width, np.uint8, workers)


def inmemory_f32(seed_offset: int = 1, d: int = 128, n_centres: int = 32) -> Mixture:
    """In-memory float workload: centres in [-1,1]^d, sigma 0.1."""
    return Mixture(SEED_BASE + seed_offset, d, n_centres, -1.0, 1.0, 0.1, "f32")


def sift_like(seed_offset: int = 2, d: int = 128, n_centres: int = 256) -> Mixture:
    """SIFT-like uint8 workload: centres in [0,255]^d, sigma 20, clipped, rounded."""
    return Mixture(SEED_BASE + seed_offset, d, n_centres, 0.0, 255.0, 20.0, "u8")


def sift_like_large(seed_offset: int = 5, d: int = 128, n_centres: int = 4096) -> Mixture:
    """The SIFT-like generator with 4,096 centres, for the 10^8-vector workload."""
    return Mixture(SEED_BASE + seed_offset, d, n_centres, 0.0, 255.0, 20.0, "u8")


def deep_like(seed_offset: int = 3, d: int = 96, n_centres: int = 1024) -> Mixture:
    """DEEP-like float workload: sigma 0.05 around centres in [-1,1]^d, unit-normalised."""
    return Mixture(SEED_BASE + seed_offset, d, n_centres, -1.0, 1.0, 0.05, "f32_unit")


# ---------------------------------------------------------------------------
# Randomness consumed by index construction (passed to whichever builder uses
# it as plain input arrays).
# ---------------------------------------------------------------------------

def kmeanspp_uniforms(seed: int, M: int, K: int = 256) -> np.ndarray:
    """M x K uniforms in [0,1): draw c of subspace m uses [m, c]."""
    return Stream(seed, STREAM_PQ).uniform((M, K))


def build_order(seed: int, n: int) -> np.ndarray:
    """A uniformly random permutation of range(n) (sort of n uniforms; ties by index)."""
    u = Stream(seed, STREAM_BUILD).uniform(n)
    return np.argsort(u, kind="stable").astype(np.int32)


def random_out_neighbours(seed: int, n: int, R: int) -> np.ndarray:
    """n x min(R, n-1) int32: per node, distinct uniformly drawn ids != node.

    Draws are taken in order from stream 4 after the build order's n draws;
    duplicates and self-loops are skipped, so the consumption per node varies
    but the result is a fixed function of (seed, n, R).
    """
    s = Stream(seed, STREAM_BUILD)
    s.raw(n)  # skip the draws the build order uses
    deg = min(R, n - 1)
    out = np.empty((n, deg), dtype=np.int32)
    buf = s.uniform(max(4 * deg, 64) * 64)
    pos = 0
    for i in range(n):
        chosen: list[int] = []
        seen = set()
        while len(chosen) < deg:
            if pos == buf.size:
                buf = s.uniform(buf.size)
                pos = 0
            j = int(buf[pos] * n)
            pos += 1
            if j >= n or j == i or j in seen:
                continue
            seen.add(j)
            chosen.append(j)
        out[i] = chosen
    return out
