// Brute-force exact k nearest neighbours on the GPU (ground truth for recall).
//
// Two kernels per chunk of queries:
//  1. dist_tile: a 64-query x 64-row tile per block, 256 threads each owning
//     a 4x4 sub-tile; query and base rows staged in shared memory.  uint8
//     distances are exact integers (__vabsdiffu4 + __dp4a); float32 uses FP32.
//  2. topk_segments + topk_merge: each row of the distance matrix is split
//     into 2^17-entry segments, one block per segment keeps the segment's
//     top-k (per-thread ascending lists, then k rounds of a block-wide
//     minimum), and one block per query merges the segments' candidates.
// Keys are (distance bits << 32 | id): the order is (distance, id) because
// non-negative float bit patterns sort like the floats they encode.
#include <cstdint>

#include "ann_internal.h"

namespace ann {
namespace {

constexpr int kTile = 64;
constexpr int kMaxK = 128;

template <bool U8>
__global__ void __launch_bounds__(256) dist_tile(const void* __restrict__ base, int64_t n, int d,
                                                 const void* __restrict__ queries, int64_t nq,
                                                 unsigned* __restrict__ out) {
  // shared: 64 query rows and 64 base rows of `wpr` 32-bit words each
  extern __shared__ unsigned sh[];
  const int wpr = U8 ? (d >> 2) : d;  // words per row
  unsigned* qs = sh;
  unsigned* xs = sh + kTile * (wpr + 1);
  const int64_t q0 = static_cast<int64_t>(blockIdx.y) * kTile;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * kTile;
  const unsigned* qw = static_cast<const unsigned*>(queries);
  const unsigned* bw = static_cast<const unsigned*>(base);
  for (int i = threadIdx.x; i < kTile * wpr; i += blockDim.x) {
    const int r = i / wpr, c = i % wpr;
    qs[r * (wpr + 1) + c] = (q0 + r < nq) ? qw[(q0 + r) * wpr + c] : 0u;
    xs[r * (wpr + 1) + c] = (r0 + r < n) ? bw[(r0 + r) * wpr + c] : 0u;
  }
  __syncthreads();
  const int tq = (threadIdx.x >> 4) * 4;  // 16 x 16 threads, 4 x 4 outputs each
  const int tr = (threadIdx.x & 15) * 4;
  unsigned acc_u[4][4] = {};
  float acc_f[4][4] = {};
  for (int c = 0; c < wpr; ++c) {
    unsigned a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      a[i] = qs[(tq + i) * (wpr + 1) + c];
      b[i] = xs[(tr + i) * (wpr + 1) + c];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (U8) {
          const unsigned t = __vabsdiffu4(a[i], b[j]);
          acc_u[i][j] = __dp4a(t, t, acc_u[i][j]);
        } else {
          const float t = __uint_as_float(a[i]) - __uint_as_float(b[j]);
          acc_f[i][j] = fmaf(t, t, acc_f[i][j]);
        }
      }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t q = q0 + tq + i, r = r0 + tr + j;
      if (q < nq && r < n) out[q * n + r] = U8 ? acc_u[i][j] : __float_as_uint(acc_f[i][j]);
    }
}

// Per-block selection of the k smallest keys among `cnt` keys produced by
// get(i): every thread keeps an ascending top-k of its strided share, then k
// rounds of a block-wide minimum pop the block's top-k (written to out[0..k)).
template <class Get>
__device__ void block_topk(Get get, int64_t cnt, int k, unsigned long long* out) {
  __shared__ unsigned long long red[256];
  unsigned long long top[kMaxK];
  const int tid = threadIdx.x;
  int have = 0;
  for (int64_t i = tid; i < cnt; i += blockDim.x) {
    const unsigned long long key = get(i);
    if (key == ~0ull || (have == k && key >= top[k - 1])) continue;
    int p = have < k ? have : k - 1;
    while (p > 0 && top[p - 1] > key) {
      top[p] = top[p - 1];
      --p;
    }
    top[p] = key;
    if (have < k) ++have;
  }
  int head = 0;
  for (int r = 0; r < k; ++r) {
    red[tid] = head < have ? top[head] : ~0ull;
    __syncthreads();
    for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
      if (tid < s && red[tid + s] < red[tid]) red[tid] = red[tid + s];
      __syncthreads();
    }
    const unsigned long long best = red[0];
    __syncthreads();
    if (head < have && top[head] == best) ++head;
    if (tid == 0) out[r] = best;
  }
}

// Stage 1: block (q, s) selects the top-k of segment s of distance row q.
__global__ void __launch_bounds__(256) topk_segments(const unsigned* __restrict__ dist, int64_t n,
                                                     int64_t seg, int k,
                                                     unsigned long long* __restrict__ part) {
  const int64_t q = blockIdx.x, s = blockIdx.y;
  const int64_t lo = s * seg, hi = lo + seg < n ? lo + seg : n;
  const unsigned* row = dist + q * n;
  block_topk([&](int64_t i) {
    const int64_t c = lo + i;
    return (static_cast<unsigned long long>(row[c]) << 32) | static_cast<unsigned>(c);
  }, hi > lo ? hi - lo : 0, k, part + (q * gridDim.y + s) * k);
}

// Stage 2: block q merges its segments' candidates into the final top-k.
__global__ void __launch_bounds__(256) topk_merge(const unsigned long long* __restrict__ part, int nseg,
                                                  int k, int32_t* __restrict__ ids,
                                                  float* __restrict__ dists, bool u8) {
  __shared__ unsigned long long best[kMaxK];
  const int64_t q = blockIdx.x;
  const unsigned long long* p = part + q * nseg * k;
  block_topk([&](int64_t i) { return p[i]; }, (int64_t)nseg * k, k, best);
  __syncthreads();
  for (int r = threadIdx.x; r < k; r += blockDim.x) {
    const unsigned long long b = best[r];
    const bool ok = b != ~0ull;
    const unsigned db = static_cast<unsigned>(b >> 32);
    ids[q * k + r] = ok ? static_cast<int32_t>(b & 0xffffffffu) : -1;
    dists[q * k + r] = ok ? (u8 ? static_cast<float>(db) : __uint_as_float(db)) : __int_as_float(0x7f800000);
  }
}

}  // namespace

cudaError_t knn_exact_device(const void* base, int dtype, int64_t n, int d, const void* queries,
                             int64_t nq, int k, int32_t* ids, float* dists, cudaStream_t stream) {
  if (k > kMaxK) return cudaErrorInvalidValue;
  const bool u8 = dtype == ANN_U8;
  const int wpr = u8 ? (d >> 2) : d;
  const size_t smem = 2ull * kTile * (wpr + 1) * sizeof(unsigned);
  // chunk of queries whose distance rows fit in ~4 GB
  int64_t chunk = (4ll << 30) / (n * 4);
  chunk = chunk / kTile * kTile;
  if (chunk < kTile) chunk = kTile;
  if (chunk > nq) chunk = (nq + kTile - 1) / kTile * kTile;
  // each distance row is scanned by nseg blocks of `seg` entries, then merged
  const int64_t seg = 1 << 17;
  const int nseg = static_cast<int>((n + seg - 1) / seg);
  unsigned* dmat = nullptr;
  unsigned long long* part = nullptr;
  cudaError_t e = cudaMalloc(&dmat, static_cast<size_t>(chunk) * n * sizeof(unsigned));
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&part, static_cast<size_t>(chunk) * nseg * k * sizeof(unsigned long long));
  if (e != cudaSuccess) {
    cudaFree(dmat);
    return e;
  }
  if (u8) e = cudaFuncSetAttribute(dist_tile<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  else e = cudaFuncSetAttribute(dist_tile<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  for (int64_t q0 = 0; q0 < nq && e == cudaSuccess; q0 += chunk) {
    const int64_t m = (nq - q0 < chunk) ? nq - q0 : chunk;
    const dim3 grid(static_cast<unsigned>((n + kTile - 1) / kTile),
                    static_cast<unsigned>((m + kTile - 1) / kTile));
    const size_t elt = u8 ? 1 : 4;
    const void* qp = static_cast<const uint8_t*>(queries) + q0 * d * elt;
    if (u8) dist_tile<true><<<grid, 256, smem, stream>>>(base, n, d, qp, m, dmat);
    else dist_tile<false><<<grid, 256, smem, stream>>>(base, n, d, qp, m, dmat);
    topk_segments<<<dim3(static_cast<unsigned>(m), nseg), 256, 0, stream>>>(dmat, n, seg, k, part);
    topk_merge<<<static_cast<unsigned>(m), 256, 0, stream>>>(part, nseg, k, ids + q0 * k, dists + q0 * k, u8);
    e = cudaGetLastError();
  }
  cudaError_t e2 = cudaStreamSynchronize(stream);
  cudaFree(dmat);
  cudaFree(part);
  return e != cudaSuccess ? e : e2;
}

}  // namespace ann
