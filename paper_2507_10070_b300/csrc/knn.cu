// Brute-force exact k nearest neighbours on the GPU (ground truth for recall).
//
// Two kernels per chunk of queries:
//  1. dist_tile: a 64-query x 64-row tile per block, 256 threads each owning
//     a 4x4 sub-tile; query and base rows staged in shared memory.  uint8
//     distances are exact integers (__vabsdiffu4 + __dp4a); float32 uses FP32.
//  2. topk_rows: one block per query scans its row of the distance matrix;
//     each thread keeps an ascending top-k of (distance, id) keys, then k
//     rounds of a block-wide minimum pop the global top-k.
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

__global__ void __launch_bounds__(256) topk_rows(const unsigned* __restrict__ dist, int64_t n,
                                                 int k, int32_t* __restrict__ ids,
                                                 float* __restrict__ dists, bool u8) {
  __shared__ unsigned long long red[256];
  unsigned long long top[kMaxK];
  const int tid = threadIdx.x;
  const unsigned* row = dist + static_cast<int64_t>(blockIdx.x) * n;
  int cnt = 0;
  for (int64_t i = tid; i < n; i += blockDim.x) {
    const unsigned long long key = (static_cast<unsigned long long>(row[i]) << 32) |
                                   static_cast<unsigned>(i);
    if (cnt == k && key >= top[k - 1]) continue;
    int p = cnt < k ? cnt : k - 1;
    while (p > 0 && top[p - 1] > key) {
      top[p] = top[p - 1];
      --p;
    }
    top[p] = key;
    if (cnt < k) ++cnt;
  }
  int head = 0;
  for (int r = 0; r < k; ++r) {
    red[tid] = head < cnt ? top[head] : ~0ull;
    __syncthreads();
    for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
      if (tid < s && red[tid + s] < red[tid]) red[tid] = red[tid + s];
      __syncthreads();
    }
    const unsigned long long best = red[0];
    __syncthreads();
    if (head < cnt && top[head] == best) ++head;
    if (tid == 0) {
      const bool ok = best != ~0ull;
      const unsigned db = static_cast<unsigned>(best >> 32);
      ids[static_cast<int64_t>(blockIdx.x) * k + r] = ok ? static_cast<int32_t>(best & 0xffffffffu) : -1;
      dists[static_cast<int64_t>(blockIdx.x) * k + r] =
          ok ? (u8 ? static_cast<float>(db) : __uint_as_float(db)) : __int_as_float(0x7f800000);
    }
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
  unsigned* dmat = nullptr;
  cudaError_t e = cudaMalloc(&dmat, static_cast<size_t>(chunk) * n * sizeof(unsigned));
  if (e != cudaSuccess) return e;
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
    topk_rows<<<static_cast<unsigned>(m), 256, 0, stream>>>(dmat, n, k, ids + q0 * k,
                                                            dists + q0 * k, u8);
    e = cudaGetLastError();
  }
  cudaError_t e2 = cudaStreamSynchronize(stream);
  cudaFree(dmat);
  return e != cudaSuccess ? e : e2;
}

}  // namespace ann
