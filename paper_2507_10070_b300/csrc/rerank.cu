// Exact FP32 rerank of a search's candidates: for each query, the exact
// squared distance of each candidate (float32 vectors in HBM, FP32
// accumulation in dimension order), then the k nearest by (distance, id).
// Used after navigation on compressed vectors (BF16, FP8-E4M3, float PQ).
#include <cstdint>

#include "ann_internal.h"

namespace ann {
namespace {

constexpr int kRerankMax = 512;

__global__ void rerank_kernel(const float* __restrict__ vectors, int d, const float* __restrict__ queries,
                              int nq, const int32_t* __restrict__ cand, const int32_t* __restrict__ id_map,
                              int kc, int k, int32_t* __restrict__ ids, float* __restrict__ dists) {
  __shared__ unsigned long long keys[4][kRerankMax];  // 16 KB
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int qi = blockIdx.x * 4 + wib;
  if (qi >= nq) return;  // warp-uniform
  unsigned long long* K = keys[wib];
  const float4* q = reinterpret_cast<const float4*>(queries + static_cast<size_t>(qi) * d);
  for (int c = lane; c < kRerankMax; c += 32) {
    unsigned long long key = ~0ull;
    if (c < kc) {
      const int id = cand[static_cast<size_t>(qi) * kc + c];
      if (id >= 0) {
        const float4* x = reinterpret_cast<const float4*>(vectors + static_cast<size_t>(id) * d);
        float acc = 0.f;
        for (int j = 0; j < d / 4; ++j) {
          const float4 u = __ldg(q + j), v = __ldg(x + j);
          float t;
          t = u.x - v.x; acc = fmaf(t, t, acc);
          t = u.y - v.y; acc = fmaf(t, t, acc);
          t = u.z - v.z; acc = fmaf(t, t, acc);
          t = u.w - v.w; acc = fmaf(t, t, acc);
        }
        key = (static_cast<unsigned long long>(__float_as_uint(acc)) << 32) | static_cast<unsigned>(id);
      }
    }
    K[c] = key;
  }
  __syncwarp();
  for (int size = 2; size <= kRerankMax; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = lane; i < kRerankMax; i += 32) {
        const int j = i ^ stride;
        if (j > i) {
          const bool asc = (i & size) == 0;
          const unsigned long long a = K[i], b = K[j];
          if ((a > b) == asc) {
            K[i] = b;
            K[j] = a;
          }
        }
      }
      __syncwarp();
    }
  }
  for (int j = lane; j < k; j += 32) {
    const unsigned long long key = K[j];
    const bool ok = key != ~0ull;
    const int32_t id = static_cast<int32_t>(key & 0xffffffffu);
    ids[static_cast<size_t>(qi) * k + j] = ok ? (id_map ? __ldg(id_map + id) : id) : -1;
    dists[static_cast<size_t>(qi) * k + j] =
        ok ? __uint_as_float(static_cast<unsigned>(key >> 32)) : __int_as_float(0x7f800000);
  }
}

}  // namespace

cudaError_t launch_rerank(const float* vectors, int d, const float* queries, int nq, const int32_t* cand,
                          const int32_t* id_map, int kc, int k, int32_t* ids, float* dists,
                          cudaStream_t st) {
  if (kc > kRerankMax || k > kc) return cudaErrorInvalidValue;
  if (nq == 0) return cudaSuccess;
  rerank_kernel<<<(nq + 3) / 4, 128, 0, st>>>(vectors, d, queries, nq, cand, id_map, kc, k, ids, dists);
  return cudaGetLastError();
}

}  // namespace ann
