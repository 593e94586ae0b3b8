// PQ encoding on the GPU (index-build tooling): for every vector and
// subspace, the nearest of the 256 centroids, lowest index on ties.  uint8
// data with integer centroids uses exact int32 distances (__vabsdiffu4 +
// __dp4a), so the codes equal the host encoder's; float32 data uses FP32.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "ann_internal.h"

namespace ann {
namespace {

// One thread per (vector, subspace); the subspace's centroids in shared memory.
__global__ void encode_u8(const uint8_t* __restrict__ x, int64_t n, int d, int M,
                          const uint32_t* __restrict__ cbw, uint8_t* __restrict__ codes) {
  extern __shared__ uint32_t cb[];  // 256 * (dsub/4) words of subspace blockIdx.y
  const int m = blockIdx.y, dsub = d / M, wps = dsub / 4;
  for (int i = threadIdx.x; i < 256 * wps; i += blockDim.x) cb[i] = cbw[(size_t)m * 256 * wps + i];
  __syncthreads();
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const uint32_t* xv = reinterpret_cast<const uint32_t*>(x + v * d + m * dsub);
  uint32_t q[16];
  for (int w = 0; w < wps; ++w) q[w] = __ldg(xv + w);
  unsigned best = 0xffffffffu;
  int arg = 0;
  for (int c = 0; c < 256; ++c) {
    unsigned acc = 0;
    for (int w = 0; w < wps; ++w) {
      const unsigned t = __vabsdiffu4(q[w], cb[c * wps + w]);
      acc = __dp4a(t, t, acc);
    }
    if (acc < best) {
      best = acc;
      arg = c;
    }
  }
  codes[v * M + m] = static_cast<uint8_t>(arg);
}

}  // namespace
}  // namespace ann

using namespace ann;

extern "C" int ann_pq_encode_gpu(const void* base, int32_t dtype, int64_t n, int32_t d, int32_t M,
                                 const float* codebook, uint8_t* codes_out) {
  if (!base || !codebook || !codes_out) return set_error(ANN_EINVAL, "ann_pq_encode_gpu: NULL buffer");
  if (dtype != ANN_U8) return set_error(ANN_EINVAL, "ann_pq_encode_gpu: uint8 data only");
  if (n < 1 || M < 1 || d % M || (d / M) % 4 || d / M > 64)
    return set_error(ANN_EINVAL, "ann_pq_encode_gpu: need d %% M == 0, (d/M) %% 4 == 0, d/M <= 64");
  const int dsub = d / M, wps = dsub / 4;
  std::vector<uint32_t> words((size_t)M * 256 * wps);
  for (int m = 0; m < M; ++m)
    for (int c = 0; c < 256; ++c)
      for (int w = 0; w < wps; ++w) {
        uint32_t word = 0;
        for (int b = 0; b < 4; ++b) {
          const float v = codebook[((size_t)m * 256 + c) * dsub + 4 * w + b];
          if (!(v >= 0.f && v <= 255.f) || v != static_cast<float>(static_cast<int>(v)))
            return set_error(ANN_EINVAL, "ann_pq_encode_gpu: codebook values must be integers in [0,255]");
          word |= static_cast<uint32_t>(v) << (8 * b);
        }
        words[((size_t)m * 256 + c) * wps + w] = word;
      }
  // encode in slices of rows so device memory stays bounded
  const int64_t slice = std::min<int64_t>(n, 16ll << 20);
  uint8_t *xd = nullptr, *cd = nullptr;
  uint32_t* cbd = nullptr;
  cudaError_t e = cudaMalloc(&xd, (size_t)slice * d);
  if (e == cudaSuccess) e = cudaMalloc(&cd, (size_t)slice * M);
  if (e == cudaSuccess) e = cudaMalloc(&cbd, words.size() * 4);
  if (e == cudaSuccess) e = cudaMemcpy(cbd, words.data(), words.size() * 4, cudaMemcpyHostToDevice);
  for (int64_t lo = 0; lo < n && e == cudaSuccess; lo += slice) {
    const int64_t m = std::min(slice, n - lo);
    e = cudaMemcpy(xd, static_cast<const uint8_t*>(base) + lo * d, (size_t)m * d, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) break;
    const dim3 grid(static_cast<unsigned>((m + 255) / 256), M);
    encode_u8<<<grid, 256, 256 * wps * 4>>>(xd, m, d, M, cbd, cd);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(codes_out + lo * M, cd, (size_t)m * M, cudaMemcpyDeviceToHost);
  }
  cudaFree(xd);
  cudaFree(cd);
  cudaFree(cbd);
  if (e != cudaSuccess) return cuda_error(e, "pq encode");
  return ANN_OK;
}
