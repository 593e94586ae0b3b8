// Storage-tier read probe: the achievable bandwidth of random node-block
// reads, issued the way the search kernel issues them (per-lane 16-byte
// cp.async into shared memory, one commit group per block), with 4 blocks in
// flight per warp and a full-occupancy grid.  Its GB/s is the denominator of
// the search kernel's roofline fraction.
#include <cstdint>

#include "ann_internal.h"

namespace ann {
namespace {

constexpr int kInFlight = 4;
constexpr int kWarpsPerBlock = 8;

__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  // splitmix64 finaliser (Steele, Lea, Flood 2014)
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

__global__ void read_probe(const uint8_t* __restrict__ region, int64_t nblocks, int block_bytes,
                           int iters, unsigned long long* sink) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  unsigned char* ws = sm + wib * kInFlight * block_bytes;
  const unsigned long long gw = static_cast<unsigned long long>(blockIdx.x) * kWarpsPerBlock + wib;
  unsigned acc = 0;
  for (int it = 0; it < iters; ++it) {
    for (int j = 0; j < kInFlight; ++j) {
      const unsigned long long r = mix64(gw * 0x100000001b3ull + it * kInFlight + j);
      const uint8_t* src = region + static_cast<size_t>(r % nblocks) * block_bytes;
      unsigned char* dst = ws + j * block_bytes;
      for (int off = lane * 16; off < block_bytes; off += 512) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(
                         static_cast<unsigned>(__cvta_generic_to_shared(dst + off))),
                     "l"(src + off)
                     : "memory");
      }
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncwarp();
    acc += reinterpret_cast<const unsigned*>(ws)[lane];
    __syncwarp();
  }
  if (acc == 0x12345678u) atomicAdd(sink, 1ull);  // keeps the reads observable
}

}  // namespace

cudaError_t launch_read_probe(const uint8_t* region, int64_t nblocks, int block_bytes, int iters,
                              unsigned long long* sink, cudaStream_t stream, float* ms_out,
                              int64_t* bytes_out) {
  const int smem = kWarpsPerBlock * kInFlight * block_bytes;
  cudaError_t e = cudaFuncSetAttribute(read_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, read_probe, 32 * kWarpsPerBlock, smem);
  if (e != cudaSuccess) return e;
  const int blocks = sms * (per_sm > 0 ? per_sm : 1);
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  // warm-up launch (TLB / link wake-up), then the timed one
  read_probe<<<blocks, 32 * kWarpsPerBlock, smem, stream>>>(region, nblocks, block_bytes,
                                                            iters > 4 ? 4 : iters, sink);
  cudaEventRecord(a, stream);
  read_probe<<<blocks, 32 * kWarpsPerBlock, smem, stream>>>(region, nblocks, block_bytes, iters, sink);
  cudaEventRecord(b, stream);
  e = cudaGetLastError();
  cudaError_t e2 = cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms_out = ms;
  *bytes_out = static_cast<int64_t>(blocks) * kWarpsPerBlock * iters * kInFlight * block_bytes;
  return e != cudaSuccess ? e : e2;
}

}  // namespace ann
