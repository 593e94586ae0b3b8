// Brute-force exact k nearest neighbours on the GPU (ground truth for recall).
//
// uint8 data with d <= 128 runs on the tensor cores (knn_tc_kernel below):
// the dot products q.x are a dense contraction, and their BF16 x BF16 ->
// FP32 products and sums are exact integers there, so the distances are
// exact.  float32 data, and uint8 data with d > 128, take the CUDA-core
// path, two kernels per chunk of queries:
//  1. dist_tile: a 64-query x 64-row tile per block, 256 threads each owning
//     a 4x4 sub-tile; query and base rows staged in shared memory.  uint8
//     distances are exact integers (__vabsdiffu4 + __dp4a); float32 uses FP32.
//  2. topk_segments + topk_merge: each row of the distance matrix is split
//     into 2^17-entry segments, one block per segment keeps the segment's
//     top-k (per-thread ascending lists, then k rounds of a block-wide
//     minimum), and one block per query merges the segments' candidates.
// Keys are (distance bits << 32 | id): the order is (distance, id) because
// non-negative float bit patterns sort like the floats they encode.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cfloat>
#include <cstdint>
#include <mutex>

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


// ---------------------------------------------------------------------------
// Tensor-core path (uint8 data, d <= 128).
//
// distance(q, x) = |q|^2 + v(q, x) with v = |x|^2 - 2 q.x; a query's ranking
// depends on v alone.  v is one dot product over K = d + 16 coordinates:
//   A row (query q): q_1 .. q_d, then 2^16, 2^8, 1, zeros;
//   B row (base x):  -2 x_1 .. -2 x_d, then the base-256 digits of |x|^2
//                    (|x|^2 >> 16, its middle byte, its low byte), zeros.
// Every operand is an integer of at most 8 significant bits or a power of
// two, so exact in BF16; every product and partial sum is an integer of
// magnitude below 2 * 128 * 255^2 = 16,646,400 < 2^24, so FP32 accumulation
// in tensor memory (tcgen05.mma, kind::f16) is exact in any order, and so is
// the distance v + |q|^2 <= 8,323,200.  The first d coordinates are 64-wide
// atoms in the 128-byte swizzled layout; the last 16 are one 32-byte-swizzled
// tile, one more MMA per tile.  The top-k selection runs in the same kernel
// on the accumulator, so the distance matrix never goes to HBM.
//
// Per CTA (two query tiles x a contiguous range of base tiles), 20 warps:
//   warp 0 (one lane)  TMA producer: the two query tiles once, then base
//                      tiles into a ring of kTcStages shared-memory stages
//                      (each: the 64-coordinate atoms, 128 B per row, and
//                      the 16-coordinate tail, 32 B per row);
//   warp 1 (one lane)  MMA issuer: for each base tile, d/16 + 1 MMAs per
//                      query tile into one of two accumulator pairs (4 x 128
//                      tensor-memory columns, all 512); tcgen05.commit frees
//                      the stage and publishes the pair;
//   warps 4-19         four epilogue warpgroups, one per accumulator (query
//                      tile qt, buffer b): thread t of warp w reads row
//                      32*(w%4)+t of its query tile with tcgen05.ld and keeps
//                      that query's ascending top-k of (distance, id) keys.
// Two query tiles share each base tile, which halves the base's L2 traffic.
// The epilogue takes v straight from the accumulator: a tree of 3-input mins
// per 32 columns and one compare against the bound k-th distance - |q|^2;
// only a lane whose minimum is within the bound looks at its candidates one
// by one (after the first tiles, the common case is that none is).  The next
// 32 columns load from tensor memory while the current ones are scanned, and
// the accumulator goes back to the MMA as soon as its last columns are in
// registers.  Rows past the end of the base have zero coordinates and the
// largest norm digits (v = 16,777,215 exceeds every real bound), and the
// candidate path checks the row index as well.  The bound starts at the
// running k-th best of the chunks already folded, and the CTAs of a query
// share a distance bound in global memory: each lowers it (atomicMin) to its
// own k-th distance and reads it once per tile (a tile ahead), so a CTA's
// first tiles no longer admit a stream of candidates that another CTA has
// already ruled out.
// Each warpgroup writes its lists as one part; a fold kernel merges the parts
// with the running top-k after each chunk of the base.  The first chunk is
// small, so that the running top-k bounds every later chunk from its start.
// Every wait on an mbarrier is bounded: past ~2 s the CTA sets an abort flag,
// every role leaves its loop, the producer waits (bounded) for the copies it
// issued, tensor memory is freed, and the host sees the error word.

constexpr int kTcM = 128;            // queries per CTA (MMA M)
constexpr int kTcN = 128;            // base rows per tile (MMA N)
constexpr int kTcQT = 2;             // query tiles per CTA
constexpr int kTcStages = 3;         // base-tile ring
constexpr int kAtomBytes = 128 * 128;  // one 64-coordinate BF16 atom of a 128-row tile
constexpr int kTailBytes = 128 * 32;   // the 16-coordinate tail of a 128-row tile
constexpr int kTail = 16;              // tail coordinates: norm digits or their weights
constexpr int kTcThreads = 128 + 4 * 128;
constexpr long long kTcWaitCycles = 4000000000ll;  // ~2 s at 2 GHz

struct TcArgs {
  const float* qn;          // [nq] query norms
  int64_t nq;
  int32_t chunk_n;          // rows of this chunk
  int64_t id0;              // id of the chunk's first row
  int32_t tiles;            // base tiles in the chunk
  int32_t splits;           // CTAs per query tile
  int32_t natoms;           // padded d / 64 (1 or 2)
  int32_t k;
  int32_t nslots;           // parts per query: 1 (running) + 2 * splits
  unsigned long long* keys; // [nq][nslots][k]
  unsigned* bound;          // [nq] a distance no query's k-th best exceeds, shared by all CTAs
  int* error;               // set to 1 if a wait ran out
};

__device__ __forceinline__ uint32_t sh_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sh_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sh_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sh_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(sh_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// As mbar_test, but the thread may sleep in the instruction until the phase
// completes or about `ns` nanoseconds pass, instead of spinning on issue
// slots that the epilogue warps of the same SM sub-partition need.
__device__ __forceinline__ bool mbar_test_sleep(uint64_t* bar, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(sh_u32(bar)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}

constexpr uint32_t kTcSleepNs = 20000;

// Wait for the phase of `bar` with this parity; false if the CTA aborted or
// the wait ran out (which aborts it).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  const long long t0 = clock64();
  for (uint32_t i = 0;; ++i) {
    if (mbar_test_sleep(bar, parity, kTcSleepNs)) return true;
    if ((i & 15u) == 15u) {
      if (*abort) return false;
      if (clock64() - t0 > kTcWaitCycles) {
        *abort = 1;
        return false;
      }
    }
  }
}

// Bounded wait that ignores the abort flag (draining copies after an abort).
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_test(bar, parity) && clock64() - t0 < kTcWaitCycles) {
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
      ::"r"(sh_u32(dst)), "l"(map), "r"(sh_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzled layout that the TMA writes: rows of 128 bytes, 8-row groups 1024
// bytes apart (stride byte offset), descriptor version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1) << 16;           // leading byte offset (unused here)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;   // stride byte offset
  d |= static_cast<uint64_t>(1) << 46;           // version
  d |= static_cast<uint64_t>(2) << 61;           // 128-byte swizzle
  return d;
}

// The same for a 32-byte-swizzled K-major tile (rows of 32 bytes = one
// 16-coordinate MMA step, 8-row groups 256 bytes apart), swizzle mode 6.
__device__ __forceinline__ uint64_t sw32_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1) << 16;           // leading byte offset (unused here)
  d |= static_cast<uint64_t>(256 >> 4) << 32;    // stride byte offset
  d |= static_cast<uint64_t>(1) << 46;           // version
  d |= static_cast<uint64_t>(6) << 61;           // 32-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                              (static_cast<uint32_t>(kTcN >> 3) << 17) |
                              (static_cast<uint32_t>(kTcM >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(sh_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

#define ANN_R32_OUT(r)                                                                                  \
  "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),            \
      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),   \
      "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), \
      "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
#define ANN_R32_INOUT(r)                                                                                \
  "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),            \
      "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),   \
      "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), \
      "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])

// Start loading 32 consecutive accumulator columns of this thread's lane;
// the registers are valid only after tmem_wait(r).
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : ANN_R32_OUT(r)
      : "r"(taddr));
}

// Wait for this thread's tensor-memory loads; naming the registers as
// operands keeps every use of them after the wait.
__device__ __forceinline__ void tmem_wait(uint32_t (&r)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" : ANN_R32_INOUT(r) : : "memory");
}

__device__ __forceinline__ float min3f(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

__global__ void __launch_bounds__(kTcThreads, 1)
    knn_tc_kernel(const __grid_constant__ CUtensorMap qmap, const __grid_constant__ CUtensorMap qtail,
                  const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap xtail,
                  TcArgs a) {
  extern __shared__ unsigned char tc_smem_raw[];
  // 1024-byte alignment for the swizzled operand tiles
  const uint32_t raw = sh_u32(tc_smem_raw);
  unsigned char* smem = tc_smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  unsigned char* sA = smem;                                   // kTcQT x 2 atoms x 16 KB
  unsigned char* sB = sA + kTcQT * 2 * kAtomBytes;            // kTcStages x 2 atoms x 16 KB
  unsigned char* sAt = sB + kTcStages * 2 * kAtomBytes;       // kTcQT tails x 4 KB
  unsigned char* sBt = sAt + kTcQT * kTailBytes;              // kTcStages tails x 4 KB
  uint64_t* bars = reinterpret_cast<uint64_t*>(sBt + kTcStages * kTailBytes);
  uint64_t* full = bars;                    // [kTcStages]
  uint64_t* empty = bars + kTcStages;       // [kTcStages]
  uint64_t* a_full = bars + 2 * kTcStages;  // [1]
  uint64_t* acc_full = a_full + 1;          // [2]
  uint64_t* acc_empty = a_full + 3;         // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(a_full + 5);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int natoms = a.natoms;
  const int64_t q0 = static_cast<int64_t>(blockIdx.x) * (kTcQT * kTcM);
  const int s = blockIdx.y;
  const int t_lo = static_cast<int>((static_cast<int64_t>(a.tiles) * s) / a.splits);
  const int t_hi = static_cast<int>((static_cast<int64_t>(a.tiles) * (s + 1)) / a.splits);
  const int my_tiles = t_hi - t_lo;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kTcStages; ++i) {
      mbar_init(full + i, 1);
      mbar_init(empty + i, 1);
    }
    mbar_init(a_full, 1);
    mbar_init(acc_full + 0, 1);
    mbar_init(acc_full + 1, 1);
    mbar_init(acc_empty + 0, 4 * kTcQT);  // the warps of the kTcQT warpgroups of a buffer
    mbar_init(acc_empty + 1, 4 * kTcQT);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {  // 2 buffers x kTcQT query tiles x 128 columns = all 512
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(sh_u32(tmem_slot)), "r"(2 * kTcQT * kTcN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int dp = natoms * 64;  // x coordinate of the tail

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    asm volatile("prefetch.tensormap [%0];" ::"l"(&qmap) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&qtail) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&xmap) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(&xtail) : "memory");
    mbar_expect_tx(a_full, kTcQT * (natoms * kAtomBytes + kTailBytes));
    for (int qt = 0; qt < kTcQT; ++qt) {
      const int row = static_cast<int>(q0 + qt * kTcM);
      for (int at = 0; at < natoms; ++at)
        tma_load_2d(sA + (qt * 2 + at) * kAtomBytes, &qmap, a_full, 64 * at, row);
      tma_load_2d(sAt + qt * kTailBytes, &qtail, a_full, dp, row);
    }
    int issued = 0;
    bool ok = true;
    for (int i = 0; i < my_tiles && ok; ++i) {
      const int st = i % kTcStages;
      const uint32_t ph = (i / kTcStages) & 1;
      if (!mbar_wait(empty + st, ph ^ 1u, abort)) { ok = false; break; }
      mbar_expect_tx(full + st, natoms * kAtomBytes + kTailBytes);
      const int row = (t_lo + i) * kTcN;
      for (int at = 0; at < natoms; ++at)
        tma_load_2d(sB + (st * 2 + at) * kAtomBytes, &xmap, full + st, 64 * at, row);
      tma_load_2d(sBt + st * kTailBytes, &xtail, full + st, dp, row);
      issued = i + 1;
    }
    if (!ok) {
      // let the copies still in flight land before the CTA exits
      mbar_drain(a_full, 0);
      for (int i = issued - kTcStages < 0 ? 0 : issued - kTcStages; i < issued; ++i)
        mbar_drain(full + (i % kTcStages), (i / kTcStages) & 1);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    if (mbar_wait(a_full, 0, abort)) {
      tc_fence_after();
      const uint32_t a_base = sh_u32(sA), at_base = sh_u32(sAt);
      for (int i = 0; i < my_tiles; ++i) {
        const int st = i % kTcStages;
        const uint32_t ph = (i / kTcStages) & 1;
        const int b = i & 1;
        const uint32_t u = static_cast<uint32_t>(i >> 1);
        if (!mbar_wait(acc_empty + b, (u & 1u) ^ 1u, abort)) break;
        if (!mbar_wait(full + st, ph, abort)) break;
        tc_fence_after();
        const uint32_t b_base = sh_u32(sB + st * 2 * kAtomBytes);
        const uint32_t bt = sh_u32(sBt + st * kTailBytes);
        for (int qt = 0; qt < kTcQT; ++qt) {
          const uint32_t d_tmem = tmem + static_cast<uint32_t>((b * kTcQT + qt) * kTcN);
          const uint32_t aq = a_base + static_cast<uint32_t>(qt * 2 * kAtomBytes);
          for (int at = 0; at < natoms; ++at)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              // a 16-coordinate step inside a 128-byte swizzled row is 32 bytes
              const uint64_t ad = sw128_desc(aq + at * kAtomBytes) + static_cast<uint64_t>(2 * kk);
              const uint64_t bd = sw128_desc(b_base + at * kAtomBytes) + static_cast<uint64_t>(2 * kk);
              tc_mma(d_tmem, ad, bd, (at | kk) != 0);
            }
          // the tail: |x|^2's digits times their weights
          tc_mma(d_tmem, sw32_desc(at_base + static_cast<uint32_t>(qt * kTailBytes)), sw32_desc(bt), 1u);
        }
        tc_commit(empty + st);
        tc_commit(acc_full + b);
      }
    }
  } else if (warp >= 4) {
    // ---- epilogue: one query per thread, its running top-k in local memory
    const int wg = (warp - 4) >> 2;
    const int qt = wg % kTcQT;      // query tile
    const int b = wg / kTcQT;       // accumulator buffer = tiles b, b+2, ...
    const int quarter = warp & 3;   // tensor-memory lanes 32*quarter .. +31
    const int64_t gq = q0 + qt * kTcM + quarter * 32 + lane;
    const bool live = gq < a.nq;
    const float qn = live ? __ldg(a.qn + gq) : 0.f;
    const int k = a.k;
    unsigned long long top[kMaxK];
    int have = 0;
    // Bounds on the keys that can still enter the final top-k: the running
    // k-th best of the chunks folded so far (keys are distinct: ids differ),
    // and the shared per-query distance bound, which every CTA lowers to its
    // own k-th distance (k keys of one range at or below it mean no key
    // above it is in the final k).  thr_f is the same bound on v; a row past
    // the query count never qualifies.
    unsigned long long thr =
        live ? a.keys[static_cast<size_t>(gq) * a.nslots * k + (k - 1)] : 0ull;
    float thr_f = !live ? -FLT_MAX
                        : (thr == ~0ull ? FLT_MAX : static_cast<float>(static_cast<unsigned>(thr >> 32)) - qn);
    unsigned published = ~0u;  // the last distance this thread lowered the shared bound to
    auto tighten = [&](unsigned dist) {
      const unsigned long long kb = (static_cast<unsigned long long>(dist) << 32) | 0xffffffffull;
      if (kb < thr) {
        thr = kb;
        thr_f = static_cast<float>(dist) - qn;
      }
    };
    const uint32_t taddr = tmem + (static_cast<uint32_t>(quarter * 32) << 16) +
                           static_cast<uint32_t>((b * kTcQT + qt) * kTcN);

    // 32 columns of v: a tree of 3-input mins, and only if the minimum is
    // within the bound, the lane's candidates one by one
    auto scan = [&](const uint32_t (&r)[32], int j0) {
      float p[8];
#pragma unroll
      for (int g = 0; g < 8; ++g)
        p[g] = min3f(__uint_as_float(r[4 * g]), __uint_as_float(r[4 * g + 1]),
                     fminf(__uint_as_float(r[4 * g + 2]), __uint_as_float(r[4 * g + 3])));
      const float m = min3f(min3f(p[0], p[1], p[2]), min3f(p[3], p[4], p[5]), fminf(p[6], p[7]));
      if (m > thr_f) return;  // the common case: nothing within the bound
      unsigned cm = 0u;
#pragma unroll
      for (int j = 0; j < 32; ++j) cm |= static_cast<unsigned>(__uint_as_float(r[j]) <= thr_f) << j;
      while (cm) {
        const int j = __ffs(cm) - 1;
        cm &= cm - 1u;
        if (j0 + j >= a.chunk_n) break;  // rows past the end (the rest are too)
        // r[j] for a run-time j without local memory: a select tree on j's bits
        uint32_t t16[16], t8[8], t4[4], t2[2];
#pragma unroll
        for (int x = 0; x < 16; ++x) t16[x] = (j & 1) ? r[2 * x + 1] : r[2 * x];
#pragma unroll
        for (int x = 0; x < 8; ++x) t8[x] = (j & 2) ? t16[2 * x + 1] : t16[2 * x];
#pragma unroll
        for (int x = 0; x < 4; ++x) t4[x] = (j & 4) ? t8[2 * x + 1] : t8[2 * x];
#pragma unroll
        for (int x = 0; x < 2; ++x) t2[x] = (j & 8) ? t4[2 * x + 1] : t4[2 * x];
        const float vj = __uint_as_float((j & 16) ? t2[1] : t2[0]);
        if (vj > thr_f) continue;  // the bound tightened after the mask was taken
        // v and |q|^2 are integers below 2^24: the sum is the exact distance
        const unsigned dist = __float2uint_rn(vj + qn);
        const unsigned long long key =
            (static_cast<unsigned long long>(dist) << 32) | static_cast<unsigned>(a.id0 + j0 + j);
        if (key >= thr) continue;
        int pos = have < k ? have : k - 1;
        while (pos > 0 && top[pos - 1] > key) {
          top[pos] = top[pos - 1];
          --pos;
        }
        top[pos] = key;
        if (have < k) ++have;
        if (have == k) {
          const unsigned long long kth = top[k - 1];
          if (kth < thr) {
            thr = kth;
            thr_f = static_cast<float>(static_cast<unsigned>(kth >> 32)) - qn;
          }
          const unsigned kd = static_cast<unsigned>(kth >> 32);
          if (kd < published) {
            atomicMin(a.bound + gq, kd);
            published = kd;
          }
        }
      }
    };

    // the shared bound is read one tile ahead, off the critical path
    unsigned next_bound = live ? __ldcg(a.bound + gq) : ~0u;
    for (int i = b; i < my_tiles; i += 2) {
      const uint32_t u = static_cast<uint32_t>(i >> 1);
      // one lane waits, so the warp stays converged for tcgen05.ld
      int ok = 1;
      if (lane == 0) ok = mbar_wait(acc_full + b, u & 1u, abort) ? 1 : 0;
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
      tc_fence_after();
      if (live) {
        tighten(next_bound);
        next_bound = __ldcg(a.bound + gq);
      }
      const int col0 = (t_lo + i) * kTcN;
      // the next 32 columns load while the current ones are scanned; the
      // accumulator goes back to the MMA once its last columns are in
      // registers
      uint32_t r0[32], r1[32];
      tmem_ld32_async(taddr, r0);
      tmem_wait(r0);
      tmem_ld32_async(taddr + 32u, r1);
      scan(r0, col0);
      tmem_wait(r1);
      tmem_ld32_async(taddr + 64u, r0);
      scan(r1, col0 + 32);
      tmem_wait(r0);
      tmem_ld32_async(taddr + 96u, r1);
      scan(r0, col0 + 64);
      tmem_wait(r1);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty + b);
      scan(r1, col0 + 96);
    }
    if (live) {
      unsigned long long* out =
          a.keys + (static_cast<size_t>(gq) * a.nslots + 1 + 2 * s + b) * static_cast<size_t>(k);
      for (int j = 0; j < k; ++j) out[j] = j < have ? top[j] : ~0ull;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x == 0 && *abort) atomicExch(a.error, 1);
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTcQT * kTcN)
                 : "memory");
  }
}

// BF16 of a small integer or power of two (exact: at most 8 significant bits).
__device__ __forceinline__ uint16_t bf16_exact(float v) {
  return static_cast<uint16_t>(__float_as_uint(v) >> 16);
}

// Base rows -> BF16 B rows of w = dp + kTail coordinates: -2 x_1 .. -2 x_d,
// zeros to dp, then the base-256 digits of |x|^2 (high, middle, low) and
// zeros.  Rows in [rows, rows_pad) get zero coordinates and digits 255, 255,
// 255: v = 2^24 - 1, above every real v.  One warp per row.
__global__ void base_rows_bf16(const uint8_t* __restrict__ x, int64_t rows, int64_t rows_pad, int d, int dp,
                               uint16_t* __restrict__ out) {
  const int64_t r = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= rows_pad) return;
  const bool real = r < rows;
  const uint8_t* src = x + (real ? r : 0) * d;
  const int w = dp + kTail;
  uint16_t* dst = out + r * w;
  unsigned sq = 0;
  for (int j = lane; j < dp; j += 32) {
    const unsigned v = (real && j < d) ? src[j] : 0u;
    sq += v * v;
    dst[j] = bf16_exact(-2.f * static_cast<float>(v));
  }
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if (lane < kTail) {
    unsigned digit = 0;
    if (lane < 3) digit = real ? (sq >> (8 * (2 - lane))) & 0xffu : 0xffu;
    dst[dp + lane] = bf16_exact(static_cast<float>(digit));
  }
}

// Query rows -> BF16 A rows: q_1 .. q_d, zeros to dp, then the digit weights
// 2^16, 2^8, 1 and zeros; and each row's squared norm (an exact integer in
// FP32).  Rows in [rows, rows_pad) are zero.  One warp per row.
__global__ void query_rows_bf16(const uint8_t* __restrict__ q, int64_t rows, int64_t rows_pad, int d, int dp,
                                uint16_t* __restrict__ out, float* __restrict__ norms) {
  const int64_t r = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= rows_pad) return;
  const bool real = r < rows;
  const uint8_t* src = q + (real ? r : 0) * d;
  const int w = dp + kTail;
  uint16_t* dst = out + r * w;
  unsigned sq = 0;
  for (int j = lane; j < dp; j += 32) {
    const unsigned v = (real && j < d) ? src[j] : 0u;
    sq += v * v;
    dst[j] = bf16_exact(static_cast<float>(v));
  }
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if (lane < kTail) {
    const float wt = (real && lane < 3) ? static_cast<float>(1u << (8 * (2 - lane))) : 0.f;
    dst[dp + lane] = bf16_exact(wt);
  }
  if (lane == 0) norms[r] = static_cast<float>(sq);
}

// Merge the parts of every query into its running top-k (slot 0) and clear
// the parts for the next chunk.
__global__ void __launch_bounds__(256) topk_fold(unsigned long long* __restrict__ keys, int nslots, int k) {
  __shared__ unsigned long long best[kMaxK];
  unsigned long long* p = keys + static_cast<size_t>(blockIdx.x) * nslots * k;
  block_topk([&](int64_t i) { return p[i]; }, static_cast<int64_t>(nslots) * k, k, best);
  __syncthreads();
  for (int i = threadIdx.x; i < nslots * k; i += blockDim.x) p[i] = i < k ? best[i] : ~0ull;
}

// Keys of slot 0 -> ids and exact integer distances.
__global__ void topk_write(const unsigned long long* __restrict__ keys, int64_t nq, int nslots, int k,
                           int32_t* __restrict__ ids, float* __restrict__ dists) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= nq * k) return;
  const int64_t q = i / k, j = i % k;
  const unsigned long long b = keys[static_cast<size_t>(q) * nslots * k + j];
  const bool ok = b != ~0ull;
  ids[i] = ok ? static_cast<int32_t>(b & 0xffffffffu) : -1;
  dists[i] = ok ? static_cast<float>(static_cast<unsigned>(b >> 32)) : __int_as_float(0x7f800000);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2-D map of `rows` BF16 rows of `w` coordinates with box_x x 128 boxes:
// 64-coordinate boxes in the 128-byte swizzle for the atoms, 16-coordinate
// boxes in the 32-byte swizzle for the tail.  Every box the kernel loads lies
// inside the buffer.
bool bf16_row_map(CUtensorMap* m, const void* ptr, int64_t rows, int w, int box_x, bool tail) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(w), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(w) * 2};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(box_x), 128};
  cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, tail ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

constexpr size_t kTcSmem = 1024 + kTcQT * 2 * kAtomBytes + kTcStages * 2 * kAtomBytes + kTcQT * kTailBytes +
                           kTcStages * kTailBytes + 256;

}  // namespace

// Exact kNN of uint8 data on the tensor cores (d <= 128, k <= 128), device
// buffers.  The base is processed in chunks of up to 2^22 rows, each
// converted to BF16 into one scratch buffer.
cudaError_t knn_exact_tc(const uint8_t* base, int64_t n, int d, const uint8_t* queries, int64_t nq, int k,
                         int32_t* ids, float* dists, cudaStream_t stream, int* timed_out) {
  if (d > 128 || k > kMaxK || n >= (1ll << 31)) return cudaErrorInvalidValue;
  if (timed_out) *timed_out = 0;
  if (nq == 0) return cudaSuccess;
  const int dp = d <= 64 ? 64 : 128;
  const int natoms = dp / 64;
  const int64_t chunk = n < (1ll << 22) ? n : (1ll << 22);
  const int64_t qblocks = (nq + kTcQT * kTcM - 1) / (kTcQT * kTcM);
  const int max_tiles = static_cast<int>((chunk + kTcN - 1) / kTcN);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // CTAs (one per SM at a time): at least four waves, each CTA over >= 8
  // tiles, and among up to 4x the least such count the one that fills its
  // last wave best
  const int s_lo = static_cast<int>((4ll * sms + qblocks - 1) / qblocks);
  const int s_hi = max_tiles / 8 < 1 ? 1 : max_tiles / 8;
  int splits = s_lo < s_hi ? s_lo : s_hi;
  double best_fill = -1.0;
  for (int sp = splits; sp <= s_hi && sp <= 4 * s_lo; ++sp) {
    const int64_t ctas = qblocks * sp;
    const int64_t waves = (ctas + sms - 1) / sms;
    const double fill = static_cast<double>(ctas) / static_cast<double>(waves * sms);
    if (fill > best_fill + 1e-9) {
      best_fill = fill;
      splits = sp;
    }
  }
  const int nslots = 1 + 2 * splits;
  uint16_t *qb = nullptr, *xb = nullptr;
  float* qn = nullptr;
  unsigned long long* keys = nullptr;
  unsigned* bound = nullptr;
  int* err = nullptr;
  // row buffers of w = dp + kTail coordinates, padded to whole boxes (see
  // base_rows_bf16 / query_rows_bf16), so every TMA box lies inside them
  const int w = dp + kTail;
  const int64_t q_rows = qblocks * kTcQT * kTcM;
  const int64_t x_rows = static_cast<int64_t>(max_tiles) * kTcN;
  cudaError_t e = cudaMalloc(&qb, static_cast<size_t>(q_rows) * w * 2);
  if (e == cudaSuccess) e = cudaMalloc(&qn, static_cast<size_t>(q_rows) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&xb, static_cast<size_t>(x_rows) * w * 2);
  if (e == cudaSuccess) e = cudaMalloc(&keys, static_cast<size_t>(nq) * nslots * k * 8);
  if (e == cudaSuccess) e = cudaMalloc(&bound, static_cast<size_t>(nq) * 4);
  if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(bound, 0xff, static_cast<size_t>(nq) * 4, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(keys, 0xff, static_cast<size_t>(nq) * nslots * k * 8, stream);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(knn_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kTcSmem));
  CUtensorMap qmap, qtail, xmap, xtail;
  if (e == cudaSuccess) {
    query_rows_bf16<<<static_cast<unsigned>((q_rows * 32 + 255) / 256), 256, 0, stream>>>(queries, nq, q_rows, d,
                                                                                        dp, qb, qn);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && (!bf16_row_map(&qmap, qb, q_rows, w, 64, false) ||
                           !bf16_row_map(&qtail, qb, q_rows, w, kTail, true)))
    e = cudaErrorInvalidValue;
  // The first chunk is small (2^17 rows): once it is folded, every query's
  // running k-th best over it bounds the keys of all later chunks, so their
  // CTAs start with a tight bound instead of each warming up its own.
  const int64_t seed_rows = chunk < (1ll << 17) ? chunk : (1ll << 17);
  for (int64_t c0 = 0; c0 < n && e == cudaSuccess;) {
    const int64_t cmax = c0 == 0 ? seed_rows : chunk;
    const int64_t cn = (n - c0 < cmax) ? n - c0 : cmax;
    const int64_t map_rows = (cn + kTcN - 1) / kTcN * kTcN;
    base_rows_bf16<<<static_cast<unsigned>((map_rows * 32 + 255) / 256), 256, 0, stream>>>(base + c0 * d, cn,
                                                                                         map_rows, d, dp, xb);
    if (!bf16_row_map(&xmap, xb, map_rows, w, 64, false) || !bf16_row_map(&xtail, xb, map_rows, w, kTail, true)) {
      e = cudaErrorInvalidValue;
      break;
    }
    TcArgs ta;
    ta.qn = qn;
    ta.nq = nq;
    ta.chunk_n = static_cast<int32_t>(cn);
    ta.id0 = c0;
    ta.tiles = static_cast<int32_t>((cn + kTcN - 1) / kTcN);
    ta.splits = splits < ta.tiles ? splits : ta.tiles;
    ta.natoms = natoms;
    ta.k = k;
    ta.nslots = nslots;
    ta.keys = keys;
    ta.bound = bound;
    ta.error = err;
    knn_tc_kernel<<<dim3(static_cast<unsigned>(qblocks), static_cast<unsigned>(ta.splits)), kTcThreads, kTcSmem,
                    stream>>>(qmap, qtail, xmap, xtail, ta);
    topk_fold<<<static_cast<unsigned>(nq), 256, 0, stream>>>(keys, nslots, k);
    e = cudaGetLastError();
    c0 += cn;
  }
  if (e == cudaSuccess) {
    topk_write<<<static_cast<unsigned>((nq * k + 255) / 256), 256, 0, stream>>>(keys, nq, nslots, k, ids, dists);
    e = cudaGetLastError();
  }
  int h_err = 0;
  cudaError_t e2 = cudaStreamSynchronize(stream);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess && err) e = cudaMemcpy(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost);
  if (timed_out) *timed_out = h_err;
  cudaFree(qb);
  cudaFree(qn);
  cudaFree(xb);
  cudaFree(keys);
  cudaFree(bound);
  cudaFree(err);
  return e;
}

cudaError_t knn_exact_cuda_cores(const void* base, int dtype, int64_t n, int d, const void* queries,
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

// Engine choice: 0 = tensor cores where the data allow (uint8, d <= 128),
// 1 = tensor cores (uint8, d <= 128 only), 2 = CUDA cores.
cudaError_t knn_exact_device(const void* base, int dtype, int64_t n, int d, const void* queries,
                             int64_t nq, int k, int32_t* ids, float* dists, cudaStream_t stream,
                             int engine, int* timed_out) {
  if (timed_out) *timed_out = 0;
  const bool tc_ok = dtype == ANN_U8 && d <= 128 && k <= kMaxK;
  if (engine == 1 && !tc_ok) return cudaErrorInvalidValue;
  if (engine != 2 && tc_ok)
    return knn_exact_tc(static_cast<const uint8_t*>(base), n, d, static_cast<const uint8_t*>(queries), nq, k,
                        ids, dists, stream, timed_out);
  return knn_exact_cuda_cores(base, dtype, n, d, queries, nq, k, ids, dists, stream);
}

}  // namespace ann
