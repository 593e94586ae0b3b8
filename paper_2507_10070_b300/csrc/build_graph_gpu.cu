// ann_build_graph_gpu: Vamana graph construction on the GPU (index-build
// tooling, off the search path).  Same algorithm and batch schedule as the
// host builder (build_graph.cpp): random start graph, one pass with alpha = 1
// and one with `alpha`, nodes inserted in batches that grow geometrically up
// to 2% of n, every search of a batch reading the graph as it stood before
// the batch.  The start graph and the insertion order are drawn on the device
// from a counter-based generator (node i's draws depend only on the seed and
// i), so they take no host time or host copy of the graph at 10^8 nodes; they
// are therefore other random draws than the host builder's.
//
// Per batch:
//  1. gather the batch's vectors;
//  2. GreedySearch(entry, x_p, L_build) for all of them at once with the
//     library's search kernel (exact navigation on the vectors in HBM,
//     depth 0); the expanded nodes nearest to x_p, up to L_build + 64 (at
//     most 256 - R), form the candidate pool -- in practice the whole
//     expanded set, as in DiskANN;
//  3. RobustPrune(p, pool u N(p)) -- for uint8 rows with d <= 128 one block
//     per node with the candidate distances on the tensor cores
//     (prune_tc_kernel), otherwise one warp per node (prune_kernel);
//  4. back edges j <- p: the (j, p) pairs are sorted on the device (CUB
//     radix sort), grouped by j, and each target appends its new sources or,
//     if they do not fit in R, prunes N(j) u sources (the prune again).
// alpha is compared with squared distances (DiskANN's convention).  Every
// step is deterministic, so the graph does not depend on timing.
#include <cub/cub.cuh>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#include "ann_internal.h"

namespace ann {
namespace {

constexpr int kCandMax = 256;  // candidates one prune task considers
constexpr unsigned kFull = 0xffffffffu;

constexpr uint64_t kGolden = 0x9e3779b97f4a7c15ull;

// splitmix64's output function (Steele, Lea and Flood, OOPSLA 2014).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Start graph: node i draws init_deg distinct out-neighbours != i from its own
// splitmix64 sequence, started at seed ^ mix64(i + 1).  The rejection loop is
// capped; past the cap (only reachable when init_deg is close to n - 1) the
// row is completed by a scan in id order.
__global__ void random_rows(int64_t n, int init_deg, uint64_t seed, int32_t* __restrict__ adj,
                            int stride) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t* row = adj + static_cast<size_t>(i) * stride;
  uint64_t s = seed ^ mix64(static_cast<uint64_t>(i) + 1);
  int c = 0;
  for (int it = 0; c < init_deg && it < 64 * init_deg + 1024; ++it) {
    s += kGolden;
    const int32_t v = static_cast<int32_t>(mix64(s) % static_cast<uint64_t>(n));
    bool dup = v == i;
    for (int j = 0; j < c; ++j) dup |= row[j] == v;
    if (!dup) row[c++] = v;
  }
  for (int64_t v = 0; c < init_deg && v < n; ++v) {
    bool dup = v == i;
    for (int j = 0; j < c; ++j) dup |= row[j] == v;
    if (!dup) row[c++] = static_cast<int32_t>(v);
  }
  for (int j = c; j < stride; ++j) row[j] = -1;
}

// Insertion order: nodes sorted by a per-node 64-bit hash (ties by id, the
// sort being stable), i.e. a uniformly random permutation.
__global__ void order_keys(int64_t n, uint64_t seed, unsigned long long* __restrict__ key,
                           int32_t* __restrict__ id) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  key[i] = mix64(mix64(seed ^ 0x5851f42d4c957f2dull) + static_cast<uint64_t>(i) * kGolden);
  id[i] = static_cast<int32_t>(i);
}

__global__ void gather_rows(const uint8_t* __restrict__ base, int row_bytes,
                            const int32_t* __restrict__ ids, int n, uint8_t* __restrict__ out) {
  const int r = blockIdx.x;
  if (r >= n) return;
  const uint32_t* src = reinterpret_cast<const uint32_t*>(base + (size_t)ids[r] * row_bytes);
  uint32_t* dst = reinterpret_cast<uint32_t*>(out + (size_t)r * row_bytes);
  for (int j = threadIdx.x; j < row_bytes / 4; j += blockDim.x) dst[j] = src[j];
}

// Squared distance between rows a and b, computed by one thread.
template <bool U8>
__device__ __forceinline__ float row_dist(const void* base, int d, int a, int b) {
  if (U8) {
    const uint4* x = reinterpret_cast<const uint4*>(static_cast<const uint8_t*>(base) + (size_t)a * d);
    const uint4* y = reinterpret_cast<const uint4*>(static_cast<const uint8_t*>(base) + (size_t)b * d);
    unsigned acc = 0;
    for (int j = 0; j < d / 16; ++j) {
      const uint4 u = __ldg(x + j), v = __ldg(y + j);
      unsigned t;
      t = __vabsdiffu4(u.x, v.x); acc = __dp4a(t, t, acc);
      t = __vabsdiffu4(u.y, v.y); acc = __dp4a(t, t, acc);
      t = __vabsdiffu4(u.z, v.z); acc = __dp4a(t, t, acc);
      t = __vabsdiffu4(u.w, v.w); acc = __dp4a(t, t, acc);
    }
    return static_cast<float>(acc);
  } else {
    const float4* x = reinterpret_cast<const float4*>(static_cast<const float*>(base) + (size_t)a * d);
    const float4* y = reinterpret_cast<const float4*>(static_cast<const float*>(base) + (size_t)b * d);
    float acc = 0.f;
    for (int j = 0; j < d / 4; ++j) {
      const float4 u = __ldg(x + j), v = __ldg(y + j);
      float t;
      t = u.x - v.x; acc = fmaf(t, t, acc);
      t = u.y - v.y; acc = fmaf(t, t, acc);
      t = u.z - v.z; acc = fmaf(t, t, acc);
      t = u.w - v.w; acc = fmaf(t, t, acc);
    }
    return acc;
  }
}

__device__ __forceinline__ unsigned long long pkey(float d, int id) {
  return (static_cast<unsigned long long>(__float_as_uint(d)) << 32) | static_cast<unsigned>(id);
}

// One warp per task: candidates = the node's current row (if include_row)
// plus extra ids; deduplicated, self removed, sorted by (distance, id).  If
// `append_if_fits` and they fit in R they become the row; otherwise
// RobustPrune keeps <= R of them.  Rows are adj_stride ids, -1 padded.
template <bool U8>
__global__ void prune_kernel(const void* __restrict__ base, int d, int R, float alpha,
                             const int32_t* __restrict__ task_node,
                             const int32_t* __restrict__ extra, const int64_t* __restrict__ extra_off,
                             const int32_t* __restrict__ extra_cnt, int ntasks, int include_row,
                             int append_if_fits, int32_t* __restrict__ adj, int adj_stride) {
  __shared__ unsigned long long keys[4][kCandMax];
  __shared__ unsigned char gone[4][kCandMax];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int task = blockIdx.x * 4 + wib;
  if (task >= ntasks) return;  // warp-uniform
  unsigned long long* K = keys[wib];
  unsigned char* G = gone[wib];
  const int p = task_node[task];
  int32_t* row = adj + (size_t)p * adj_stride;
  // collect candidate ids
  int nrow = 0;
  if (include_row)
    for (int j = 0; j < R; ++j) {
      if (row[j] < 0) break;
      ++nrow;
    }
  const int ne = min(extra_cnt[task], kCandMax - nrow);
  const int32_t* ex = extra + extra_off[task];
  const int nc = nrow + ne;
  for (int c = lane; c < kCandMax; c += 32) {
    unsigned long long key = ~0ull;
    if (c < nc) {
      const int id = c < nrow ? row[c] : ex[c - nrow];
      if (id >= 0 && id != p) key = pkey(row_dist<U8>(base, d, p, id), id);
    }
    K[c] = key;
  }
  __syncwarp();
  // sort the keys (bitonic, shared memory): only the first P, the least
  // power of two >= the candidate count, since every later key is the ~0
  // sentinel and already in place
  int P = 32;
  while (P < nc) P <<= 1;
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = lane; i < P; i += 32) {
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
  // drop duplicates (equal keys are adjacent), count valid
  for (int c = lane; c < kCandMax; c += 32) G[c] = (K[c] == ~0ull || (c > 0 && K[c] == K[c - 1])) ? 1 : 0;
  __syncwarp();
  int valid = 0;
  for (int c = lane; c < kCandMax; c += 32) valid += G[c] ? 0 : 1;
  for (int o = 16; o > 0; o >>= 1) valid += __shfl_xor_sync(kFull, valid, o);
  int kept = 0;
  if (append_if_fits && valid <= R) {
    // every unique candidate fits: it becomes the row
    for (int c = 0; c < kCandMax; ++c) {
      if (G[c]) continue;
      if (lane == 0) row[kept] = static_cast<int32_t>(K[c] & 0xffffffffu);
      ++kept;
    }
  } else {
    for (int i = 0; i < kCandMax && kept < R; ++i) {
      if (G[i]) continue;  // warp-uniform (shared memory, synced)
      const int ci = static_cast<int>(K[i] & 0xffffffffu);
      if (lane == 0) row[kept] = ci;
      ++kept;
      for (int j = i + 1 + lane; j < kCandMax; j += 32) {
        if (G[j]) continue;
        const int cj = static_cast<int>(K[j] & 0xffffffffu);
        const float dpj = __uint_as_float(static_cast<unsigned>(K[j] >> 32));
        if (alpha * row_dist<U8>(base, d, ci, cj) <= dpj) G[j] = 1;
      }
      __syncwarp();
    }
  }
  __syncwarp();
  for (int j = kept + lane; j < adj_stride; j += 32) row[j] = -1;
}

// RobustPrune for uint8 rows with d <= 128 with the candidate distances on the
// tensor cores.  One block of four warps per task.
//  1. The candidates' rows are staged in shared memory as BF16 (exact for
//     8-bit values), with each row's squared norm and its exact integer
//     distance to p (8 threads per row, __vabsdiffu4 + __dp4a).
//  2. (distance to p, id) keys are sorted (bitonic, 256 entries) and
//     deduplicated into the unique candidates in prune order.
//  3. If the task may append and they fit in R, they become the row.
//     Otherwise every pair i < j of them gets d(c_i, c_j) = |c_i|^2 +
//     |c_j|^2 - 2 c_i.c_j from BF16 MMAs with FP32 accumulation
//     (mma.sync m16n8k16).  For uint8 rows with d <= 128 every partial sum is
//     an integer below 2^24, so this is exact in any order.  The result is
//     a bit matrix B[i][j] = (alpha * d(c_i, c_j) <= d(p, c_j)).
//  4. One warp walks the candidates in order: a candidate not yet pruned is
//     kept, and its row of B prunes the later ones, until R are kept.
// Every comparison is the one prune_kernel<true> makes, on the same exact
// float values, so both give the same rows.
constexpr int kTcPruneStride = 136;  // BF16 elements per staged row: 128 + 8 (bank spread)
constexpr int kTcPruneThreads = 128;
constexpr size_t kTcPruneSmem = (size_t)(kCandMax + 1) * kTcPruneStride * 2  // rows + one zero row
                                + kCandMax * 8                               // keys
                                + kCandMax * 4 * 2                           // norms, ids
                                + kCandMax * 2                               // sorted -> slot, unique -> sorted
                                + kCandMax * 32                              // bit matrix
                                + 16;

__device__ __forceinline__ uint32_t bf16x2_of_bytes(uint32_t w, int hi) {
  // bytes 2*hi and 2*hi+1 of w as two BF16 values (exact: 8-bit integers)
  const uint32_t b0 = (w >> (16 * hi)) & 0xffu, b1 = (w >> (16 * hi + 8)) & 0xffu;
  const uint32_t h0 = __float_as_uint(static_cast<float>(b0)) >> 16;
  const uint32_t h1 = __float_as_uint(static_cast<float>(b1)) >> 16;
  return h0 | (h1 << 16);
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t& r0, uint32_t& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}

__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(kTcPruneThreads)
    prune_tc_kernel(const uint8_t* __restrict__ base, int d, int R, float alpha,
                    const int32_t* __restrict__ task_node, const int32_t* __restrict__ extra,
                    const int64_t* __restrict__ extra_off, const int32_t* __restrict__ extra_cnt,
                    int include_row, int append_if_fits, int32_t* __restrict__ adj, int adj_stride) {
  extern __shared__ __align__(16) unsigned char prune_smem[];
  uint16_t* X = reinterpret_cast<uint16_t*>(prune_smem);                        // [257][136] BF16
  unsigned long long* K = reinterpret_cast<unsigned long long*>(X + (kCandMax + 1) * kTcPruneStride);
  float* nrm = reinterpret_cast<float*>(K + kCandMax);                          // |x|^2 by slot
  int32_t* cid = reinterpret_cast<int32_t*>(nrm + kCandMax);                    // id by slot (-1: none)
  uint8_t* slot = reinterpret_cast<uint8_t*>(cid + kCandMax);                   // sorted position -> slot
  uint8_t* U = slot + kCandMax;                                                 // unique position -> sorted
  uint32_t* bits = reinterpret_cast<uint32_t*>(U + kCandMax);                   // [256][8]
  int* misc = reinterpret_cast<int*>(bits + kCandMax * 8);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int task = blockIdx.x;
  const int p = task_node[task];
  int32_t* row = adj + (size_t)p * adj_stride;
  if (tid == 0) {
    int nrow = 0;
    if (include_row)
      while (nrow < R && row[nrow] >= 0) ++nrow;
    misc[0] = nrow;
  }
  __syncthreads();
  const int nrow = misc[0];
  const int ne = min(extra_cnt[task], kCandMax - nrow);
  const int32_t* ex = extra + extra_off[task];
  const int nc = nrow + ne;
  for (int c = tid; c < kCandMax; c += kTcPruneThreads) {
    int id = -1;
    if (c < nc) {
      id = c < nrow ? row[c] : ex[c - nrow];
      if (id == p) id = -1;
    }
    cid[c] = id;
    slot[c] = static_cast<uint8_t>(c);
  }
  // the zero row that fills MMA tiles past the last candidate
  for (int j = tid; j < kTcPruneStride / 2; j += kTcPruneThreads)
    reinterpret_cast<uint32_t*>(X + kCandMax * kTcPruneStride)[j] = 0u;
  __syncthreads();

  // 1. stage rows, norms and exact distances to p: 8 threads per row, 16
  // coordinates each
  const int segs = d >> 4, sub = tid & 7, grp = tid >> 3;
  uint4 pv = make_uint4(0u, 0u, 0u, 0u);
  if (sub < segs) pv = __ldg(reinterpret_cast<const uint4*>(base + (size_t)p * d) + sub);
  constexpr int kRowsPerPass = kTcPruneThreads / 8;
  constexpr int kBatch = 8;  // row loads a thread has in flight at once
  for (int c00 = 0; c00 < kCandMax; c00 += kRowsPerPass * kBatch) {
    uint4 vb[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int id = cid[c00 + u * kRowsPerPass + grp];
      vb[u] = (id >= 0 && sub < segs) ? __ldg(reinterpret_cast<const uint4*>(base + (size_t)id * d) + sub)
                                      : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int c = c00 + u * kRowsPerPass + grp;
      const int id = cid[c];
      const uint4 v = vb[u];
      unsigned nn = 0, dd = 0, t;
      nn = __dp4a(v.x, v.x, nn);
      nn = __dp4a(v.y, v.y, nn);
      nn = __dp4a(v.z, v.z, nn);
      nn = __dp4a(v.w, v.w, nn);
      t = __vabsdiffu4(v.x, pv.x); dd = __dp4a(t, t, dd);
      t = __vabsdiffu4(v.y, pv.y); dd = __dp4a(t, t, dd);
      t = __vabsdiffu4(v.z, pv.z); dd = __dp4a(t, t, dd);
      t = __vabsdiffu4(v.w, pv.w); dd = __dp4a(t, t, dd);
      if (sub < segs) {
        uint4 w0, w1;
        w0.x = bf16x2_of_bytes(v.x, 0); w0.y = bf16x2_of_bytes(v.x, 1);
        w0.z = bf16x2_of_bytes(v.y, 0); w0.w = bf16x2_of_bytes(v.y, 1);
        w1.x = bf16x2_of_bytes(v.z, 0); w1.y = bf16x2_of_bytes(v.z, 1);
        w1.z = bf16x2_of_bytes(v.w, 0); w1.w = bf16x2_of_bytes(v.w, 1);
        uint4* dst = reinterpret_cast<uint4*>(X + c * kTcPruneStride + sub * 16);
        dst[0] = w0;
        dst[1] = w1;
      }
      for (int o = 1; o < 8; o <<= 1) {
        nn += __shfl_xor_sync(kFull, nn, o);
        dd += __shfl_xor_sync(kFull, dd, o);
      }
      if (sub == 0) {
        nrm[c] = static_cast<float>(nn);
        K[c] = id >= 0 ? pkey(static_cast<float>(dd), id) : ~0ull;
      }
    }
  }
  __syncthreads();

  // 2. sort (key, slot) ascending over the first P keys, the least power of
  // two >= the candidate count (every later key is the ~0 sentinel)
  int P = 32;
  while (P < nc) P <<= 1;
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (tid < P / 2) {
        const int i = (tid / stride) * 2 * stride + (tid % stride), j = i + stride;
        const bool asc = (i & size) == 0;
        const unsigned long long a = K[i], b = K[j];
        if ((a > b) == asc) {
          K[i] = b;
          K[j] = a;
          const uint8_t t = slot[i];
          slot[i] = slot[j];
          slot[j] = t;
        }
      }
      __syncthreads();
    }
  }
  // deduplicate (equal keys are the same id) into prune order
  if (warp == 0) {
    int nu = 0;
    for (int c0 = 0; c0 < kCandMax; c0 += 32) {
      const int c = c0 + lane;
      const unsigned long long k = K[c];
      const bool keep = k != ~0ull && (c == 0 || K[c - 1] != k);
      const unsigned m = __ballot_sync(kFull, keep);
      if (keep) U[nu + __popc(m & ((1u << lane) - 1u))] = static_cast<uint8_t>(c);
      nu += __popc(m);
    }
    if (lane == 0) misc[1] = nu;
  }
  for (int w = tid; w < kCandMax * 8; w += kTcPruneThreads) bits[w] = 0u;
  __syncthreads();
  const int V = misc[1];

  if (append_if_fits && V <= R) {
    // every unique candidate fits: it becomes the row
    if (warp == 0) {
      for (int u = lane; u < V; u += 32) row[u] = static_cast<int32_t>(K[U[u]] & 0xffffffffu);
      for (int j = V + lane; j < adj_stride; j += 32) row[j] = -1;
    }
    return;
  }

  // 3. the pruning relation of every pair i < j, as bits
  const uint32_t xs = static_cast<uint32_t>(__cvta_generic_to_shared(X));
  const int nti = (V + 15) >> 4, ntj = (V + 7) >> 3;
  const int g = lane >> 2, cq = lane & 3;
  for (int ti = warp; ti < nti; ti += kTcPruneThreads / 32) {
    // A fragments of rows ti*16 .. +15, every k step (16 coordinates)
    uint32_t af[8][4];
    {
      const int r = (lane & 7) + ((lane >> 3) & 1) * 8, kofs = (lane >> 4) * 8;
      const int i = ti * 16 + r;
      const int srow = i < V ? slot[U[i]] : kCandMax;
      const uint32_t rowaddr = xs + static_cast<uint32_t>((srow * kTcPruneStride + kofs) * 2);
#pragma unroll
      for (int kk = 0; kk < 8; ++kk)
        if (kk < segs) ldsm_x4(rowaddr + kk * 32, af[kk][0], af[kk][1], af[kk][2], af[kk][3]);
    }
    // this thread's two rows of the accumulator: g and g + 8
    const int i0 = ti * 16 + g, i1 = i0 + 8;
    const float n0 = i0 < V ? nrm[slot[U[i0]]] : 0.f, n1 = i1 < V ? nrm[slot[U[i1]]] : 0.f;
    for (int tj = (ti * 16) >> 3; tj < ntj; ++tj) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      {
        const int n = lane & 7, kofs = ((lane >> 3) & 1) * 8 + (lane >> 4) * 16;
        const int j = tj * 8 + n;
        const int srow = j < V ? slot[U[j]] : kCandMax;
        const uint32_t rowaddr = xs + static_cast<uint32_t>((srow * kTcPruneStride) * 2);
#pragma unroll
        for (int kk = 0; kk < 8; kk += 2) {
          if (kk + 1 < segs) {
            uint32_t b0, b1, b2, b3;
            ldsm_x4(rowaddr + static_cast<uint32_t>((kk * 16 + kofs) * 2), b0, b1, b2, b3);
            mma_bf16_16816(acc, af[kk], b0, b1);
            mma_bf16_16816(acc, af[kk + 1], b2, b3);
          } else if (kk < segs) {
            uint32_t b0, b1;
            ldsm_x2(rowaddr + static_cast<uint32_t>((kk * 16 + (kofs & 8)) * 2), b0, b1);
            mma_bf16_16816(acc, af[kk], b0, b1);
          }
        }
      }
      // accumulator (row g / g+8, columns 2cq, 2cq+1) -> pruning bits
      unsigned byte0 = 0u, byte1 = 0u;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int j = tj * 8 + 2 * cq + e;
        if (j < V) {
          const int sj = slot[U[j]];
          const float nj = nrm[sj];
          const float dpj = __uint_as_float(static_cast<unsigned>(K[U[j]] >> 32));
          // |c_i|^2 + |c_j|^2 and 2 c_i.c_j are exact integers below 2^24, so
          // is their difference: the same float row_dist gives
          const float d0 = (n0 + nj) - 2.f * acc[e];
          const float d1 = (n1 + nj) - 2.f * acc[2 + e];
          if (i0 < j && alpha * d0 <= dpj) byte0 |= 1u << (2 * cq + e);
          if (i1 < j && alpha * d1 <= dpj) byte1 |= 1u << (2 * cq + e);
        }
      }
      byte0 |= __shfl_xor_sync(kFull, byte0, 1);
      byte0 |= __shfl_xor_sync(kFull, byte0, 2);
      byte1 |= __shfl_xor_sync(kFull, byte1, 1);
      byte1 |= __shfl_xor_sync(kFull, byte1, 2);
      if (cq == 0) {
        uint8_t* bb = reinterpret_cast<uint8_t*>(bits);
        if (i0 < V) bb[i0 * 32 + tj] = static_cast<uint8_t>(byte0);
        if (i1 < V) bb[i1 * 32 + tj] = static_cast<uint8_t>(byte1);
      }
    }
  }
  __syncthreads();

  // 4. keep candidates in order; each kept one prunes the later ones of its row
  if (warp == 0) {
    unsigned gone = 0u;  // lane w < 8: candidates 32w .. 32w + 31
    int kept = 0;
    for (int i = 0; i < V && kept < R; ++i) {
      const unsigned gw = __shfl_sync(kFull, gone, i >> 5);
      if ((gw >> (i & 31)) & 1u) continue;
      if (lane == 0) row[kept] = static_cast<int32_t>(K[U[i]] & 0xffffffffu);
      ++kept;
      if (lane < 8) gone |= bits[i * 8 + lane];
    }
    for (int j = kept + lane; j < adj_stride; j += 32) row[j] = -1;
  }
}

// (j << 32 | p) for every new edge p -> j of the batch; ~0 for empty slots.
__global__ void edge_pairs(const int32_t* __restrict__ nodes, int b, const int32_t* __restrict__ adj,
                           int adj_stride, int R, unsigned long long* __restrict__ pairs) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= b * R) return;
  const int i = t / R, j = t % R;
  const int p = nodes[i];
  const int q = adj[(size_t)p * adj_stride + j];
  pairs[t] = q >= 0 ? ((static_cast<unsigned long long>(q) << 32) | static_cast<unsigned>(p)) : ~0ull;
}

// Group starts of the sorted pairs: flags and the source ids; the empty
// (~0) keys sort last and the first of them marks the number of valid pairs
// (meta[1], preset to m).
__global__ void group_marks(const unsigned long long* __restrict__ sorted, int m,
                            int32_t* __restrict__ src, int32_t* __restrict__ is_start,
                            int32_t* __restrict__ target, int32_t* __restrict__ meta) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  const unsigned long long k = sorted[t];
  src[t] = static_cast<int32_t>(k & 0xffffffffu);
  target[t] = static_cast<int32_t>(k >> 32);
  is_start[t] = (k != ~0ull) && (t == 0 || (sorted[t - 1] >> 32) != (k >> 32));
  if (k == ~0ull && (t == 0 || sorted[t - 1] != ~0ull)) meta[1] = t;
}

__global__ void group_tasks(const int32_t* __restrict__ starts, int g, int m_valid,
                            const int32_t* __restrict__ target, int32_t* __restrict__ task_node,
                            int64_t* __restrict__ off, int32_t* __restrict__ cnt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g) return;
  const int s = starts[t];
  const int e = t + 1 < g ? starts[t + 1] : m_valid;
  task_node[t] = target[s];
  off[t] = s;
  cnt[t] = e - s;
}

__global__ void iota(int32_t* __restrict__ out, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = t;
}

__global__ void fill_pool_meta(int b, int Lb, int64_t* __restrict__ off, int32_t* __restrict__ cnt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= b) return;
  off[t] = (int64_t)t * Lb;
  cnt[t] = Lb;
}

template <class T>
cudaError_t dmalloc(T** p, size_t n) {
  return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T));
}

}  // namespace
}  // namespace ann

using namespace ann;

extern "C" int ann_build_graph_gpu_ex(const void* base, int32_t dtype, int64_t n, int32_t d, int32_t R,
                                      float alpha, int32_t L_build, uint64_t seed, int32_t engine,
                                      int32_t* adj_out, int32_t* entry_out) {
  if (!base || !adj_out) return set_error(ANN_EINVAL, "ann_build_graph_gpu: NULL buffer");
  if (dtype != ANN_U8 && dtype != ANN_F32) return set_error(ANN_EINVAL, "ann_build_graph_gpu: unknown dtype");
  if (engine < ANN_BUILD_AUTO || engine > ANN_BUILD_CUDA_CORES)
    return set_error(ANN_EINVAL, "ann_build_graph_gpu: unknown engine %d", engine);
  const bool tc_ok = dtype == ANN_U8 && d <= 128;
  if (engine == ANN_BUILD_TENSOR_CORES && !tc_ok)
    return set_error(ANN_EINVAL, "ann_build_graph_gpu: the tensor-core prune needs uint8 data with d <= 128 (d=%d)", d);
  const bool use_tc = tc_ok && engine != ANN_BUILD_CUDA_CORES;
  if (n < 2 || n >= INT32_MAX || R < 1 || R > kMaxR || L_build < R || L_build > kCandMax - R ||
      d < 16 || d % 16 || d > kMaxD || !(alpha >= 1.0f))
    return set_error(ANN_EINVAL,
                     "ann_build_graph_gpu: need 2 <= n, 1 <= R <= %d, R <= L_build <= %d - R, d %% 16 == 0 "
                     "(n=%lld d=%d R=%d L=%d)", kMaxR, kCandMax, (long long)n, d, R, L_build);
  const int elt = dtype == ANN_U8 ? 1 : 4;
  const int row_bytes = d * elt;
  const int stride = align_up(R, 4);
  // medoid on the host (float64 mean, lowest id on ties), as the host builder
  int64_t entry = 0;
  {
    const int th = std::max(1u, std::thread::hardware_concurrency());
    std::vector<double> mean(d, 0.0);
    std::vector<std::vector<double>> part(th, std::vector<double>(d, 0.0));
    std::vector<std::thread> pool;
    for (int t = 0; t < th; ++t)
      pool.emplace_back([&, t] {
        for (int64_t i = t * n / th; i < (t + 1) * n / th; ++i)
          for (int j = 0; j < d; ++j)
            part[t][j] += dtype == ANN_U8 ? static_cast<const uint8_t*>(base)[i * d + j]
                                          : static_cast<double>(static_cast<const float*>(base)[i * d + j]);
      });
    for (auto& x : pool) x.join();
    pool.clear();
    for (int t = 0; t < th; ++t)
      for (int j = 0; j < d; ++j) mean[j] += part[t][j];
    for (double& m : mean) m /= static_cast<double>(n);
    std::vector<double> bd(th, INFINITY);
    std::vector<int64_t> bi(th, -1);
    for (int t = 0; t < th; ++t)
      pool.emplace_back([&, t] {
        for (int64_t i = t * n / th; i < (t + 1) * n / th; ++i) {
          double s = 0.0;
          for (int j = 0; j < d; ++j) {
            const double v = (dtype == ANN_U8 ? static_cast<const uint8_t*>(base)[i * d + j]
                                              : static_cast<double>(static_cast<const float*>(base)[i * d + j])) - mean[j];
            s += v * v;
          }
          if (s < bd[t]) {
            bd[t] = s;
            bi[t] = i;
          }
        }
      });
    for (auto& x : pool) x.join();
    double best = INFINITY;
    for (int t = 0; t < th; ++t)
      if (bi[t] >= 0 && bd[t] < best) {
        best = bd[t];
        entry = bi[t];
      }
  }
  const int init_deg = static_cast<int>(std::min<int64_t>(R, n - 1));
  const int64_t max_batch = std::max<int64_t>(1, n / 50);
  const int mode = dtype == ANN_U8 ? kModeExactU8 : kModeExactF32;
  const int pool = std::min(L_build + 64, kCandMax - R);  // results kept per search
  SearchPlan plan;
  cudaError_t e = plan_search(mode, R, 0, d, stride * 4, 0, L_build, pool, max_batch, &plan, n);
  if (e != cudaSuccess) return cuda_error(e, "plan build search");
  const size_t nwarps = (size_t)plan.blocks * plan.warps_per_block;
  uint8_t *base_d = nullptr, *qbuf = nullptr;
  int32_t *adj_d = nullptr, *order_d = nullptr, *cand_ids = nullptr, *counters = nullptr;
  float* cand_d = nullptr;
  uint32_t *vis = nullptr, *vlog = nullptr;
  unsigned long long *exp_d = nullptr, *pairs = nullptr, *sorted = nullptr;
  int32_t *src = nullptr, *is_start = nullptr, *target = nullptr, *starts = nullptr, *nsel = nullptr;
  int32_t *task_node = nullptr, *cnt = nullptr, *idx = nullptr;
  int64_t* off = nullptr;
  void* cub_tmp = nullptr;
  size_t cub_bytes = 0, sel_bytes = 0;
  const size_t pmax = (size_t)max_batch * R;
  auto cleanup = [&]() {
    cudaFree(base_d); cudaFree(qbuf); cudaFree(adj_d); cudaFree(order_d); cudaFree(cand_ids);
    cudaFree(counters); cudaFree(cand_d); cudaFree(vis); cudaFree(vlog); cudaFree(exp_d);
    cudaFree(pairs); cudaFree(sorted); cudaFree(src); cudaFree(is_start); cudaFree(target);
    cudaFree(starts); cudaFree(nsel); cudaFree(task_node); cudaFree(cnt); cudaFree(off); cudaFree(cub_tmp);
    cudaFree(idx);
  };
#define GB_TRY(call, what)          \
  do {                              \
    e = (call);                     \
    if (e != cudaSuccess) {         \
      cleanup();                    \
      return cuda_error(e, what);   \
    }                               \
  } while (0)
  GB_TRY(dmalloc(&base_d, (size_t)n * row_bytes), "cudaMalloc vectors");
  GB_TRY(cudaMemcpy(base_d, base, (size_t)n * row_bytes, cudaMemcpyHostToDevice), "upload vectors");
  // random start graph and insertion order, on the device
  const unsigned gn = static_cast<unsigned>((n + 255) / 256);
  GB_TRY(dmalloc(&adj_d, (size_t)n * stride), "cudaMalloc adjacency");
  random_rows<<<gn, 256>>>(n, init_deg, seed, adj_d, stride);
  GB_TRY(dmalloc(&order_d, (size_t)n), "cudaMalloc order");
  {
    unsigned long long *k0 = nullptr, *k1 = nullptr;
    int32_t* i0 = nullptr;
    void* tmp = nullptr;
    size_t tmp_bytes = 0;
    e = dmalloc(&k0, (size_t)n);
    if (e == cudaSuccess) e = dmalloc(&k1, (size_t)n);
    if (e == cudaSuccess) e = dmalloc(&i0, (size_t)n);
    if (e == cudaSuccess) {
      order_keys<<<gn, 256>>>(n, seed, k0, i0);
      e = cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, k0, k1, i0, order_d, (int)n);
    }
    if (e == cudaSuccess) e = cudaMalloc(&tmp, std::max<size_t>(tmp_bytes, 1));
    if (e == cudaSuccess) e = cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, k0, k1, i0, order_d, (int)n);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(k0);
    cudaFree(k1);
    cudaFree(i0);
    cudaFree(tmp);
    if (e != cudaSuccess) {
      cleanup();
      return cuda_error(e, "start graph / insertion order");
    }
  }
  GB_TRY(dmalloc(&qbuf, (size_t)max_batch * row_bytes), "cudaMalloc batch");
  GB_TRY(dmalloc(&cand_ids, (size_t)max_batch * pool), "cudaMalloc candidates");
  GB_TRY(dmalloc(&cand_d, (size_t)max_batch * pool), "cudaMalloc candidates");
  GB_TRY(dmalloc(&vis, nwarps * plan.vis_words), "cudaMalloc visited");
  GB_TRY(cudaMemset(vis, 0, nwarps * plan.vis_words * 4), "cudaMemset");
  GB_TRY(dmalloc(&vlog, nwarps * plan.vis_log_cap), "cudaMalloc visited log");
  GB_TRY(dmalloc(&counters, 4), "cudaMalloc counters");
  GB_TRY(dmalloc(&exp_d, 1), "cudaMalloc counters");
  GB_TRY(dmalloc(&pairs, pmax), "cudaMalloc pairs");
  GB_TRY(dmalloc(&sorted, pmax), "cudaMalloc pairs");
  GB_TRY(dmalloc(&src, pmax), "cudaMalloc pairs");
  GB_TRY(dmalloc(&is_start, pmax), "cudaMalloc pairs");
  GB_TRY(dmalloc(&target, pmax), "cudaMalloc pairs");
  GB_TRY(dmalloc(&starts, pmax), "cudaMalloc pairs");
  GB_TRY(dmalloc(&nsel, 2), "cudaMalloc pairs");  // [0] groups, [1] valid pairs
  GB_TRY(dmalloc(&idx, pmax), "cudaMalloc pairs");
  iota<<<(unsigned)((pmax + 255) / 256), 256>>>(idx, (int)pmax);
  GB_TRY(dmalloc(&task_node, std::max<size_t>(pmax, (size_t)max_batch)), "cudaMalloc tasks");
  GB_TRY(dmalloc(&cnt, std::max<size_t>(pmax, (size_t)max_batch)), "cudaMalloc tasks");
  GB_TRY(dmalloc(&off, std::max<size_t>(pmax, (size_t)max_batch)), "cudaMalloc tasks");
  GB_TRY(cub::DeviceRadixSort::SortKeys(nullptr, cub_bytes, pairs, sorted, (int)pmax), "cub sizing");
  GB_TRY(cub::DeviceSelect::Flagged(nullptr, sel_bytes, idx, is_start,
                                    starts, nsel, (int)pmax), "cub sizing");
  GB_TRY(dmalloc(reinterpret_cast<uint8_t**>(&cub_tmp), std::max(cub_bytes, sel_bytes)), "cudaMalloc sort scratch");
  cudaStream_t st = 0;
  if (use_tc)
    GB_TRY(cudaFuncSetAttribute(prune_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(kTcPruneSmem)), "prune shared memory");

  SearchArgs a{};
  a.n = (int32_t)n;
  a.d = d;
  a.R = R;
  a.entry = (int32_t)entry;
  a.M = 0;
  a.vectors = base_d;
  a.adj = adj_d;
  a.adj_stride = stride;
  a.slot_bytes = stride * 4;
  a.block_bytes = stride * 4;
  a.queries = qbuf;
  a.k = pool;  // more results than list entries: every expanded node, not only the L best
  a.L = L_build;
  a.depth = 0;
  a.ids = cand_ids;
  a.dists = cand_d;
  a.vis = vis;
  a.vis_words = plan.vis_words;
  a.vis_log = vlog;
  a.vis_log_cap = plan.vis_log_cap;
  a.counters = counters;
  a.expansions = exp_d;

  const size_t max_cub = std::max(cub_bytes, sel_bytes);
  for (int pass = 0; pass < 2; ++pass) {
    const float al = pass == 0 ? 1.0f : alpha;
    int64_t done = 0, batch = 1;
    while (done < n) {
      const int b = (int)std::min(batch, n - done);
      const int32_t* nodes = order_d + done;
      gather_rows<<<b, 128, 0, st>>>(base_d, row_bytes, nodes, b, qbuf);
      GB_TRY(cudaMemsetAsync(counters, 0, 4 * sizeof(int32_t), st), "reset counter");
      SearchPlan pb = plan;
      pb.blocks = (int)std::min<int64_t>(plan.blocks, b);
      a.nq = b;
      GB_TRY(launch_search(a, pb, st), "build search");
      // forward prune: pool = the search results, plus the current row
      fill_pool_meta<<<(b + 255) / 256, 256, 0, st>>>(b, pool, off, cnt);
      if (use_tc)
        prune_tc_kernel<<<b, kTcPruneThreads, kTcPruneSmem, st>>>(base_d, d, R, al, nodes, cand_ids, off, cnt, 1, 0,
                                                                  adj_d, stride);
      else if (dtype == ANN_U8)
        prune_kernel<true><<<(b + 3) / 4, 128, 0, st>>>(base_d, d, R, al, nodes, cand_ids, off, cnt, b, 1, 0, adj_d, stride);
      else
        prune_kernel<false><<<(b + 3) / 4, 128, 0, st>>>(base_d, d, R, al, nodes, cand_ids, off, cnt, b, 1, 0, adj_d, stride);
      // back edges
      const int m = b * R;
      edge_pairs<<<(m + 255) / 256, 256, 0, st>>>(nodes, b, adj_d, stride, R, pairs);
      size_t tb = max_cub;
      GB_TRY(cub::DeviceRadixSort::SortKeys(cub_tmp, tb, pairs, sorted, m, 0, 64, st), "sort edges");
      const int32_t preset[2] = {0, m};
      GB_TRY(cudaMemcpyAsync(nsel, preset, sizeof(preset), cudaMemcpyHostToDevice, st), "group meta");
      group_marks<<<(m + 255) / 256, 256, 0, st>>>(sorted, m, src, is_start, target, nsel);
      tb = max_cub;
      GB_TRY(cub::DeviceSelect::Flagged(cub_tmp, tb, idx, is_start, starts,
                                        nsel, m, st), "group edges");
      int32_t meta[2] = {0, 0};
      GB_TRY(cudaMemcpyAsync(meta, nsel, sizeof(meta), cudaMemcpyDeviceToHost, st), "group count");
      GB_TRY(cudaStreamSynchronize(st), "build batch");
      const int32_t g = meta[0], m_valid = meta[1];
      if (g > 0) {
        group_tasks<<<(g + 255) / 256, 256, 0, st>>>(starts, g, m_valid, target, task_node, off, cnt);
        // back edges: mostly a few sources appended to a row that has room, so
        // the warp-per-node kernel (whose fixed cost per task is lower)
        // serves them with either engine
        if (dtype == ANN_U8)
          prune_kernel<true><<<(g + 3) / 4, 128, 0, st>>>(base_d, d, R, al, task_node, src, off, cnt, g, 1, 1, adj_d, stride);
        else
          prune_kernel<false><<<(g + 3) / 4, 128, 0, st>>>(base_d, d, R, al, task_node, src, off, cnt, g, 1, 1, adj_d, stride);
      }
      GB_TRY(cudaGetLastError(), "build kernels");
      done += b;
      batch = std::min<int64_t>(batch * 2, max_batch);
    }
  }
  GB_TRY(cudaStreamSynchronize(st), "build");
  GB_TRY(cudaMemcpy2D(adj_out, (size_t)R * 4, adj_d, (size_t)stride * 4, (size_t)R * 4, (size_t)n,
                      cudaMemcpyDeviceToHost), "download adjacency");
  if (entry_out) *entry_out = (int32_t)entry;
  cleanup();
#undef GB_TRY
  return ANN_OK;
}

extern "C" int ann_build_graph_gpu(const void* base, int32_t dtype, int64_t n, int32_t d, int32_t R,
                                   float alpha, int32_t L_build, uint64_t seed, int32_t* adj_out,
                                   int32_t* entry_out) {
  return ann_build_graph_gpu_ex(base, dtype, n, d, R, alpha, L_build, seed, ANN_BUILD_AUTO, adj_out, entry_out);
}
