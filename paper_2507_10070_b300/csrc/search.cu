// Persistent relaxed-pipeline graph search kernel for sm_103a.
//
// One warp runs one query at a time and takes the next query index from a
// global counter when it finishes (persistent grid sized to the SMs'
// residency).  Per query the warp:
//   a1  builds the PQ lookup table of the query in its shared memory
//       (T[m][c] = squared distance between query subvector m and centroid c,
//       an exact integer from __vabsdiffu4 + __dp4a);
//   a2  seeds the candidate list with the entry node;
//   then loops over search steps (Section "Data-Dependency in Traditional
//   Best-First Search": pop the closest candidate, read its node, compute
//   its neighbours' distances, insert them):
//   a3  select: first candidate not yet chosen for a fetch;
//   a4  fetch: copy its node block (vector + degree + neighbour ids) from the
//       storage tier (host pinned memory over PCIe, or HBM) into a ring slot
//       in shared memory with per-lane 16-byte cp.async -- one group per
//       fetch, owned by this warp alone (query-grained I/O, Section
//       "Resource-Efficient Query-Grained Concurrent I/O Stack");
//   a5  wait: only when more than `depth` fetches are in flight does the warp
//       wait, and only for its own oldest fetch (cp.async.wait_group) -- so
//       the node fetched at step i was chosen before the expansions of the
//       previous `depth` steps were merged (Section "Dependency Relaxed
//       Strategy"; depth 0 is the synchronous search);
//   a6  exact distance of the expanded node into the sorted top-k results;
//   a7  neighbour ids -> exact visited set (per-warp open-addressing table in
//       global memory, atomicCAS inserts, cleared after each query);
//   a8  PQ codes of the unseen neighbours gathered from HBM (16-byte loads)
//       and their asymmetric distances summed from the lookup table;
//   a9  warp bitonic sort of the new (distance, id) keys, merge-path merge
//       into the candidate list, truncation to L;
//   a10 stop when nothing is selectable and nothing is in flight;
//   a11 write the k results.
// The exact-navigation modes replace a1/a8 by exact distances of neighbour
// vectors gathered from HBM, and fetch the node's adjacency row instead of a
// node block; the result distance of an expanded node is its list distance.
#include <cuda_fp8.h>

#include <cstdint>

#include "ann_internal.h"

namespace ann {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned long long kNoKey = ~0ull;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async_16(void* smem_dst, const void* gmem_src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(smem_dst)),
               "l"(gmem_src)
               : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Wait until at most n of this thread's cp.async groups are pending.
__device__ __forceinline__ void cp_async_wait_pending(int n) {
  switch (n) {
    case 0: asm volatile("cp.async.wait_group 0;\n" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;\n" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;\n" ::: "memory"); break;
    case 3: asm volatile("cp.async.wait_group 3;\n" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 4;\n" ::: "memory"); break;
  }
}

__device__ __forceinline__ unsigned ld_relaxed_sys_u32(const void* p) {
  unsigned v;
  asm volatile("ld.relaxed.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed_sys_u32(void* p, unsigned v) {
  asm volatile("st.relaxed.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// 16 bytes of host-mapped memory, read afresh (not from a cached copy).
__device__ __forceinline__ uint4 ld_cv_u4(const void* p) {
  uint4 v;
  asm volatile("ld.global.cv.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p)
               : "memory");
  return v;
}

__device__ __forceinline__ long long global_timer_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned warp_sum_u32(unsigned v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Squared distance of 4 packed uint8 pairs, exact.
__device__ __forceinline__ unsigned sq4(unsigned a, unsigned b, unsigned acc) {
  unsigned t = __vabsdiffu4(a, b);
  return __dp4a(t, t, acc);
}

__device__ __forceinline__ unsigned long long make_key(unsigned dist, unsigned id) {
  return (static_cast<unsigned long long>(dist) << 32) | id;
}

// Ascending bitonic sort of 32*NB keys; element i = t*32 + lane lives in v[t].
template <int NB>
__device__ __forceinline__ void warp_bitonic_sort(unsigned long long (&v)[NB], int lane) {
  constexpr int N = 32 * NB;
#pragma unroll
  for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride >= 32) {
        const int ts = stride >> 5;
#pragma unroll
        for (int t = 0; t < NB; ++t) {
          if ((t & ts) == 0) {
            const int t2 = t | ts;
            const bool asc = (((t << 5) | lane) & size) == 0;
            unsigned long long a = v[t], b = v[t2];
            const bool swap = asc ? (a > b) : (a < b);
            v[t] = swap ? b : a;
            v[t2] = swap ? a : b;
          }
        }
      } else {
#pragma unroll
        for (int t = 0; t < NB; ++t) {
          const unsigned long long mine = v[t];
          const unsigned long long other = __shfl_xor_sync(kFull, mine, stride);
          const int i = (t << 5) | lane;
          const bool asc = (i & size) == 0;
          const bool lower = (lane & stride) == 0;
          const bool take_min = (lower == asc);
          v[t] = take_min ? (mine < other ? mine : other) : (mine < other ? other : mine);
        }
      }
    }
  }
}

// Number of entries of sorted a[0..len) that are < x.
__device__ __forceinline__ int lower_bound_u64(const unsigned long long* a, int len,
                                               unsigned long long x) {
  int lo = 0, hi = len;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// The r-th smallest (0-based) of the union of sorted, distinct a[0..na) and
// b[0..nb), r < na + nb: take i from a and r+1-i from b, the smallest i for
// which a[i] follows b[r-i].
__device__ __forceinline__ unsigned long long kth_of_two(const unsigned long long* a, int na,
                                                         const unsigned long long* b, int nb, int r) {
  int lo = r + 1 - nb > 0 ? r + 1 - nb : 0;
  int hi = r + 1 < na ? r + 1 : na;
  while (lo < hi) {
    const int i = (lo + hi) >> 1;
    if (a[i] < b[r - i]) lo = i + 1; else hi = i;
  }
  const int j = r + 1 - lo;
  const unsigned long long x = lo > 0 ? a[lo - 1] : 0ull;
  const unsigned long long y = j > 0 ? b[j - 1] : 0ull;
  return x > y ? x : y;
}

// ---- Kernel-grained I/O, the ablation of the query-grained I/O stack
// (Section "Resource-Efficient Query-Grained Concurrent I/O Stack" compares
// against CAM, where the kernel waits for every request of the batch): with
// a.grid_bar set, every resident warp meets at a grid-wide barrier after
// each fetch wait, so no query expands a node before the fetches of all
// warps in that round have arrived.  bar: [0] arrivals, [1] generation,
// [2] warps still searching, [3] 1 once every warp has stopped searching
// (written by the last arrival of a round).  Needs a cooperative launch
// (all blocks resident).  Waits are bounded: past the limit the warp sets
// counters[3] and gives up, and every other waiting warp gives up with it.
constexpr unsigned kRoundSpinLimit = 1u << 22;  // x >= 100 ns sleeps: ~0.5 s or more

__device__ __forceinline__ unsigned ld_acquire_gpu_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// One barrier round for the calling warp.  Returns false if the wait ran
// out; *all_done = every warp had stopped searching when the round closed.
__device__ bool grid_round(unsigned* bar, int* timed_out, int lane, int* all_done) {
  const unsigned total = gridDim.x * (blockDim.x >> 5);
  int ok = 1, fin = 0;
  if (lane == 0) {
    const unsigned gen = ld_acquire_gpu_u32(bar + 1);
    __threadfence();
    if (atomicAdd(bar, 1u) == total - 1) {
      // every other warp is waiting here, so the searching count is final
      fin = atomicAdd(bar + 2, 0u) == 0u;
      bar[3] = static_cast<unsigned>(fin);
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned spins = 0;
      while (ld_acquire_gpu_u32(bar + 1) == gen) {
        if (++spins > kRoundSpinLimit || ld_acquire_gpu_u32(reinterpret_cast<unsigned*>(timed_out))) {
          atomicExch(timed_out, 1);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
      if (ok) fin = static_cast<int>(ld_acquire_gpu_u32(bar + 3));
    }
  }
  *all_done = __shfl_sync(kFull, fin, 0);
  return __shfl_sync(kFull, ok, 0) != 0;
}

// Empty a query's visited bitset after the query: through the log of the
// words it set while the log held them all and that is the smaller job,
// otherwise every word.  `part` of `parts` warps takes its share.
__device__ __forceinline__ void clear_visited(uint32_t* vis, const uint32_t* vlog, int visited,
                                              int log_cap, int64_t words, int lane, int part,
                                              int parts) {
  if (visited <= log_cap && static_cast<int64_t>(visited) * 8 <= words) {
    // eight log entries per lane in flight: the log is read back from L2
    for (int j0 = part * 256; j0 < visited; j0 += 256 * parts) {
      unsigned wd[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + 32 * u + lane;
        wd[u] = j < visited ? vlog[j] : 0xffffffffu;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (wd[u] != 0xffffffffu) vis[wd[u]] = 0u;
    }
  } else {
    uint4* v4 = reinterpret_cast<uint4*>(vis);  // words is a multiple of 32
    for (int64_t j = part * 32 + lane; j < (words >> 2); j += 32 * parts) v4[j] = make_uint4(0u, 0u, 0u, 0u);
  }
}

struct QueryState {
  unsigned long long* keys;  // candidate list, ascending (nav distance, id)
  unsigned char* flags;      // 1 = chosen for a fetch already
  int* rank;                 // scratch: list rank of each new candidate
  int len;
  int nres;
};

// Insert key x into the ascending top-k result buffer res[0..nres).
__device__ __forceinline__ void result_insert(unsigned long long* res, int& nres, int k,
                                              unsigned long long x, int lane) {
  if (nres == k && x >= res[k - 1]) return;  // res is read by every lane: uniform
  int pos = 0;
  for (int b = 0; b < nres; b += 32) {
    const int j = b + lane;
    pos += __popc(__ballot_sync(kFull, j < nres && res[j] < x));
  }
  const int last = nres < k ? nres : k - 1;  // entries [pos, last) move up by one
  for (int b = ((last - 1) >> 5) << 5; b >= pos - 31 && b >= 0; b -= 32) {
    const int j = b + lane;
    unsigned long long val = 0;
    const bool mv = j >= pos && j < last;
    if (mv) val = res[j];
    __syncwarp();
    if (mv) res[j + 1] = val;
    __syncwarp();
  }
  if (lane == 0) res[pos] = x;
  __syncwarp();
  nres = nres < k ? nres + 1 : k;
}

// Merge the sorted new candidates cand[0..c) into the list in place and keep
// L entries.  rank_j = number of list entries below cand[j]; list entry i moves
// to i + #{j : rank_j <= i} and cand[j] to j + rank_j.  Entries only move
// right, so sweeping the tail in blocks from the top down never overwrites
// an entry not yet read; the candidates then fill the holes.
// Entries before rank_0 keep their place.  Returns rank_0 (the first position
// whose entry changed), or L if nothing entered.
__device__ __forceinline__ int merge_candidates(QueryState& s, const unsigned long long* cand,
                                                int c, int L, int lane,
                                                const unsigned char* cflags = nullptr) {
  if (c == 0) return L;
  if (s.len == L && cand[0] > s.keys[L - 1]) return L;  // nothing would enter
  for (int j = lane; j < c; j += 32) s.rank[j] = lower_bound_u64(s.keys, s.len, cand[j]);
  __syncwarp();
  const int pos0 = s.rank[0];
  // Sweep the tail top-down in 128-entry blocks (four entries per lane, all
  // read before any write).  p = #{j : rank_j <= top of the current block}.
  constexpr int kB = 128;
  int p = c;
  const int top_block = ((s.len - 1) / kB) * kB;
  while (p > 0 && s.rank[p - 1] > top_block + kB - 1) --p;
  for (int b = top_block; b >= (pos0 / kB) * kB; b -= kB) {
    unsigned long long key[4];
    unsigned char flag[4];
    int r[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int i = b + t * 32 + lane;
      const bool live = i >= pos0 && i < s.len;
      key[t] = live ? s.keys[i] : 0ull;
      flag[t] = live ? s.flags[i] : 0;
      r[t] = p;
    }
    // r(i) = p - #{j : i < rank_j <= b + kB - 1}: walk the ranks inside this block
    while (p > 0 && s.rank[p - 1] >= b) {
      --p;
      const int rk = s.rank[p];
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (b + t * 32 + lane < rk) --r[t];
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int i = b + t * 32 + lane;
      const int np = i + r[t];
      if (i >= pos0 && i < s.len && np < L) {
        s.keys[np] = key[t];
        s.flags[np] = flag[t];
      }
    }
    __syncwarp();
  }
  for (int j = lane; j < c; j += 32) {
    const int np = j + s.rank[j];
    if (np < L) {
      s.keys[np] = cand[j];
      s.flags[np] = cflags ? cflags[j] : 0;
    }
  }
  __syncwarp();
  s.len = (s.len + c < L) ? s.len + c : L;
  return pos0;
}

// Exact squared distance between the query (in shared memory) and base vector w.
template <int MODE>
__device__ __forceinline__ unsigned exact_dist_warp(const SearchArgs& a, const unsigned char* qs,
                                                    int w, int lane) {
  if (MODE == kModeExactF32) {
    const float4* x = reinterpret_cast<const float4*>(static_cast<const float*>(a.vectors) +
                                                      static_cast<size_t>(w) * a.d);
    const float4* q = reinterpret_cast<const float4*>(qs);
    float acc = 0.f;
    for (int j = lane; j < (a.d >> 2); j += 32) {
      const float4 xv = __ldg(x + j), qv = q[j];
      float t;
      t = qv.x - xv.x; acc = fmaf(t, t, acc);
      t = qv.y - xv.y; acc = fmaf(t, t, acc);
      t = qv.z - xv.z; acc = fmaf(t, t, acc);
      t = qv.w - xv.w; acc = fmaf(t, t, acc);
    }
    return __float_as_uint(warp_sum_f32(acc));
  } else {
    const unsigned* x = reinterpret_cast<const unsigned*>(static_cast<const uint8_t*>(a.vectors) +
                                                          static_cast<size_t>(w) * a.d);
    const unsigned* q = reinterpret_cast<const unsigned*>(qs);
    unsigned acc = 0;
    for (int j = lane; j < (a.d >> 2); j += 32) acc = sq4(q[j], __ldg(x + j), acc);
    return warp_sum_u32(acc);
  }
}

// One query's parameters and output locations.
struct QueryJob {
  const void* query;   // query vector; NULL if the caller already put it in shared memory
  int k, L;
  int qi;              // query number, for failure reporting
  int32_t* ids;        // [k]
  float* dists;        // [k]
  int32_t* steps;      // single values, each may be NULL
  int32_t* status;
  int64_t* t_begin;
  int64_t* t_end;
};

// Navigation distance from a compressed copy (BF16 or FP8-E4M3 x scale) of
// base vector w, FP32 accumulation.  BF16 -> float is the 16-bit shift;
// FP8 -> float uses CUDA's own conversion.
template <int MODE>
__device__ __forceinline__ unsigned nav_dist_warp(const SearchArgs& a, const unsigned char* qs,
                                                  int w, int lane) {
  const float4* q = reinterpret_cast<const float4*>(qs);
  float acc = 0.f;
  if (MODE == kModeBF16) {
    const uint2* x = reinterpret_cast<const uint2*>(static_cast<const uint16_t*>(a.nav) +
                                                    static_cast<size_t>(w) * a.d);
    for (int j = lane; j < (a.d >> 2); j += 32) {
      const uint2 v = __ldg(x + j);
      const float4 qv = q[j];
      float t;
      t = qv.x - __uint_as_float(v.x << 16); acc = fmaf(t, t, acc);
      t = qv.y - __uint_as_float(v.x & 0xffff0000u); acc = fmaf(t, t, acc);
      t = qv.z - __uint_as_float(v.y << 16); acc = fmaf(t, t, acc);
      t = qv.w - __uint_as_float(v.y & 0xffff0000u); acc = fmaf(t, t, acc);
    }
  } else {
    const unsigned* x = reinterpret_cast<const unsigned*>(static_cast<const uint8_t*>(a.nav) +
                                                          static_cast<size_t>(w) * a.d);
    const float s = a.nav_inv_scale;
    for (int j = lane; j < (a.d >> 2); j += 32) {
      __nv_fp8x4_e4m3 f;
      f.__x = __ldg(x + j);
      const float4 xv = static_cast<float4>(f);
      const float4 qv = q[j];
      float t;
      t = qv.x - xv.x * s; acc = fmaf(t, t, acc);
      t = qv.y - xv.y * s; acc = fmaf(t, t, acc);
      t = qv.z - xv.z * s; acc = fmaf(t, t, acc);
      t = qv.w - xv.w * s; acc = fmaf(t, t, acc);
    }
  }
  return __float_as_uint(warp_sum_f32(acc));
}

// Partial navigation distance for the grouped evaluation: this lane sums
// chunks sub, sub + lpg, ... of node w's vector (a chunk is 4 coordinates);
// the group then adds its lanes' partial sums.  Same arithmetic per chunk as
// the warp-wide functions above.
template <int MODE>
__device__ __forceinline__ float nav_partial_f32(const SearchArgs& a, const unsigned char* qs, int w,
                                                 int sub, int lpg) {
  const float4* q = reinterpret_cast<const float4*>(qs);
  const int chunks = a.d >> 2;
  float acc = 0.f;
  if (MODE == kModeExactF32) {
    const float4* x = reinterpret_cast<const float4*>(static_cast<const float*>(a.vectors) +
                                                      static_cast<size_t>(w) * a.d);
    for (int j = sub; j < chunks; j += lpg) {
      const float4 xv = __ldg(x + j), qv = q[j];
      float t;
      t = qv.x - xv.x; acc = fmaf(t, t, acc);
      t = qv.y - xv.y; acc = fmaf(t, t, acc);
      t = qv.z - xv.z; acc = fmaf(t, t, acc);
      t = qv.w - xv.w; acc = fmaf(t, t, acc);
    }
  } else if (MODE == kModeBF16) {
    const uint2* x = reinterpret_cast<const uint2*>(static_cast<const uint16_t*>(a.nav) +
                                                    static_cast<size_t>(w) * a.d);
    for (int j = sub; j < chunks; j += lpg) {
      const uint2 v = __ldg(x + j);
      const float4 qv = q[j];
      float t;
      t = qv.x - __uint_as_float(v.x << 16); acc = fmaf(t, t, acc);
      t = qv.y - __uint_as_float(v.x & 0xffff0000u); acc = fmaf(t, t, acc);
      t = qv.z - __uint_as_float(v.y << 16); acc = fmaf(t, t, acc);
      t = qv.w - __uint_as_float(v.y & 0xffff0000u); acc = fmaf(t, t, acc);
    }
  } else if (MODE == kModeFP8) {
    const unsigned* x = reinterpret_cast<const unsigned*>(static_cast<const uint8_t*>(a.nav) +
                                                          static_cast<size_t>(w) * a.d);
    const float s = a.nav_inv_scale;
    for (int j = sub; j < chunks; j += lpg) {
      __nv_fp8x4_e4m3 f;
      f.__x = __ldg(x + j);
      const float4 xv = static_cast<float4>(f);
      const float4 qv = q[j];
      float t;
      t = qv.x - xv.x * s; acc = fmaf(t, t, acc);
      t = qv.y - xv.y * s; acc = fmaf(t, t, acc);
      t = qv.z - xv.z * s; acc = fmaf(t, t, acc);
      t = qv.w - xv.w * s; acc = fmaf(t, t, acc);
    }
  }
  return acc;
}

__device__ __forceinline__ unsigned nav_partial_u8(const SearchArgs& a, const unsigned char* qs, int w,
                                                   int sub, int lpg) {
  const unsigned* x = reinterpret_cast<const unsigned*>(static_cast<const uint8_t*>(a.vectors) +
                                                        static_cast<size_t>(w) * a.d);
  const unsigned* q = reinterpret_cast<const unsigned*>(qs);
  unsigned acc = 0;
  for (int j = sub; j < (a.d >> 2); j += lpg) acc = sq4(q[j], __ldg(x + j), acc);
  return acc;
}

// Navigation distance of node w for the non-PQ modes.
template <int MODE>
__device__ __forceinline__ unsigned navigation_dist(const SearchArgs& a, const unsigned char* qs,
                                                    int w, int lane) {
  if (MODE == kModeBF16 || MODE == kModeFP8) return nav_dist_warp<MODE>(a, qs, w, lane);
  return exact_dist_warp<MODE>(a, qs, w, lane);
}

// CPU-agent I/O: post the request of entry e (lane 0).  The node goes first,
// the new sequence number last, with a system-scope fence between them, so
// a host thread that sees the number also sees the node.
__device__ __forceinline__ void agent_post(const SearchArgs& a, size_t e, unsigned node) {
  const unsigned sq = a.agent_seq[e] + 1u;
  a.agent_seq[e] = sq;
  st_relaxed_sys_u32(&a.agent_req[e].node, node);
  __threadfence_system();
  st_relaxed_sys_u32(&a.agent_req[e].seq, sq);
}

// Wait (lane 0) until the host has served entry e's latest request, at most
// a.agent_wait_ns; false if the wait ran out.  The completion word is read
// over PCIe, so the polls back off.
__device__ bool agent_wait(const SearchArgs& a, size_t e) {
  const unsigned want = a.agent_seq[e];
  const long long t0 = global_timer_ns();
  unsigned ns = 32;
  for (;;) {
    if (ld_relaxed_sys_u32(a.agent_done + e) == want) {
      __threadfence_system();  // the staging slot's bytes are read after this
      return true;
    }
    if (global_timer_ns() - t0 > a.agent_wait_ns) return false;
    __nanosleep(ns);
    if (ns < 1024) ns <<= 1;
  }
}

template <int MODE, int NB, bool PF = false>
__device__ void run_query(const SearchArgs& a, const QueryJob& job, unsigned char* ws,
                          const WarpSmem& lay, uint32_t* vis, uint32_t* vlog, int lane) {
  const long long t0 = global_timer_ns();
  const int d = a.d, L = job.L, k = job.k, D = a.depth, n = a.n;
  const int log_cap = a.vis_log_cap;

  unsigned* lut = reinterpret_cast<unsigned*>(ws + lay.lut);
  unsigned char* ring = ws + lay.ring;
  unsigned char* qs = ws + lay.q;
  unsigned long long* res = reinterpret_cast<unsigned long long*>(ws + lay.res);
  unsigned long long* cand = reinterpret_cast<unsigned long long*>(ws + lay.cand);
  unsigned long long* ring_key = reinterpret_cast<unsigned long long*>(ws + lay.ring_key);
  const int slot_bytes = a.slot_bytes;

  QueryState s;
  s.keys = reinterpret_cast<unsigned long long*>(ws + lay.keys);
  s.flags = ws + lay.flags;
  s.rank = reinterpret_cast<int*>(ws + lay.rank);
  // Pending buffer: each step's entering candidates are merged into this
  // short sorted buffer, and the buffer into the list only when it is full,
  // so the list's tail moves once per many steps instead of every step.  The
  // candidate list of the search is the first L entries of the union of the
  // two: selection takes the first unselected entry of the union if its rank
  // in the union is below L, and the bound for entering is the union's L-th
  // key.  An entry pushed past rank L never returns (the union only grows
  // until a merge drops such entries), so this is the same list.  Used from
  // L = kLazyL on: below it the tail is short, and merging straight into the
  // list costs less than the union's bookkeeping.
  const bool lazy = L >= kLazyL;
  QueryState pend;
  pend.keys = reinterpret_cast<unsigned long long*>(ws + lay.pkeys);
  pend.flags = ws + lay.pflags;
  pend.rank = s.rank;
  pend.len = 0;
  int pfirst_open = 0;  // every pending entry before this position is selected

  // ---- query vector into shared memory
  if (job.query) {
    const int qbytes = mode_f32(MODE) ? d * 4 : d;
    const unsigned* src = static_cast<const unsigned*>(job.query);
    unsigned* dst = reinterpret_cast<unsigned*>(qs);
    for (int j = lane; j < (qbytes >> 2); j += 32) dst[j] = __ldg(src + j);
  }
  __syncwarp();

  // ---- a1: lookup table T[m][c], exact integers.  The codebook comes from
  // L2 (shared memory leaves little L1), so each lane keeps two subspaces'
  // eight centroids (16 loads) in flight instead of paying the latency once
  // per entry; M is a multiple of 16.
  if (MODE == kModePqU8) {
    const int wps = a.dsub >> 2;  // 32-bit words per subvector
    const unsigned* qw = reinterpret_cast<const unsigned*>(qs);
    for (int m = 0; m < a.M; m += 2) {
      unsigned acc[2][8];
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[h][j] = 0u;
      for (int w = 0; w < wps; ++w) {
        unsigned cv[2][8];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int j = 0; j < 8; ++j)
            cv[h][j] = __ldg(a.cb_words + (static_cast<size_t>(m + h) * 256 + lane + 32 * j) * wps + w);
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[h][j] = sq4(qw[(m + h) * wps + w], cv[h][j], acc[h][j]);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 8; ++j) lut[(m + h) * 256 + lane + 32 * j] = acc[h][j];
    }
    __syncwarp();
  }
  // float PQ: T[m][c] in FP32 (float codebook)
  float* lutf = reinterpret_cast<float*>(ws + lay.lut);
  if (MODE == kModePqF32) {
    const float* qf = reinterpret_cast<const float*>(qs);
    const int dsub = a.dsub;
    for (int m = 0; m < a.M; ++m) {
      // eight centroids per lane in flight; each sums its coordinates in order
      float acc[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] = 0.f;
      for (int j = 0; j < dsub; ++j) {
        float cv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          cv[u] = __ldg(a.cb_f32 + (static_cast<size_t>(m) * 256 + lane + 32 * u) * dsub + j);
        const float qv = qf[m * dsub + j];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float t = qv - cv[u];
          acc[u] = fmaf(t, t, acc[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) lutf[m * 256 + lane + 32 * u] = acc[u];
    }
    __syncwarp();
  }

  // ---- a2: entry node
  unsigned entry_dist;
  if (MODE == kModePqU8) {
    const uint8_t* code = a.codes + static_cast<size_t>(a.entry) * a.M;
    unsigned part = 0;
    for (int m = lane; m < a.M; m += 32) part += lut[m * 256 + code[m]];
    entry_dist = warp_sum_u32(part);
  } else if (MODE == kModePqF32) {
    // same summation order as the neighbours' lookups (m ascending)
    float acc = 0.f;
    const uint8_t* code = a.codes + static_cast<size_t>(a.entry) * a.M;
    for (int m = 0; m < a.M; ++m) acc += lutf[m * 256 + code[m]];
    entry_dist = __float_as_uint(acc);
  } else {
    entry_dist = navigation_dist<MODE>(a, qs, a.entry, lane);
  }
  if (lane == 0) {
    s.keys[0] = make_key(entry_dist, a.entry);
    s.flags[0] = 0;
    atomicOr(vis + (static_cast<unsigned>(a.entry) >> 5), 1u << (a.entry & 31));
    vlog[0] = static_cast<unsigned>(a.entry) >> 5;
  }
  for (int j = lane; j < k; j += 32) res[j] = kNoKey;
  __syncwarp();
  s.len = 1;
  s.nres = 0;
  int head = 0, inflight = 0, steps = 0, visited = 1, status = ANN_OK;
  int first_open = 0;  // every list entry before this position is selected
  const int max_steps = n + 1;  // each node is expanded at most once
  // Next-node prefetch (PQ navigation, depth >= 2): once a step has the
  // asymmetric distances of its node, the next node in the fetch FIFO --
  // issued at least one step earlier, so its block has landed -- gets its
  // code gathers and visited-bit atomics issued, and their round trip to
  // L2/HBM overlaps this step's sort and merge.  The visited set sees the
  // same inserts in the same order (the next node's atomics follow this
  // node's, which have returned), and the list merge of its candidates still
  // happens in its own step, so the search is unchanged.  A separate
  // instance (PF), so that depths 0 and 1 keep the leaner kernel.
  const bool prefetch = PF && MODE == kModePqU8 && D >= 2 && !a.grid_bar && !a.agent_req;
  // CPU-agent I/O: this warp's D + 1 request entries
  const size_t agent_base =
      (static_cast<size_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5)) * static_cast<size_t>(D + 1);
  bool pre = false;  // the node at the FIFO head has its loads in flight
  int pw[NB];
  unsigned pword[NB], pold[NB];
  uint4 pcode[NB][kMaxM / 16];
  const int deg = a.R;
  // read the ids of the block at `blk`, issue their code gathers and
  // visited-bit atomics
  auto issue_neighbours = [&](const unsigned char* blk, int (&w)[NB], unsigned (&word)[NB],
                              uint4 (&code)[NB][kMaxM / 16], unsigned (&old)[NB]) {
    // Neighbour ids are -1 padded, so the degree word need not be fetched.
    const int32_t* nbr = reinterpret_cast<const int32_t*>(blk + (MODE == kModePqU8 ? a.ids_off : 0));
#pragma unroll
    for (int t = 0; t < NB; ++t) {
      const int j = t * 32 + lane;
      int id = j < deg ? nbr[j] : -1;
      if (id >= n) id = -1;  // validated at load; never trusted blindly
      w[t] = id;
      word[t] = id >= 0 ? static_cast<unsigned>(id) >> 5 : 0u;
    }
    // PQ codes of every listed neighbour, issued before the visited atomics
    // so that both round trips overlap.
    if (mode_pq(MODE)) {
#pragma unroll
      for (int t = 0; t < NB; ++t) {
        if (w[t] >= 0) {
          const uint4* cp = reinterpret_cast<const uint4*>(a.codes + static_cast<size_t>(w[t]) * a.M);
#pragma unroll
          for (int c = 0; c < kMaxM / 16; ++c)
            if (c < (a.M >> 4)) code[t][c] = __ldg(cp + c);
        }
      }
    }
    // Visited set: one atomicOr per neighbour on its bit; the neighbour is
    // new if its bit was clear (a repeated id in the row finds it set).
#pragma unroll
    for (int t = 0; t < NB; ++t)
      old[t] = w[t] >= 0 ? atomicOr(vis + word[t], 1u << (w[t] & 31)) : 0u;
  };

  for (;;) {
    // ---- a3: select the first candidate not chosen yet: the first
    // unselected entry of the list or of the pending buffer, whichever is
    // smaller, if its rank in their union is below L
    int ia = -1, ib = -1;
    for (int b = first_open; b < s.len; b += 32) {
      const int i = b + lane;
      const unsigned m = __ballot_sync(kFull, i < s.len && s.flags[i] == 0);
      if (m) {
        ia = b + __ffs(m) - 1;
        break;
      }
    }
    for (int b = pfirst_open; b < pend.len; b += 32) {
      const int i = b + lane;
      const unsigned m = __ballot_sync(kFull, i < pend.len && pend.flags[i] == 0);
      if (m) {
        ib = b + __ffs(m) - 1;
        break;
      }
    }
    first_open = ia >= 0 ? ia : s.len;
    pfirst_open = ib >= 0 ? ib : pend.len;
    int sel = -1;  // 0: list entry ia, 1: pending entry ib
    unsigned long long key = 0;
    if (ia >= 0 && (ib < 0 || s.keys[ia] < pend.keys[ib])) {
      key = s.keys[ia];
      if (pend.len == 0 || ia + lower_bound_u64(pend.keys, pend.len, key) < L) sel = 0;
    } else if (ib >= 0) {
      key = pend.keys[ib];
      if (ib + lower_bound_u64(s.keys, s.len, key) < L) sel = 1;
    }
    if (sel == 0) first_open = ia + 1;
    if (sel == 1) pfirst_open = ib + 1;
    if (sel >= 0) {
      // ---- a4: issue the fetch of its block into the next ring slot
      const unsigned v = static_cast<unsigned>(key);
      int slot = head + inflight;
      if (slot > D) slot -= D + 1;
      __syncwarp();
      if (lane == 0) {
        if (sel == 0) s.flags[ia] = 1; else pend.flags[ib] = 1;
        ring_key[slot] = key;
      }
      if (MODE == kModePqU8 && a.agent_req) {
        // the host agent copies the block into this entry's staging slot
        if (lane == 0) agent_post(a, agent_base + slot, v);
      } else {
        const uint8_t* src = (MODE == kModePqU8)
                                 ? a.blocks + static_cast<size_t>(v) * a.block_bytes
                                 : reinterpret_cast<const uint8_t*>(
                                       a.adj + static_cast<size_t>(v) * a.adj_stride);
        unsigned char* dst = ring + slot * slot_bytes;
        for (int off = lane * 16; off < slot_bytes; off += 512) cp_async_16(dst + off, src + off);
        cp_async_commit();
      }
      ++inflight;
      __syncwarp();  // lane 0's flag and ring_key writes are seen by every lane
    }
    if (inflight > D || (sel < 0 && inflight > 0)) {
      // ---- a5: wait for this warp's oldest fetch only
      if (MODE == kModePqU8 && a.agent_req) {
        int ok = 1;
        if (lane == 0) ok = agent_wait(a, agent_base + head) ? 1 : 0;
        if (!__shfl_sync(kFull, ok, 0)) {
          status = ANN_ETIMEOUT;
          break;
        }
        const uint8_t* stg = a.agent_stage + (agent_base + head) * static_cast<size_t>(slot_bytes);
        unsigned char* dst = ring + head * slot_bytes;
        for (int off = lane * 16; off < slot_bytes; off += 512)
          *reinterpret_cast<uint4*>(dst + off) = ld_cv_u4(stg + off);
      } else {
        cp_async_wait_pending(inflight - 1);
      }
      __syncwarp();
      if (a.grid_bar) {  // kernel-grained ablation: the round's fetches all land first
        int all_done;
        if (!grid_round(a.grid_bar, a.counters + 3, lane, &all_done)) {
          status = ANN_ETIMEOUT;
          break;
        }
      }
      const unsigned char* blk = ring + head * slot_bytes;
      const unsigned long long ukey = ring_key[head];
      const unsigned u = static_cast<unsigned>(ukey);
      head = (head == D) ? 0 : head + 1;
      --inflight;
      ++steps;

      // ---- a6: exact distance of u into the results (the other modes keep
      // their navigation distance here; a rerank pass follows where needed)
      unsigned long long rkey;
      if (MODE == kModePqU8) {
        const unsigned* xw = reinterpret_cast<const unsigned*>(blk);
        const unsigned* qw = reinterpret_cast<const unsigned*>(qs);
        unsigned acc = 0;
        for (int j = lane; j < (d >> 2); j += 32) acc = sq4(qw[j], xw[j], acc);
        rkey = make_key(warp_sum_u32(acc), u);
      } else {
        rkey = ukey;  // exact navigation: the list distance is the exact distance
      }
      result_insert(res, s.nres, k, rkey, lane);

      // ---- a7: neighbour ids and the visited set (issued one step early
      // when the node was prefetched)
      int w[NB];
      unsigned word[NB];
      bool fresh[NB];
      uint4 code[NB][kMaxM / 16];
      unsigned old[NB];
      if (pre) {
#pragma unroll
        for (int t = 0; t < NB; ++t) {
          w[t] = pw[t];
          word[t] = pword[t];
          old[t] = pold[t];
#pragma unroll
          for (int c = 0; c < kMaxM / 16; ++c) code[t][c] = pcode[t][c];
        }
        pre = false;
      } else {
        issue_neighbours(blk, w, word, code, old);
      }
#pragma unroll
      for (int t = 0; t < NB; ++t) fresh[t] = w[t] >= 0 && ((old[t] >> (w[t] & 31)) & 1u) == 0u;

      // ---- a8: navigation distances of the new neighbours
      unsigned long long key[NB];
      if (MODE == kModePqF32) {
#pragma unroll
        for (int t = 0; t < NB; ++t) {
          key[t] = kNoKey;
          if (fresh[t]) {
            float dist = 0.f;
#pragma unroll
            for (int c = 0; c < kMaxM / 16; ++c) {
              if (c < (a.M >> 4)) {
                const unsigned wd[4] = {code[t][c].x, code[t][c].y, code[t][c].z, code[t][c].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                  const int m0 = c * 16 + e * 4;
                  dist += lutf[(m0 + 0) * 256 + (wd[e] & 0xff)];
                  dist += lutf[(m0 + 1) * 256 + ((wd[e] >> 8) & 0xff)];
                  dist += lutf[(m0 + 2) * 256 + ((wd[e] >> 16) & 0xff)];
                  dist += lutf[(m0 + 3) * 256 + (wd[e] >> 24)];
                }
              }
            }
            key[t] = make_key(__float_as_uint(dist), static_cast<unsigned>(w[t]));
          }
        }
      } else if (MODE == kModePqU8) {
#pragma unroll
        for (int t = 0; t < NB; ++t) {
          key[t] = kNoKey;
          if (fresh[t]) {
            unsigned dist = 0;
#pragma unroll
            for (int c = 0; c < kMaxM / 16; ++c) {
              if (c < (a.M >> 4)) {
                const unsigned wd[4] = {code[t][c].x, code[t][c].y, code[t][c].z, code[t][c].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                  const int m0 = c * 16 + e * 4;
                  dist += lut[(m0 + 0) * 256 + (wd[e] & 0xff)];
                  dist += lut[(m0 + 1) * 256 + ((wd[e] >> 8) & 0xff)];
                  dist += lut[(m0 + 2) * 256 + ((wd[e] >> 16) & 0xff)];
                  dist += lut[(m0 + 3) * 256 + (wd[e] >> 24)];
                }
              }
            }
            key[t] = make_key(dist, static_cast<unsigned>(w[t]));
          }
        }
      } else {
        // Vector modes: the warp splits into groups of lpg lanes (a power of
        // two with at most 8 chunks per lane), each group summing one
        // neighbour, so 32/lpg neighbours' gathers are in flight at once
        // instead of one.  Per node the summation order is fixed by lpg.
        const int chunks = a.d >> 2;
        int lpg = 1;
        while (lpg < 32 && lpg * 8 < chunks) lpg <<= 1;
        const int groups = 32 / lpg;
        const int grp = lane / lpg, sub = lane % lpg;
        const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
        for (int t = 0; t < NB; ++t) {
          key[t] = kNoKey;
          unsigned m = __ballot_sync(kFull, fresh[t]);
          while (m) {
            // group g evaluates the neighbour held by the g-th set lane of m
            unsigned mm = m;
            for (int i = 0; i < grp && mm; ++i) mm &= mm - 1;
            const int src = mm ? __ffs(mm) - 1 : -1;
            const int id = __shfl_sync(kFull, w[t], src < 0 ? 0 : src);
            unsigned bits;
            if (MODE == kModeExactU8) {
              unsigned acc = src >= 0 ? nav_partial_u8(a, qs, id, sub, lpg) : 0u;
              for (int off = lpg >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
              bits = acc;
            } else {
              float acc = src >= 0 ? nav_partial_f32<MODE>(a, qs, id, sub, lpg) : 0.f;
              for (int off = lpg >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
              bits = __float_as_uint(acc);
            }
            // the neighbour's own lane takes its group's sum
            const int r = __popc(m & lt_mask);
            const unsigned got = __shfl_sync(kFull, bits, (r < groups ? r : 0) * lpg);
            if (((m >> lane) & 1u) && r < groups) key[t] = make_key(got, static_cast<unsigned>(w[t]));
            for (int i = 0; i < groups && m; ++i) m &= m - 1;
          }
        }
      }

      // the next node's loads, overlapping the sort and merge below
      if (prefetch && inflight >= 2) {
        cp_async_wait_pending(inflight - 1);  // the next node's block (issued a step ago or more)
        __syncwarp();
        issue_neighbours(ring + head * slot_bytes, pw, pword, pcode, pold);
        pre = true;
      }

      // A key at or above the L-th entry of a full list cannot enter it (the
      // list is the first L entries of list and pending buffer together).
      const unsigned long long thr =
          pend.len == 0 ? (s.len == L ? s.keys[L - 1] : kNoKey)
                        : (s.len + pend.len >= L ? kth_of_two(s.keys, s.len, pend.keys, pend.len, L - 1) : kNoKey);
#pragma unroll
      for (int t = 0; t < NB; ++t)
        if (!fresh[t]) key[t] = kNoKey;

      // log the words of the new nodes' bits (while the log has room), so
      // the clear after the query touches only those
      int nfresh = 0;
      const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
      for (int t = 0; t < NB; ++t) {
        const unsigned m = __ballot_sync(kFull, fresh[t]);
        const int at = visited + nfresh + __popc(m & lt_mask);
        if (fresh[t] && at < log_cap) vlog[at] = word[t];
        nfresh += __popc(m);
      }
      visited += nfresh;

      // ---- a9: sort the new keys that can enter (below the L-th entry of a
      // full list), merge them into the list, truncate to L
      if (nfresh > 0) {
        int c = 0;
        unsigned keep_mask[NB];
#pragma unroll
        for (int t = 0; t < NB; ++t) {
          keep_mask[t] = __ballot_sync(kFull, key[t] < thr);
          c += __popc(keep_mask[t]);
        }
        if (c > 0 && c <= 32) {
          // compact the entering keys into one register per lane, sort 32
          int base = 0;
#pragma unroll
          for (int t = 0; t < NB; ++t) {
            if ((keep_mask[t] >> lane) & 1u) cand[base + __popc(keep_mask[t] & lt_mask)] = key[t];
            base += __popc(keep_mask[t]);
          }
          __syncwarp();
          unsigned long long one[1] = {lane < c ? cand[lane] : kNoKey};
          __syncwarp();
          warp_bitonic_sort<1>(one, lane);
          cand[lane] = one[0];
          __syncwarp();
        } else if (c > 32) {
#pragma unroll
          for (int t = 0; t < NB; ++t) key[t] = key[t] < thr ? key[t] : kNoKey;
          warp_bitonic_sort<NB>(key, lane);
#pragma unroll
          for (int t = 0; t < NB; ++t) cand[t * 32 + lane] = key[t];
          __syncwarp();
        }
        if (c > 0 && !lazy) {
          const int changed = merge_candidates(s, cand, c, L, lane);
          if (changed < first_open) first_open = changed;
        } else if (c > 0) {
          if (pend.len + c > kPend) {
            // the pending buffer is full: merge it, selected flags and all,
            // into the list (entries past rank L fall off), then empty it
            const int changed = merge_candidates(s, pend.keys, pend.len, L, lane, pend.flags);
            if (changed < first_open) first_open = changed;
            pend.len = 0;
            pfirst_open = 0;
            __syncwarp();
          }
          const int pchanged = merge_candidates(pend, cand, c, kPend, lane);
          if (pchanged < pfirst_open) pfirst_open = pchanged;
        }
      }
      __syncwarp();

      if (steps >= max_steps) {  // cannot happen: each node is expanded at most once
        status = ANN_ENOMEM;
        break;
      }
    } else if (sel < 0) {
      break;  // ---- a10: nothing selectable, nothing in flight
    }
  }
  // Drain fetches still in flight after an early stop (none on normal exit).
  cp_async_wait_pending(0);
  __syncwarp();

  // ---- a11: results
  for (int j = lane; j < k; j += 32) {
    const unsigned long long r = j < s.nres ? res[j] : kNoKey;
    const bool ok = r != kNoKey;
    const int32_t id = static_cast<int32_t>(r & 0xffffffffu);
    job.ids[j] = ok ? (a.id_map ? __ldg(a.id_map + id) : id) : -1;
    const unsigned dbits = static_cast<unsigned>(r >> 32);
    job.dists[j] = ok ? (mode_f32(MODE) ? __uint_as_float(dbits) : static_cast<float>(dbits))
                      : __int_as_float(0x7f800000);
  }
  // Clear the bits this query set, so the set is empty for the next query
  // of this warp.  (After an early stop a prefetched node's bits are not in
  // the log: clear every word then.)
  __syncwarp();
  clear_visited(vis, vlog, pre ? log_cap + 1 : visited, log_cap, a.vis_words, lane, 0, 1);
  if (lane == 0) {
    if (job.steps) *job.steps = steps;
    if (job.status) *job.status = status;
    if (job.t_begin) *job.t_begin = t0;
    if (job.t_end) *job.t_end = global_timer_ns();
    atomicAdd(a.expansions, static_cast<unsigned long long>(steps));
    if (status != ANN_OK) {
      atomicAdd(&a.counters[1], 1);
      atomicMin(&a.counters[2], job.qi);
    }
  }
  __syncwarp();
}

template <int MODE, int NB, bool PF = false>
__global__ void search_kernel(SearchArgs a, int smem_per_warp) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int warps = blockDim.x >> 5;
  unsigned char* ws = smem + wib * smem_per_warp;
  const WarpSmem lay = warp_smem_layout(MODE, a.M, a.d, a.slot_bytes, a.depth, a.L, a.k, NB);
  const size_t gw = static_cast<size_t>(blockIdx.x) * warps + wib;
  uint32_t* vis = a.vis + gw * static_cast<size_t>(a.vis_words);
  uint32_t* vlog = a.vis_log + gw * static_cast<size_t>(a.vis_log_cap);
  for (;;) {
    if (a.grid_bar && ld_acquire_gpu_u32(reinterpret_cast<const unsigned*>(a.counters + 3))) break;
    int qi = 0;
    if (lane == 0) qi = atomicAdd(&a.counters[0], 1);
    qi = __shfl_sync(kFull, qi, 0);
    if (qi >= a.nq) break;
    QueryJob job;
    const int qbytes = mode_f32(MODE) ? a.d * 4 : a.d;
    job.query = static_cast<const uint8_t*>(a.queries) + static_cast<size_t>(qi) * qbytes;
    job.k = a.k;
    job.L = a.L;
    job.qi = qi;
    job.ids = a.ids + static_cast<size_t>(qi) * a.k;
    job.dists = a.dists + static_cast<size_t>(qi) * a.k;
    job.steps = a.steps ? a.steps + qi : nullptr;
    job.status = a.status ? a.status + qi : nullptr;
    job.t_begin = a.t_begin ? a.t_begin + qi : nullptr;
    job.t_end = a.t_end ? a.t_end + qi : nullptr;
    run_query<MODE, NB, PF>(a, job, ws, lay, vis, vlog, lane);
  }
  if (a.grid_bar) {
    // kernel-grained ablation: stop searching, but keep meeting the other
    // warps' rounds until every warp has stopped
    if (lane == 0) {
      __threadfence();
      atomicSub(a.grid_bar + 2, 1u);
    }
    __syncwarp();
    for (;;) {
      int all_done = 0;
      if (!grid_round(a.grid_bar, a.counters + 3, lane, &all_done) || all_done) break;
    }
  }
}

// ---- Warp group per query (PQ navigation, uint8 data).
//
// W warps -- one block -- share one query's state in shared memory: its
// lookup table (built W subspace pairs at a time), candidate list, results
// and fetch ring, and one visited table.  Warp 0 keeps the pipeline exactly
// as the warp-per-query kernel does (selection, fetch issue, the wait for its
// own oldest fetch), so the schedule of fetches and expansions is the same.
// Per expansion the other warps join in: each warp takes R/W of the node's
// neighbour positions (visited set, code gathers, asymmetric distances), and
// the merge of the step's new candidates into the list is split across the
// warps.  Lists, steps and results therefore equal the warp-per-query
// kernel's for every W; what changes is the time one step takes.
struct WgCtl {
  unsigned long long ukey;  // node expanded this step (its list key)
  int act;                  // 1 = expand, 2 = stop
  int slot;                 // ring slot holding its block
  int len;                  // list length before this step's merge
  int plen;                 // pending-buffer length before this step's merge
  int pf_slot;              // ring slot of the next node whose loads go out early, or -1
  int vis_count;            // visited-log entries of the query so far
  int cand_count;           // candidates entering the list this step
  int qi;                   // query the block works on
};
constexpr int kWgCtlBytes = 128;  // control words after the query's shared memory
static_assert(sizeof(WgCtl) <= kWgCtlBytes, "control words");

// Number of entries of sorted a[0..len) that are <= x.
__device__ __forceinline__ int upper_bound_i32(const int* a, int len, int x) {
  int lo = 0, hi = len;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

template <int NB, int W>
__device__ void run_query_wg(const SearchArgs& a, const QueryJob& job, unsigned char* ws,
                             const WarpSmem& lay, uint32_t* vis, uint32_t* vlog, int warp,
                             int lane, WgCtl* ctl) {
  constexpr int kChunk = 32 * NB / W;                  // neighbour positions per warp
  constexpr int NBW = kChunk >= 32 ? kChunk / 32 : 1;  // of them per lane
  const long long t0 = global_timer_ns();
  const int d = a.d, L = job.L, k = job.k, D = a.depth, n = a.n;
  const int log_cap = a.vis_log_cap;
  const int tid = warp * 32 + lane;

  unsigned* lut = reinterpret_cast<unsigned*>(ws + lay.lut);
  unsigned char* ring = ws + lay.ring;
  unsigned char* qs = ws + lay.q;
  unsigned long long* res = reinterpret_cast<unsigned long long*>(ws + lay.res);
  unsigned long long* cand = reinterpret_cast<unsigned long long*>(ws + lay.cand);
  unsigned long long* ring_key = reinterpret_cast<unsigned long long*>(ws + lay.ring_key);
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(ws + lay.keys);
  unsigned char* flags = ws + lay.flags;
  int* rank = reinterpret_cast<int*>(ws + lay.rank);
  const int slot_bytes = a.slot_bytes;

  // ---- query vector into shared memory
  {
    const unsigned* src = static_cast<const unsigned*>(job.query);
    unsigned* dst = reinterpret_cast<unsigned*>(qs);
    for (int j = tid; j < (d >> 2); j += 32 * W) dst[j] = __ldg(src + j);
  }
  __syncthreads();

  // ---- a1: lookup table, subspace pairs split across the warps
  {
    const int wps = a.dsub >> 2;
    const unsigned* qw = reinterpret_cast<const unsigned*>(qs);
    for (int m = 2 * warp; m < a.M; m += 2 * W) {
      unsigned acc[2][8];
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[h][j] = 0u;
      for (int w = 0; w < wps; ++w) {
        unsigned cv[2][8];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int j = 0; j < 8; ++j)
            cv[h][j] = __ldg(a.cb_words + (static_cast<size_t>(m + h) * 256 + lane + 32 * j) * wps + w);
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[h][j] = sq4(qw[(m + h) * wps + w], cv[h][j], acc[h][j]);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int j = 0; j < 8; ++j) lut[(m + h) * 256 + lane + 32 * j] = acc[h][j];
    }
  }
  __syncthreads();

  // ---- a2: entry node (warp 0)
  int len = 1, nres = 0, head = 0, inflight = 0, steps = 0, status = ANN_OK, first_open = 0;
  // From L = kLazyL on, as in run_query: the step's candidates go to a sorted
  // pending buffer (warp 0), merged into the list by all warps when full;
  // the list is the first L entries of the union of both.
  const bool lazy = L >= kLazyL;
  unsigned long long* pkeys = reinterpret_cast<unsigned long long*>(ws + lay.pkeys);
  unsigned char* pflags = ws + lay.pflags;
  int plen = 0, pfirst_open = 0;
  const int max_steps = n + 1;
  if (warp == 0) {
    const uint8_t* code = a.codes + static_cast<size_t>(a.entry) * a.M;
    unsigned part = 0;
    for (int m = lane; m < a.M; m += 32) part += lut[m * 256 + code[m]];
    const unsigned entry_dist = warp_sum_u32(part);
    if (lane == 0) {
      keys[0] = make_key(entry_dist, a.entry);
      flags[0] = 0;
      atomicOr(vis + (static_cast<unsigned>(a.entry) >> 5), 1u << (a.entry & 31));
      vlog[0] = static_cast<unsigned>(a.entry) >> 5;
      ctl->vis_count = 1;
    }
    for (int j = lane; j < k; j += 32) res[j] = kNoKey;
    __syncwarp();
  }

  // Merge sorted src[0..cs) (flags sf, or 0) into the list of length lv in
  // place, all warps: rank them, move the list's tail right in rounds of W
  // blocks (all reads of a round before its writes; entries only move right,
  // so the rounds run top-down), then drop the new entries into their
  // places; entries pushed past L fall off.  Returns the first changed
  // position.  Ends with every thread synchronised.
  auto wg_merge = [&](const unsigned long long* src, const unsigned char* sf, int cs, int lv) -> int {
    for (int j = tid; j < cs; j += 32 * W) rank[j] = lower_bound_u64(keys, lv, src[j]);
    __syncthreads();
    const int pos0 = rank[0];
    constexpr int kB = 256;  // entries per warp per round (8 per lane)
    const int top_block = ((lv - 1) / kB) * kB;
    const int low_block = (pos0 / kB) * kB;
    for (int r0 = top_block; r0 >= low_block; r0 -= W * kB) {
      const int b = r0 - warp * kB;
      unsigned long long kv[8];
      unsigned char fv[8];
      int np[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int i = b + t * 32 + lane;
        const bool live = b >= low_block && i >= pos0 && i < lv;
        kv[t] = live ? keys[i] : 0ull;
        fv[t] = live ? flags[i] : 0;
        np[t] = !live ? L : (i >= rank[cs - 1] ? i + cs : i + upper_bound_i32(rank, cs, i));
      }
      __syncthreads();
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if (np[t] < L) {
          keys[np[t]] = kv[t];
          flags[np[t]] = fv[t];
        }
      }
      __syncthreads();
    }
    for (int j = tid; j < cs; j += 32 * W) {
      const int p = j + rank[j];
      if (p < L) {
        keys[p] = src[j];
        flags[p] = sf ? sf[j] : 0;
      }
    }
    __syncthreads();
    return pos0;
  };

  // Next-node prefetch (depth >= 2), as in run_query: once this step's
  // candidates are in, the next node's block has landed (warp 0 waits for
  // it), and every warp issues the code gathers and visited-bit atomics of
  // its share of that node's neighbours, so their round trip overlaps this
  // step's sort and merge and the next step's selection.  The block barrier
  // before them orders them after this node's atomics (whose results every
  // warp has already used), so the visited set sees the same inserts in the
  // same order.
  const bool prefetch = D >= 2;
  bool pre = false;
  int pw[NBW];
  unsigned pword[NBW], pold[NBW];
  uint4 pcode[NBW][kMaxM / 16];
  // this warp's share of the neighbours of the block at `b`: ids, code
  // gathers, visited-bit atomics
  auto issue_share = [&](const unsigned char* b, int (&w)[NBW], unsigned (&word)[NBW],
                         uint4 (&code)[NBW][kMaxM / 16], unsigned (&old)[NBW]) {
    const int32_t* nbr = reinterpret_cast<const int32_t*>(b + a.ids_off);
#pragma unroll
    for (int t = 0; t < NBW; ++t) {
      const int jj = t * 32 + lane;
      const int j = warp * kChunk + jj;
      int id = (jj < kChunk && j < a.R) ? nbr[j] : -1;
      if (id >= n) id = -1;
      w[t] = id;
      word[t] = id >= 0 ? static_cast<unsigned>(id) >> 5 : 0u;
    }
#pragma unroll
    for (int t = 0; t < NBW; ++t) {
      if (w[t] >= 0) {
        const uint4* cp = reinterpret_cast<const uint4*>(a.codes + static_cast<size_t>(w[t]) * a.M);
#pragma unroll
        for (int c = 0; c < kMaxM / 16; ++c)
          if (c < (a.M >> 4)) code[t][c] = __ldg(cp + c);
      }
    }
#pragma unroll
    for (int t = 0; t < NBW; ++t)
      old[t] = w[t] >= 0 ? atomicOr(vis + word[t], 1u << (w[t] & 31)) : 0u;
  };

  for (;;) {
    // ---- a3-a5 (warp 0): select, issue fetches, and wait for the oldest
    // when more than D are in flight or nothing is selectable
    if (warp == 0) {
      int act = 0, slot_u = 0;
      unsigned long long ukey = 0;
      do {
        int sel = -1, src = 0;  // src 0: list entry sel, 1: pending entry sel
        unsigned long long key = 0;
        if (status == ANN_OK) {
          int ia = -1, ib = -1;
          for (int b = first_open; b < len; b += 32) {
            const int i = b + lane;
            const unsigned m = __ballot_sync(kFull, i < len && flags[i] == 0);
            if (m) {
              ia = b + __ffs(m) - 1;
              break;
            }
          }
          for (int b = pfirst_open; b < plen; b += 32) {
            const int i = b + lane;
            const unsigned m = __ballot_sync(kFull, i < plen && pflags[i] == 0);
            if (m) {
              ib = b + __ffs(m) - 1;
              break;
            }
          }
          first_open = ia >= 0 ? ia : len;
          pfirst_open = ib >= 0 ? ib : plen;
          // the smaller of the two, if its rank in the union is below L
          if (ia >= 0 && (ib < 0 || keys[ia] < pkeys[ib])) {
            key = keys[ia];
            if (plen == 0 || ia + lower_bound_u64(pkeys, plen, key) < L) sel = ia;
          } else if (ib >= 0) {
            key = pkeys[ib];
            if (ib + lower_bound_u64(keys, len, key) < L) {
              sel = ib;
              src = 1;
            }
          }
          if (sel >= 0 && src == 0) first_open = sel + 1;
          if (sel >= 0 && src == 1) pfirst_open = sel + 1;
        }
        if (sel >= 0) {
          const unsigned v = static_cast<unsigned>(key);
          int slot = head + inflight;
          if (slot > D) slot -= D + 1;
          __syncwarp();
          if (lane == 0) {
            if (src == 0) flags[sel] = 1; else pflags[sel] = 1;
            ring_key[slot] = key;
          }
          const uint8_t* src = a.blocks + static_cast<size_t>(v) * a.block_bytes;
          unsigned char* dst = ring + slot * slot_bytes;
          for (int off = lane * 16; off < slot_bytes; off += 512) cp_async_16(dst + off, src + off);
          cp_async_commit();
          ++inflight;
          __syncwarp();
        }
        if (inflight > D || (sel < 0 && inflight > 0)) {
          if (status != ANN_OK) {  // stopping early: drain, expand nothing more
            cp_async_wait_pending(0);
            __syncwarp();
            inflight = 0;
            act = 2;
          } else {
            cp_async_wait_pending(inflight - 1);
            __syncwarp();
            slot_u = head;
            ukey = ring_key[head];
            head = (head == D) ? 0 : head + 1;
            --inflight;
            ++steps;
            act = 1;
          }
        } else if (sel < 0) {
          act = 2;  // ---- a10: nothing selectable, nothing in flight
        }
      } while (act == 0);
      if (lane == 0) {
        ctl->act = act;
        ctl->slot = slot_u;
        ctl->ukey = ukey;
        ctl->len = len;
        ctl->plen = plen;
        ctl->cand_count = 0;
      }
    }
    __syncthreads();  // the block landed (warp 0 waited for it); control published
    if (ctl->act == 2) break;
    const unsigned char* blk = ring + ctl->slot * slot_bytes;
    const int lenv = ctl->len;
    const int plenv = ctl->plen;
    // a key at or above the L-th of list and pending buffer together cannot enter
    const unsigned long long thr =
        plenv == 0 ? ((lenv == L) ? keys[L - 1] : kNoKey)
                   : (lenv + plenv >= L ? kth_of_two(keys, lenv, pkeys, plenv, L - 1) : kNoKey);

    // ---- a6 (warp 0): exact distance of the expanded node into the results
    if (warp == 0) {
      const unsigned* xw = reinterpret_cast<const unsigned*>(blk);
      const unsigned* qw = reinterpret_cast<const unsigned*>(qs);
      unsigned acc = 0;
      for (int j = lane; j < (d >> 2); j += 32) acc = sq4(qw[j], xw[j], acc);
      result_insert(res, nres, k, make_key(warp_sum_u32(acc), static_cast<unsigned>(ctl->ukey)), lane);
    }

    // ---- a7: this warp's neighbour positions and the visited set (issued
    // one step early when the node was prefetched)
    int w[NBW];
    unsigned word[NBW];
    bool fresh[NBW];
    uint4 code[NBW][kMaxM / 16];
    unsigned old[NBW];
    if (pre) {
#pragma unroll
      for (int t = 0; t < NBW; ++t) {
        w[t] = pw[t];
        word[t] = pword[t];
        old[t] = pold[t];
#pragma unroll
        for (int c = 0; c < kMaxM / 16; ++c) code[t][c] = pcode[t][c];
      }
      pre = false;
    } else {
      issue_share(blk, w, word, code, old);
    }
#pragma unroll
    for (int t = 0; t < NBW; ++t) fresh[t] = w[t] >= 0 && ((old[t] >> (w[t] & 31)) & 1u) == 0u;
    // ---- a8: asymmetric distances from the lookup table
    unsigned long long key[NBW];
#pragma unroll
    for (int t = 0; t < NBW; ++t) {
      key[t] = kNoKey;
      if (fresh[t]) {
        unsigned dist = 0;
#pragma unroll
        for (int c = 0; c < kMaxM / 16; ++c) {
          if (c < (a.M >> 4)) {
            const unsigned wd[4] = {code[t][c].x, code[t][c].y, code[t][c].z, code[t][c].w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int m0 = c * 16 + e * 4;
              dist += lut[(m0 + 0) * 256 + (wd[e] & 0xff)];
              dist += lut[(m0 + 1) * 256 + ((wd[e] >> 8) & 0xff)];
              dist += lut[(m0 + 2) * 256 + ((wd[e] >> 16) & 0xff)];
              dist += lut[(m0 + 3) * 256 + (wd[e] >> 24)];
            }
          }
        }
        key[t] = make_key(dist, static_cast<unsigned>(w[t]));
      }
    }
    // new nodes' words to the clear log, entering keys to the step's candidates
    const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int t = 0; t < NBW; ++t) {
      const unsigned mf = __ballot_sync(kFull, fresh[t]);
      if (mf) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&ctl->vis_count, __popc(mf));
        base = __shfl_sync(kFull, base, 0);
        const int at = base + __popc(mf & lt_mask);
        if (fresh[t] && at < log_cap) vlog[at] = word[t];
      }
      const bool enter = fresh[t] && key[t] < thr;
      const unsigned me = __ballot_sync(kFull, enter);
      if (me) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&ctl->cand_count, __popc(me));
        base = __shfl_sync(kFull, base, 0);
        if (enter) cand[base + __popc(me & lt_mask)] = key[t];
      }
    }
    __syncthreads();  // every warp's candidates and log entries are in

    // the next node's loads, overlapping the sort and merge below
    if (prefetch) {
      if (warp == 0) {
        int ps = -1;
        if (inflight >= 2) {
          cp_async_wait_pending(inflight - 1);  // the next node's block (issued a step ago or more)
          ps = head;
        }
        __syncwarp();
        if (lane == 0) ctl->pf_slot = ps;
      }
      __syncthreads();  // its block is visible to every warp
      const int ps = ctl->pf_slot;
      if (ps >= 0) {
        issue_share(ring + ps * slot_bytes, pw, pword, pcode, pold);
        pre = true;
      }
    }

    // ---- a9: sort the candidates (warp 0), then merge them into the list
    // (all warps), or, for long lists, into the pending buffer (warp 0)
    const int c = ctl->cand_count;
    if (c > 0) {
      if (warp == 0) {
        if (c <= 32) {
          unsigned long long one[1] = {lane < c ? cand[lane] : kNoKey};
          __syncwarp();
          warp_bitonic_sort<1>(one, lane);
          cand[lane] = one[0];
        } else {
          unsigned long long v[NB];
#pragma unroll
          for (int t = 0; t < NB; ++t) v[t] = (t * 32 + lane < c) ? cand[t * 32 + lane] : kNoKey;
          __syncwarp();
          warp_bitonic_sort<NB>(v, lane);
#pragma unroll
          for (int t = 0; t < NB; ++t) cand[t * 32 + lane] = v[t];
        }
      }
      __syncthreads();
      if (!lazy) {
        const int pos0 = wg_merge(cand, nullptr, c, lenv);
        if (warp == 0) {
          len = (lenv + c < L) ? lenv + c : L;
          if (pos0 < first_open) first_open = pos0;
        }
      } else {
        if (plenv + c > kPend) {
          // the pending buffer is full: all warps merge it, selected flags
          // and all, into the list (entries past rank L fall off)
          const int pos0 = wg_merge(pkeys, pflags, plenv, lenv);
          if (warp == 0) {
            len = (lenv + plenv < L) ? lenv + plenv : L;
            if (pos0 < first_open) first_open = pos0;
            plen = 0;
            pfirst_open = 0;
          }
        }
        if (warp == 0) {
          // this step's candidates into the pending buffer (one warp)
          QueryState pend;
          pend.keys = pkeys;
          pend.flags = pflags;
          pend.rank = rank;
          pend.len = plen;
          const int pchanged = merge_candidates(pend, cand, c, kPend, lane);
          plen = pend.len;
          if (pchanged < pfirst_open) pfirst_open = pchanged;
        }
      }
    }
    if (warp == 0 && steps >= max_steps) status = ANN_ENOMEM;  // cannot happen (each node expands once)
  }

  // ---- a11: results (warp 0); the visited slots are cleared by every warp
  if (warp == 0) {
    for (int j = lane; j < k; j += 32) {
      const unsigned long long r = j < nres ? res[j] : kNoKey;
      const bool ok = r != kNoKey;
      const int32_t id = static_cast<int32_t>(r & 0xffffffffu);
      job.ids[j] = ok ? (a.id_map ? __ldg(a.id_map + id) : id) : -1;
      job.dists[j] = ok ? static_cast<float>(static_cast<unsigned>(r >> 32)) : __int_as_float(0x7f800000);
    }
  }
  // a stop with a prefetched node left its visited bits out of the log:
  // clear the whole table then, as run_query does
  clear_visited(vis, vlog, pre ? log_cap + 1 : ctl->vis_count, log_cap, a.vis_words, lane, warp, W);
  if (warp == 0 && lane == 0) {
    if (job.steps) *job.steps = steps;
    if (job.status) *job.status = status;
    if (job.t_begin) *job.t_begin = t0;
    if (job.t_end) *job.t_end = global_timer_ns();
    atomicAdd(a.expansions, static_cast<unsigned long long>(steps));
    if (status != ANN_OK) {
      atomicAdd(&a.counters[1], 1);
      atomicMin(&a.counters[2], job.qi);
    }
  }
  __syncthreads();  // the table is clear and the control words free for the next query
}

// Persistent warp-group kernel: one query per block of W warps.
template <int NB, int W>
__global__ void __launch_bounds__(32 * W) search_kernel_wg(SearchArgs a, int smem_per_query) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WgCtl* ctl = reinterpret_cast<WgCtl*>(smem + smem_per_query);
  const WarpSmem lay = warp_smem_layout(kModePqU8, a.M, a.d, a.slot_bytes, a.depth, a.L, a.k, NB);
  uint32_t* vis = a.vis + static_cast<size_t>(blockIdx.x) * a.vis_words;
  uint32_t* vlog = a.vis_log + static_cast<size_t>(blockIdx.x) * a.vis_log_cap;
  for (;;) {
    if (threadIdx.x == 0) ctl->qi = atomicAdd(&a.counters[0], 1);
    __syncthreads();
    const int qi = ctl->qi;
    if (qi >= a.nq) break;
    QueryJob job;
    job.query = static_cast<const uint8_t*>(a.queries) + static_cast<size_t>(qi) * a.d;
    job.k = a.k;
    job.L = a.L;
    job.qi = qi;
    job.ids = a.ids + static_cast<size_t>(qi) * a.k;
    job.dists = a.dists + static_cast<size_t>(qi) * a.k;
    job.steps = a.steps ? a.steps + qi : nullptr;
    job.status = a.status ? a.status + qi : nullptr;
    job.t_begin = a.t_begin ? a.t_begin + qi : nullptr;
    job.t_end = a.t_end ? a.t_end + qi : nullptr;
    run_query_wg<NB, W>(a, job, smem, lay, vis, vlog, warp, lane, ctl);
  }
}

// Persistent serving kernel: every warp claims published work items one at a
// time (atomicCAS on the device head, against the published tail), runs the
// search for it and writes the results straight into mapped host memory,
// then the item's done word.  Work items of different requests and of
// different k and L share the warps as they free up (continuous batching).
// Only one warp in kPollEvery keeps reading the host-written tail over PCIe
// (relaxed loads) while idle, folding it into a device-memory mirror; the
// other idle warps look at the mirror, so idle polling costs PCIe round trips
// only from a few warps.
// An idle warp backs off (longer for non-polling warps) and returns once no
// warp of the kernel has claimed work for s.idle_ns (a kernel-wide decision,
// so the kernel never dwindles to a few warps under light load), or when the
// host sets s.stop; the host relaunches the kernel when new items arrive.  A claim is followed by a
// system-scope fence, and host-written memory is read with system-scope
// loads (never through the non-coherent cache), so a reused slot never
// yields stale data.
template <int MODE, int NB>
__global__ void serve_kernel(SearchArgs a, ServeArgs s, int smem_per_warp) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int warps = blockDim.x >> 5;
  unsigned char* ws = smem + wib * smem_per_warp;
  const WarpSmem lay = warp_smem_layout(MODE, a.M, a.d, a.slot_bytes, a.depth, a.L, a.k, NB);
  const size_t gw = static_cast<size_t>(blockIdx.x) * warps + wib;
  uint32_t* vis = a.vis + gw * static_cast<size_t>(a.vis_words);
  uint32_t* vlog = a.vis_log + gw * static_cast<size_t>(a.vis_log_cap);
  constexpr int kPollEvery = 32;
  const bool poller = (gw % kPollEvery) == 0;
  const unsigned max_backoff = poller ? 16384u : 65536u;
  const long long started = global_timer_ns();
  unsigned backoff = 128;
  for (;;) {
    long long got = -1;
    if (lane == 0) {
      unsigned long long t = *reinterpret_cast<volatile unsigned long long*>(s.tail_mirror);
      unsigned long long h = *reinterpret_cast<volatile unsigned long long*>(s.head);
      // the host tail is read by polling warps, and by any warp right after it
      // finished a query (backoff reset), so fresh work is never left waiting
      // for a poller that is busy
      if (h >= t && (poller || backoff == 128u)) {
        unsigned long long th;
        asm volatile("ld.relaxed.sys.global.u64 %0, [%1];" : "=l"(th) : "l"(s.tail) : "memory");
        if (th > t) {
          atomicMax(s.tail_mirror, th);
          t = th;
        }
      }
      while (h < t) {
        const unsigned long long prev = atomicCAS(s.head, h, h + 1);
        if (prev == h) {
          got = static_cast<long long>(h);
          break;
        }
        h = prev;
      }
      if (got >= 0) {
        atomicMax(s.last_claim, static_cast<unsigned long long>(global_timer_ns()));
        asm volatile("fence.acq_rel.sys;" ::: "memory");
      }
    }
    got = __shfl_sync(kFull, got, 0);
    if (got < 0) {
      int stop = 0;
      if (lane == 0 && poller) stop = static_cast<int>(ld_relaxed_sys_u32(s.stop));
      stop = __shfl_sync(kFull, stop, 0);
      long long ref = static_cast<long long>(*reinterpret_cast<volatile unsigned long long*>(s.last_claim));
      if (ref < started) ref = started;
      if (stop || global_timer_ns() - ref > s.idle_ns) break;
      __nanosleep(backoff);
      backoff = backoff < max_backoff ? backoff * 2 : max_backoff;
      continue;
    }
    const int slot = static_cast<int>(got % s.slots);
    // the query into shared memory (system-scope loads of host memory)
    {
      const unsigned char* src = s.qbuf + static_cast<size_t>(slot) * s.qbytes;
      unsigned* dst = reinterpret_cast<unsigned*>(ws + lay.q);
      for (int j = lane; j < (s.qbytes >> 2); j += 32) dst[j] = ld_relaxed_sys_u32(src + 4 * j);
    }
    QueryJob job;
    job.query = nullptr;
    job.k = static_cast<int>(ld_relaxed_sys_u32(s.item_kL + 2 * slot));
    job.L = static_cast<int>(ld_relaxed_sys_u32(s.item_kL + 2 * slot + 1));
    job.qi = slot;
    job.ids = s.rids + static_cast<size_t>(slot) * s.max_k;
    job.dists = s.rdists + static_cast<size_t>(slot) * s.max_k;
    job.steps = s.rsteps + slot;
    job.status = s.rstatus + slot;
    job.t_begin = s.rtimes + 2 * slot;
    job.t_end = s.rtimes + 2 * slot + 1;
    if (job.k < 1 || job.k > a.k || job.L < job.k || job.L > a.L) {
      // rejected at submission; guards the shared-memory layout all the same
      if (lane == 0) *job.status = ANN_EINVAL;
    } else {
      run_query<MODE, NB>(a, job, ws, lay, vis, vlog, lane);
    }
    __syncwarp();
    if (lane == 0) {
      __threadfence_system();  // results before the done word
      *reinterpret_cast<volatile unsigned long long*>(s.done + slot) =
          static_cast<unsigned long long>(got) + 1ull;
    }
    backoff = 128;
  }
}

template <int MODE, int NB>
cudaError_t launch_serve_t(const SearchArgs& a, const ServeArgs& s, const SearchPlan& p,
                           cudaStream_t st) {
  const int smem = p.smem_per_warp * p.warps_per_block;
  cudaError_t e = cudaFuncSetAttribute(serve_kernel<MODE, NB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  serve_kernel<MODE, NB><<<p.blocks, 32 * p.warps_per_block, smem, st>>>(a, s, p.smem_per_warp);
  return cudaGetLastError();
}

template <int MODE, int NB, bool PF = false>
cudaError_t launch_t(const SearchArgs& a, const SearchPlan& p, cudaStream_t st) {
  const int smem = p.smem_per_warp * p.warps_per_block;
  cudaError_t e = cudaFuncSetAttribute(search_kernel<MODE, NB, PF>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  search_kernel<MODE, NB, PF><<<p.blocks, 32 * p.warps_per_block, smem, st>>>(a, p.smem_per_warp);
  return cudaGetLastError();
}

template <int MODE, int NB>
cudaError_t launch_coop_t(const SearchArgs& a, const SearchPlan& p, cudaStream_t st) {
  const int smem = p.smem_per_warp * p.warps_per_block;
  cudaError_t e = cudaFuncSetAttribute(search_kernel<MODE, NB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  SearchArgs args = a;
  int spw = p.smem_per_warp;
  void* params[] = {&args, &spw};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(search_kernel<MODE, NB>),
                                     dim3(p.blocks), dim3(32 * p.warps_per_block), params,
                                     static_cast<size_t>(smem), st);
}

template <int NB, int W>
cudaError_t launch_wg_t(const SearchArgs& a, const SearchPlan& p, cudaStream_t st) {
  const int smem = p.smem_per_warp + kWgCtlBytes;
  cudaError_t e = cudaFuncSetAttribute(search_kernel_wg<NB, W>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  search_kernel_wg<NB, W><<<p.blocks, 32 * W, smem, st>>>(a, p.smem_per_warp);
  return cudaGetLastError();
}

template <int NB, int W>
cudaError_t occupancy_wg_t(int smem_block, int threads, int* blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(search_kernel_wg<NB, W>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem_block);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, search_kernel_wg<NB, W>,
                                                       threads, smem_block);
}

template <int MODE, int NB, bool PF = false>
cudaError_t occupancy_t(int smem_block, int threads, int* blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(search_kernel<MODE, NB, PF>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem_block);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, search_kernel<MODE, NB, PF>,
                                                       threads, smem_block);
}

using LaunchFn = cudaError_t (*)(const SearchArgs&, const SearchPlan&, cudaStream_t);
using OccFn = cudaError_t (*)(int, int, int*);

int nb_index(int nb) { return nb == 1 ? 0 : (nb == 2 ? 1 : 2); }

// PQ navigation with the next-node prefetch (depth >= 2, one warp per query)
LaunchFn launch_pf_table(int nb) {
  static const LaunchFn t[3] = {launch_t<kModePqU8, 1, true>, launch_t<kModePqU8, 2, true>,
                                launch_t<kModePqU8, 4, true>};
  return t[nb_index(nb)];
}

OccFn occ_pf_table(int nb) {
  static const OccFn t[3] = {occupancy_t<kModePqU8, 1, true>, occupancy_t<kModePqU8, 2, true>,
                             occupancy_t<kModePqU8, 4, true>};
  return t[nb_index(nb)];
}

// Warp-group kernels: [nb][W == 4]
LaunchFn launch_wg_table(int nb, int w) {
  static const LaunchFn t[3][2] = {{launch_wg_t<1, 2>, launch_wg_t<1, 4>},
                                   {launch_wg_t<2, 2>, launch_wg_t<2, 4>},
                                   {launch_wg_t<4, 2>, launch_wg_t<4, 4>}};
  return t[nb_index(nb)][w == 4 ? 1 : 0];
}

OccFn occ_wg_table(int nb, int w) {
  static const OccFn t[3][2] = {{occupancy_wg_t<1, 2>, occupancy_wg_t<1, 4>},
                                {occupancy_wg_t<2, 2>, occupancy_wg_t<2, 4>},
                                {occupancy_wg_t<4, 2>, occupancy_wg_t<4, 4>}};
  return t[nb_index(nb)][w == 4 ? 1 : 0];
}

LaunchFn launch_table(int mode, int nb) {
  static const LaunchFn t[kNumModes][3] = {
      {launch_t<kModePqU8, 1>, launch_t<kModePqU8, 2>, launch_t<kModePqU8, 4>},
      {launch_t<kModeExactU8, 1>, launch_t<kModeExactU8, 2>, launch_t<kModeExactU8, 4>},
      {launch_t<kModeExactF32, 1>, launch_t<kModeExactF32, 2>, launch_t<kModeExactF32, 4>},
      {launch_t<kModeBF16, 1>, launch_t<kModeBF16, 2>, launch_t<kModeBF16, 4>},
      {launch_t<kModeFP8, 1>, launch_t<kModeFP8, 2>, launch_t<kModeFP8, 4>},
      {launch_t<kModePqF32, 1>, launch_t<kModePqF32, 2>, launch_t<kModePqF32, 4>}};
  return t[mode][nb_index(nb)];
}

OccFn occ_table(int mode, int nb) {
  static const OccFn t[kNumModes][3] = {
      {occupancy_t<kModePqU8, 1>, occupancy_t<kModePqU8, 2>, occupancy_t<kModePqU8, 4>},
      {occupancy_t<kModeExactU8, 1>, occupancy_t<kModeExactU8, 2>, occupancy_t<kModeExactU8, 4>},
      {occupancy_t<kModeExactF32, 1>, occupancy_t<kModeExactF32, 2>, occupancy_t<kModeExactF32, 4>},
      {occupancy_t<kModeBF16, 1>, occupancy_t<kModeBF16, 2>, occupancy_t<kModeBF16, 4>},
      {occupancy_t<kModeFP8, 1>, occupancy_t<kModeFP8, 2>, occupancy_t<kModeFP8, 4>},
      {occupancy_t<kModePqF32, 1>, occupancy_t<kModePqF32, 2>, occupancy_t<kModePqF32, 4>}};
  return t[mode][nb_index(nb)];
}

}  // namespace

cudaError_t plan_search(int mode, int R, int M, int d, int slot_bytes, int depth, int L, int k,
                        int64_t nq, SearchPlan* plan, int64_t n_index, int wpq) {
  SearchPlan p;
  p.mode = mode;
  p.nb = R <= 32 ? 1 : (R <= 64 ? 2 : 4);
  const WarpSmem lay = warp_smem_layout(mode, M, d, slot_bytes, depth, L, k, p.nb);
  p.smem_per_warp = lay.total;
  p.warps_per_block = 1;
  // a warp group per query: PQ navigation only; W warps share one query
  p.wpq = (mode == kModePqU8 && (wpq == 2 || wpq == 4)) ? wpq : 1;
  // Visited set: one bit per node of the index, so it can neither overflow
  // nor collide (one atomicOr per neighbour, no probing).  Words per query,
  // rounded to 128 bytes; the clear log keeps up to kVisLog word indices.
  p.vis_words = ((n_index > 0 ? n_index : 1) + 1023) / 1024 * 32;
  p.vis_log_cap = kVisLog;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  p.pf = mode == kModePqU8 && p.wpq == 1 && depth >= 2;
  if (p.wpq > 1)
    e = occ_wg_table(p.nb, p.wpq)(p.smem_per_warp + kWgCtlBytes, 32 * p.wpq, &per_sm);
  else if (p.pf)  // (never more blocks than the plain kernel: safe for the cooperative launch)
    e = occ_pf_table(p.nb)(p.smem_per_warp * p.warps_per_block, 32 * p.warps_per_block, &per_sm);
  else
    e = occ_table(mode, p.nb)(p.smem_per_warp * p.warps_per_block, 32 * p.warps_per_block, &per_sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t blocks = static_cast<int64_t>(sms) * per_sm;
  const int64_t need = p.wpq > 1 ? nq : (nq + p.warps_per_block - 1) / p.warps_per_block;
  if (blocks > need) blocks = need > 0 ? need : 1;
  p.blocks = static_cast<int>(blocks);
  p.tables = p.wpq > 1 ? p.blocks : p.blocks * p.warps_per_block;
  *plan = p;
  return cudaSuccess;
}

cudaError_t launch_search(const SearchArgs& a, const SearchPlan& plan, cudaStream_t stream) {
  if (plan.wpq > 1) return launch_wg_table(plan.nb, plan.wpq)(a, plan, stream);
  if (plan.pf && !a.grid_bar && !a.agent_req) return launch_pf_table(plan.nb)(a, plan, stream);
  return launch_table(plan.mode, plan.nb)(a, plan, stream);
}

cudaError_t launch_search_coop(const SearchArgs& a, const SearchPlan& plan, cudaStream_t stream) {
  static const LaunchFn t[kNumModes][3] = {
      {launch_coop_t<kModePqU8, 1>, launch_coop_t<kModePqU8, 2>, launch_coop_t<kModePqU8, 4>},
      {launch_coop_t<kModeExactU8, 1>, launch_coop_t<kModeExactU8, 2>, launch_coop_t<kModeExactU8, 4>},
      {launch_coop_t<kModeExactF32, 1>, launch_coop_t<kModeExactF32, 2>, launch_coop_t<kModeExactF32, 4>},
      {launch_coop_t<kModeBF16, 1>, launch_coop_t<kModeBF16, 2>, launch_coop_t<kModeBF16, 4>},
      {launch_coop_t<kModeFP8, 1>, launch_coop_t<kModeFP8, 2>, launch_coop_t<kModeFP8, 4>},
      {launch_coop_t<kModePqF32, 1>, launch_coop_t<kModePqF32, 2>, launch_coop_t<kModePqF32, 4>}};
  return t[plan.mode][nb_index(plan.nb)](a, plan, stream);
}

cudaError_t launch_serve(const SearchArgs& a, const ServeArgs& s, const SearchPlan& plan,
                         cudaStream_t stream) {
  using ServeFn = cudaError_t (*)(const SearchArgs&, const ServeArgs&, const SearchPlan&, cudaStream_t);
  static const ServeFn t[kNumModes][3] = {
      {launch_serve_t<kModePqU8, 1>, launch_serve_t<kModePqU8, 2>, launch_serve_t<kModePqU8, 4>},
      {launch_serve_t<kModeExactU8, 1>, launch_serve_t<kModeExactU8, 2>, launch_serve_t<kModeExactU8, 4>},
      {launch_serve_t<kModeExactF32, 1>, launch_serve_t<kModeExactF32, 2>, launch_serve_t<kModeExactF32, 4>},
      {launch_serve_t<kModeBF16, 1>, launch_serve_t<kModeBF16, 2>, launch_serve_t<kModeBF16, 4>},
      {launch_serve_t<kModeFP8, 1>, launch_serve_t<kModeFP8, 2>, launch_serve_t<kModeFP8, 4>},
      {launch_serve_t<kModePqF32, 1>, launch_serve_t<kModePqF32, 2>, launch_serve_t<kModePqF32, 4>}};
  return t[plan.mode][nb_index(plan.nb)](a, s, plan, stream);
}

}  // namespace ann
