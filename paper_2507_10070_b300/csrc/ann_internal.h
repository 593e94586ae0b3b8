// Internal declarations of libann (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>

#include "../../include/ann.h"

namespace ann {

// Navigation / fetch modes of the search kernel.
enum Mode : int {
  kModePqU8 = 0,     // PQ navigation, node blocks in the storage tier (uint8 data)
  kModeExactU8 = 1,  // exact navigation on uint8 vectors in HBM
  kModeExactF32 = 2, // exact navigation on float32 vectors in HBM
  kModeBF16 = 3,     // navigation on BF16 copies of float32 vectors (HBM), FP32 accumulation
  kModeFP8 = 4,      // navigation on FP8-E4M3 copies (x * scale), FP32 accumulation
  kModePqF32 = 5,    // PQ navigation with a float codebook (float32 data), FP32 lookup table
  kNumModes = 6
};

// Modes whose query and distances are float32 (keys hold float bit patterns).
__host__ __device__ constexpr bool mode_f32(int m) {
  return m == kModeExactF32 || m == kModeBF16 || m == kModeFP8 || m == kModePqF32;
}
__host__ __device__ constexpr bool mode_pq(int m) { return m == kModePqU8 || m == kModePqF32; }

constexpr int kMaxL = 16384;
constexpr int kMaxDepth = 4;
constexpr int kMaxR = 128;
constexpr int kMaxD = 512;
constexpr int kMaxM = 64;
constexpr int kVisLog = 8192;  // entries of a query's visited-set clear log

// One CPU-agent request: the node whose block a warp wants, and a sequence
// number (written last) that tells the host the entry is new.
struct AgentReq {
  int32_t node;
  uint32_t seq;
};

// Everything one launch of the search kernel reads or writes.
struct SearchArgs {
  // index
  int32_t n, d, R, entry, M, dsub;
  const uint8_t* blocks;    // PQ mode: n node blocks (host-mapped or HBM)
  int32_t block_bytes;      // bytes per node block (multiple of 16)
  int32_t ids_off;          // byte offset of the neighbour ids in a block
  int32_t deg_off;          // byte offset of the degree in a block (not fetched)
  int32_t slot_bytes;       // bytes fetched per expansion into a ring slot (multiple of 16)
  const uint8_t* codes;     // PQ mode: n*M codes (HBM)
  const uint32_t* cb_words; // PQ mode: M*256*(dsub/4) words, 4 uint8 coordinates each
  const float* cb_f32;      // float PQ mode: M*256*dsub centroid coordinates
  const void* nav;          // BF16 / FP8 modes: n*d navigation copies (HBM)
  float nav_inv_scale;      // FP8 mode: 1 / the encoding scale
  const void* vectors;      // exact modes: n*d elements (HBM)
  const int32_t* adj;       // exact modes: n*adj_stride ids (HBM)
  int32_t adj_stride;       // ids per adjacency row (multiple of 4)
  const int32_t* id_map;    // caller's id of each stored node, written to the results (HBM), or null
  unsigned* grid_bar;       // kernel-grained I/O ablation: grid barrier state (4 words), or null
  // CPU-agent I/O (the paper's mapped request array, an ablation); agent_req
  // null = the warps read node blocks themselves.  Per resident warp, D + 1
  // entries: the warp writes a request (node, sequence number) into
  // agent_req, a host thread copies the block into that entry's staging slot
  // and then writes the sequence number into agent_done.
  AgentReq* agent_req;      // [warps * (D + 1)], host-mapped, written by the GPU
  const unsigned* agent_done;      // [warps * (D + 1)], host-mapped, written by the host
  const uint8_t* agent_stage;      // [warps * (D + 1) * slot_bytes], host-mapped, written by the host
  unsigned* agent_seq;      // [warps * (D + 1)] last sequence number issued (device memory)
  int64_t agent_wait_ns;    // bound on one wait for a completion
  // batch
  const void* queries;
  int32_t nq, k, L, depth;
  int32_t* ids;
  float* dists;
  int32_t* steps;
  int32_t* status;
  int64_t* t_begin;
  int64_t* t_end;
  // scratch
  uint32_t* vis;            // per-query visited bitsets (one bit per node), all zero between queries
  int64_t vis_words;        // 32-bit words per bitset (a multiple of 32)
  uint32_t* vis_log;        // per-bitset log of the words a query set (to clear them)
  int32_t vis_log_cap;      // entries per bitset in vis_log
  int32_t* counters;        // [0] next query, [1] failed queries, [2] first failed query
  unsigned long long* expansions;  // running total of expansions
};

// The serving kernel's view of a server's shared state.  Fields marked
// "host" are mapped pinned host memory written or read by the host while the
// kernel runs; the rest is device memory.
struct ServeArgs {
  const unsigned long long* tail;  // host: number of work items published
  const int* stop;                 // host: nonzero asks the kernel to return
  unsigned long long* head;        // device: number of work items claimed
  unsigned long long* tail_mirror; // device: latest tail value seen by a polling warp
  unsigned long long* last_claim;  // device: device timer at the latest claim by any warp
  const int32_t* item_kL;          // host: [slots][2] k and L of each item
  const uint8_t* qbuf;             // host: [slots][qbytes] query vectors
  int32_t* rids;                   // host: [slots][max_k]
  float* rdists;                   // host: [slots][max_k]
  int32_t* rsteps;                 // host: [slots]
  int32_t* rstatus;                // host: [slots]
  int64_t* rtimes;                 // host: [slots][2] device timer at start and end
  unsigned long long* done;        // host: [slots] item number + 1 once its results are written
  int32_t slots, qbytes, max_k;
  long long idle_ns;               // return after this long without work
};

// Launch geometry and shared-memory layout derived from the arguments.
struct SearchPlan {
  int mode;
  int nb;              // neighbour slots per lane: ceil(R/32) rounded to 1, 2 or 4
  int smem_per_warp;   // bytes of one query's state
  int warps_per_block;
  int wpq;             // warps per query: 1, or 2 / 4 (one query per block, PQ mode)
  bool pf;             // PQ mode, one warp, depth >= 2: the next-node prefetch instance
  int blocks;          // grid size (persistent)
  int tables;          // visited tables (and clear logs) the launch uses
  int64_t vis_words;   // words per visited bitset
  int vis_log_cap;
};

// Per-warp shared-memory layout (byte offsets), identical on host and device.
struct WarpSmem {
  int lut, ring, q, keys, flags, res, cand, rank, ring_key, pkeys, pflags, total;
};

// Entries of a query's pending buffer: the sorted candidates of the latest
// steps, merged into the list only when it fills (see run_query).
constexpr int kPend = 128;
constexpr int kLazyL = 2048;  // lists at least this long use the pending buffer

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

__host__ __device__ inline WarpSmem warp_smem_layout(int mode, int M, int d, int slot_bytes,
                                                     int depth, int L, int k, int nb) {
  WarpSmem s;
  int off = 0;
  s.lut = off;
  off += mode_pq(mode) ? M * 256 * 4 : 0;
  off = align_up(off, 16);
  s.ring = off;
  off += (depth + 1) * slot_bytes;
  off = align_up(off, 16);
  s.q = off;
  off += mode_f32(mode) ? d * 4 : d;
  off = align_up(off, 16);
  s.keys = off;
  off += L * 8;
  s.res = off;
  off += k * 8;
  s.cand = off;
  off += 32 * nb * 8;
  s.ring_key = off;
  off += (depth + 1) * 8;
  s.rank = off;
  off += (32 * nb > kPend ? 32 * nb : kPend) * 4;
  s.pkeys = off;
  off += kPend * 8;
  s.flags = off;
  off += align_up(L, 16);
  s.pflags = off;
  off += kPend;
  s.total = align_up(off, 128);
  return s;
}

// Plans and launches one batched search.  Returns cudaSuccess or the error.
// n_index: nodes of the index (sizes the visited tables; 0 = small index).
// wpq: warps per query requested (1, 2 or 4; more than 1 applies to PQ
// navigation only).
cudaError_t plan_search(int mode, int R, int M, int d, int slot_bytes, int depth, int L, int k,
                        int64_t nq, SearchPlan* plan, int64_t n_index = 0, int wpq = 1);
cudaError_t launch_search(const SearchArgs& a, const SearchPlan& plan, cudaStream_t stream);
// The same kernel as a cooperative launch (every block resident), for the
// kernel-grained I/O ablation (a.grid_bar set).
cudaError_t launch_search_coop(const SearchArgs& a, const SearchPlan& plan, cudaStream_t stream);
// Persistent serving kernel (a.L / a.k are the largest L / k it accepts).
cudaError_t launch_serve(const SearchArgs& a, const ServeArgs& s, const SearchPlan& plan,
                         cudaStream_t stream);

// Exact FP32 rerank of kc candidates per query down to k (kc <= 256).
cudaError_t launch_rerank(const float* vectors, int d, const float* queries, int nq, const int32_t* cand,
                          const int32_t* id_map,
                          int kc, int k, int32_t* ids, float* dists, cudaStream_t st);

// Storage-tier read probe kernel launcher.
cudaError_t launch_read_probe(const uint8_t* region, int64_t nblocks, int block_bytes, int iters,
                              unsigned long long* sink, cudaStream_t stream, float* ms_out,
                              int64_t* bytes_out);

// Brute-force exact kNN (device buffers).  engine: 0 = tensor cores where
// the data allow (uint8, d <= 128), 1 = tensor cores only, 2 = CUDA cores.
// *timed_out is set if a bounded wait of the tensor-core kernel ran out.
cudaError_t knn_exact_device(const void* base, int dtype, int64_t n, int d, const void* queries,
                             int64_t nq, int k, int32_t* ids, float* dists, cudaStream_t stream,
                             int engine, int* timed_out);

// Error reporting (thread-local message).
int set_error(int status, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* what);

}  // namespace ann
