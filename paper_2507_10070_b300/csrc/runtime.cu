// libann host runtime: the C ABI of include/ann.h.
//
// Owns the index (node-block tier in host pinned memory or HBM, PQ codes and
// codebook in HBM, exact-mode vectors/adjacency in HBM), the per-index search
// scratch (visited tables, counters, staging buffers for host calls) and the
// launches of the search kernel.  No step of the search runs on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "ann_internal.h"

namespace ann {

static thread_local std::string g_err;

int set_error(int status, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return status;
}

int cuda_error(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation)
    return set_error(ANN_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  return set_error(ANN_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace ann

using namespace ann;

// Grow-only device buffer.
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (p && cap >= bytes) return cudaSuccess;
    cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&p, bytes > 0 ? bytes : 1);
    if (e == cudaSuccess) cap = bytes;
    return e;
  }
  void release() {
    cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

struct ann_index {
  int64_t n = 0;
  int d = 0, dtype = 0, R = 0, entry = 0, M = 0, dsub = 0, tier = 0, mode = 0;
  int block_bytes = 0, ids_off = 0, deg_off = 0, adj_stride = 0;
  int slot_bytes = 0;  // bytes fetched per expansion (vector + ids, or an adjacency row)
  uint8_t* blocks_host = nullptr;  // pinned host tier
  uint8_t* blocks_dev = nullptr;   // device-visible address of the blocks
  bool blocks_in_hbm = false;
  uint8_t* codes = nullptr;
  uint32_t* cb_words = nullptr;
  float* cb_f32 = nullptr;   // float PQ codebook (precision variant)
  void* nav = nullptr;       // BF16 / FP8 navigation copies
  float nav_inv_scale = 1.f;
  int rerank_mult = 4;
  int wpq = 1;               // warps per query of ann_search / ann_search_dev (PQ mode)
  DevBuf rr_ids, rr_d;       // candidates before the exact rerank
  DevBuf grid_bar;           // kernel-grained I/O ablation: grid barrier state
  void* vectors = nullptr;
  int32_t* adj = nullptr;
  int32_t* id_map = nullptr;  // caller's id of each stored node (HBM), or null
  // scratch
  uint32_t* vis = nullptr;
  size_t vis_words = 0;
  DevBuf vis_log;
  int32_t* counters = nullptr;              // device [4]
  unsigned long long* expansions = nullptr; // device [1]
  int64_t pending_queries = 0;              // ann_search_dev calls since ann_sync
  // host-call staging (grow-only device buffers)
  cudaStream_t stream = nullptr;
  DevBuf q_stage, ids_stage, dists_stage, steps_stage, status_stage, tb_stage, te_stage;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::atomic<int> busy{0};
};

namespace {

int elt_size(int dtype) { return dtype == ANN_U8 ? 1 : 4; }

// Static split of [0, n) over the host's hardware threads.
template <class F>
void host_parallel(int64_t n, F&& fn) {
  const int th = static_cast<int>(std::min<int64_t>(std::max(1u, std::thread::hardware_concurrency()),
                                                    std::max<int64_t>(1, n / 65536)));
  if (th <= 1) {
    fn(0, n);
    return;
  }
  std::vector<std::thread> pool;
  for (int t = 0; t < th; ++t) pool.emplace_back([&, t] { fn(n * t / th, n * (t + 1) / th); });
  for (auto& x : pool) x.join();
}

void release(ann_index* ix) {
  if (!ix) return;
  if (ix->blocks_host) cudaFreeHost(ix->blocks_host);
  if (ix->blocks_in_hbm && ix->blocks_dev) cudaFree(ix->blocks_dev);
  cudaFree(ix->codes);
  cudaFree(ix->cb_words);
  cudaFree(ix->cb_f32);
  cudaFree(ix->nav);
  ix->rr_ids.release();
  ix->rr_d.release();
  ix->grid_bar.release();
  cudaFree(ix->vectors);
  cudaFree(ix->adj);
  cudaFree(ix->id_map);
  cudaFree(ix->vis);
  cudaFree(ix->counters);
  cudaFree(ix->expansions);
  for (DevBuf* b : {&ix->q_stage, &ix->ids_stage, &ix->dists_stage, &ix->steps_stage,
                    &ix->status_stage, &ix->tb_stage, &ix->te_stage, &ix->vis_log})
    b->release();
  if (ix->ev0) cudaEventDestroy(ix->ev0);
  if (ix->ev1) cudaEventDestroy(ix->ev1);
  if (ix->stream) cudaStreamDestroy(ix->stream);
  delete ix;
}

int validate_desc(const ann_graph_desc* g) {
  if (!g) return set_error(ANN_EINVAL, "ann_load_graph: desc is NULL");
  if (g->n < 1 || g->n >= INT32_MAX) return set_error(ANN_EINVAL, "n=%lld out of range", (long long)g->n);
  if (g->d < 4 || g->d > kMaxD || g->d % 4) return set_error(ANN_EINVAL, "d=%d must be a multiple of 4 in [4,%d]", g->d, kMaxD);
  if (g->dtype != ANN_U8 && g->dtype != ANN_F32) return set_error(ANN_EINVAL, "unknown dtype %d", g->dtype);
  if (g->R < 1 || g->R > kMaxR) return set_error(ANN_EINVAL, "R=%d out of range [1,%d]", g->R, kMaxR);
  if (g->entry < 0 || g->entry >= g->n) return set_error(ANN_EINVAL, "entry %d out of range", g->entry);
  if (!g->vectors || !g->adj) return set_error(ANN_EINVAL, "vectors and adj are required");
  if (g->tier != ANN_TIER_HOST_PINNED && g->tier != ANN_TIER_HBM) return set_error(ANN_EINVAL, "unknown tier %d", g->tier);
  if (g->M < 0) return set_error(ANN_EINVAL, "M=%d < 0", g->M);
  if (g->nav < ANN_NAV_AUTO || g->nav > ANN_NAV_FP8) return set_error(ANN_EINVAL, "unknown nav %d", g->nav);
  if (g->rerank_mult < 0 || g->rerank_mult > 64) return set_error(ANN_EINVAL, "rerank_mult %d out of [0,64]", g->rerank_mult);
  if (g->nav != ANN_NAV_AUTO) {
    if (g->dtype != ANN_F32 || g->M != 0 || g->tier != ANN_TIER_HBM)
      return set_error(ANN_EINVAL, "BF16 / FP8 navigation needs float32 data, M == 0 and ANN_TIER_HBM");
    if (g->nav == ANN_NAV_FP8 && !(g->nav_scale > 0.f)) return set_error(ANN_EINVAL, "FP8 navigation needs nav_scale > 0");
  }
  if (g->M > 0 && g->dtype == ANN_F32) {
    if (g->M % 16 || g->M > kMaxM || g->d % g->M)
      return set_error(ANN_EINVAL, "float PQ needs M %% 16 == 0, M <= %d, d %% M == 0 (d=%d, M=%d)", kMaxM, g->d, g->M);
    if (!g->codebook || !g->codes) return set_error(ANN_EINVAL, "PQ navigation needs codebook and codes");
    if (g->tier != ANN_TIER_HBM) return set_error(ANN_EINVAL, "float PQ navigation keeps vectors in HBM: use ANN_TIER_HBM");
  } else if (g->M > 0) {
    if (g->dtype != ANN_U8) return set_error(ANN_EINVAL, "PQ navigation needs uint8 data");
    if (g->M % 16 || g->M > kMaxM || g->d % g->M || (g->d / g->M) % 4)
      return set_error(ANN_EINVAL, "PQ needs M %% 16 == 0, M <= %d, d %% M == 0, (d/M) %% 4 == 0 (d=%d, M=%d)", kMaxM, g->d, g->M);
    if (!g->codebook || !g->codes) return set_error(ANN_EINVAL, "PQ navigation needs codebook and codes");
    const int64_t ncb = (int64_t)g->M * 256 * (g->d / g->M);
    for (int64_t i = 0; i < ncb; ++i) {
      const float v = g->codebook[i];
      if (!(v >= 0.f && v <= 255.f) || v != std::floor(v))
        return set_error(ANN_EINVAL, "codebook value %g at %lld is not an integer in [0,255]", v, (long long)i);
    }
  } else if (g->tier != ANN_TIER_HBM) {
    return set_error(ANN_EINVAL, "exact navigation keeps vectors in HBM: use ANN_TIER_HBM");
  }
  std::atomic<int64_t> bad{-1};
  host_parallel(g->n * g->R, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) {
      const int32_t v = g->adj[i];
      if (v < -1 || v >= g->n) {
        int64_t expect = -1;
        bad.compare_exchange_strong(expect, i);
        return;
      }
    }
  });
  if (bad.load() >= 0)
    return set_error(ANN_EINVAL, "adjacency id %d at row %lld out of range", g->adj[bad.load()],
                     (long long)(bad.load() / g->R));
  return ANN_OK;
}

}  // namespace

extern "C" {

const char* ann_last_error(void) { return g_err.c_str(); }

const char* ann_version(void) { return "libann 0.1 (sm_103a)"; }

int64_t ann_index_block_bytes(const ann_index* ix) { return ix ? ix->block_bytes : 0; }
int64_t ann_index_size(const ann_index* ix) { return ix ? ix->n : 0; }

int ann_set_warps_per_query(ann_index* ix, int32_t w) {
  if (!ix) return set_error(ANN_EINVAL, "index is NULL");
  if (w != 1 && w != 2 && w != 4) return set_error(ANN_EINVAL, "warps per query must be 1, 2 or 4 (got %d)", w);
  if (w > 1 && ix->mode != kModePqU8)
    return set_error(ANN_EINVAL, "a warp group per query needs PQ navigation on uint8 data");
  if (ix->busy.load()) return set_error(ANN_EBUSY, "the index is in use by a search");
  ix->wpq = w;
  return ANN_OK;
}

void ann_free(ann_index* ix) { release(ix); }

int ann_load_graph(ann_index** out, const ann_graph_desc* g) {
  if (!out) return set_error(ANN_EINVAL, "ann_load_graph: out is NULL");
  *out = nullptr;
  int rc = validate_desc(g);
  if (rc != ANN_OK) return rc;
  ann_index* ix = new ann_index();
  ix->n = g->n;
  ix->d = g->d;
  ix->dtype = g->dtype;
  ix->R = g->R;
  ix->entry = g->entry;
  ix->M = g->M;
  ix->dsub = g->M > 0 ? g->d / g->M : 0;
  ix->tier = g->tier;
  if (g->M > 0) ix->mode = g->dtype == ANN_U8 ? kModePqU8 : kModePqF32;
  else if (g->nav == ANN_NAV_BF16) ix->mode = kModeBF16;
  else if (g->nav == ANN_NAV_FP8) ix->mode = kModeFP8;
  else ix->mode = g->dtype == ANN_U8 ? kModeExactU8 : kModeExactF32;
  ix->rerank_mult = g->rerank_mult > 0 ? g->rerank_mult : 4;
  const int64_t n = g->n;
  const int R = g->R, d = g->d;
  cudaError_t e;
#define ANN_TRY(call, what)                   \
  do {                                        \
    e = (call);                               \
    if (e != cudaSuccess) {                   \
      release(ix);                            \
      return cuda_error(e, what);             \
    }                                         \
  } while (0)
  ANN_TRY(cudaStreamCreateWithFlags(&ix->stream, cudaStreamNonBlocking), "cudaStreamCreate");
  ANN_TRY(cudaEventCreate(&ix->ev0), "cudaEventCreate");
  ANN_TRY(cudaEventCreate(&ix->ev1), "cudaEventCreate");
  ANN_TRY(cudaMalloc(&ix->counters, 4 * sizeof(int32_t)), "cudaMalloc counters");
  ANN_TRY(cudaMalloc(&ix->expansions, sizeof(unsigned long long)), "cudaMalloc counters");
  {
    const int32_t init[4] = {0, 0, INT32_MAX, 0};
    ANN_TRY(cudaMemcpy(ix->counters, init, sizeof(init), cudaMemcpyHostToDevice), "upload counters");
    ANN_TRY(cudaMemset(ix->expansions, 0, sizeof(unsigned long long)), "cudaMemset");
  }
  if (g->id_map) {
    ANN_TRY(cudaMalloc(&ix->id_map, (size_t)n * 4), "cudaMalloc id map");
    ANN_TRY(cudaMemcpy(ix->id_map, g->id_map, (size_t)n * 4, cudaMemcpyHostToDevice), "upload id map");
  }
  if (ix->mode == kModePqU8) {
    // Node block: [vector d bytes][R int32 ids][uint32 degree][zero pad to 128 B]
    ix->ids_off = d;
    ix->deg_off = d + 4 * R;
    ix->block_bytes = align_up(d + 4 * R + 4, 128);
    ix->slot_bytes = align_up(d + 4 * R, 16);
    const size_t total = (size_t)n * ix->block_bytes;
    std::vector<uint8_t> tmp;
    uint8_t* dst;
    if (g->tier == ANN_TIER_HOST_PINNED) {
      ANN_TRY(cudaHostAlloc(reinterpret_cast<void**>(&ix->blocks_host), total,
                            cudaHostAllocMapped | cudaHostAllocPortable), "cudaHostAlloc node blocks");
      dst = ix->blocks_host;
    } else {
      tmp.resize(total);
      dst = tmp.data();
    }
    const uint8_t* vec = static_cast<const uint8_t*>(g->vectors);
    host_parallel(n, [&](int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i) {
        uint8_t* b = dst + (size_t)i * ix->block_bytes;
        std::memset(b, 0, ix->block_bytes);
        std::memcpy(b, vec + (size_t)i * d, d);
        int32_t* ids = reinterpret_cast<int32_t*>(b + ix->ids_off);
        uint32_t deg = 0;
        for (int j = 0; j < R; ++j) {
          const int32_t v = g->adj[(size_t)i * R + j];
          if (v < 0) break;
          ids[deg++] = v;
        }
        for (int j = deg; j < R; ++j) ids[j] = -1;
        std::memcpy(b + ix->deg_off, &deg, 4);
      }
    });
    if (g->tier == ANN_TIER_HOST_PINNED) {
      ANN_TRY(cudaHostGetDevicePointer(reinterpret_cast<void**>(&ix->blocks_dev), ix->blocks_host, 0),
              "cudaHostGetDevicePointer");
    } else {
      ANN_TRY(cudaMalloc(&ix->blocks_dev, total), "cudaMalloc node blocks");
      ix->blocks_in_hbm = true;
      ANN_TRY(cudaMemcpy(ix->blocks_dev, tmp.data(), total, cudaMemcpyHostToDevice), "upload node blocks");
    }
    ANN_TRY(cudaMalloc(&ix->codes, (size_t)n * g->M), "cudaMalloc codes");
    ANN_TRY(cudaMemcpy(ix->codes, g->codes, (size_t)n * g->M, cudaMemcpyHostToDevice), "upload codes");
    const int wps = ix->dsub / 4;
    std::vector<uint32_t> words((size_t)g->M * 256 * wps);
    for (int m = 0; m < g->M; ++m)
      for (int c = 0; c < 256; ++c)
        for (int w = 0; w < wps; ++w) {
          uint32_t word = 0;
          for (int b = 0; b < 4; ++b) {
            const float v = g->codebook[((size_t)m * 256 + c) * ix->dsub + 4 * w + b];
            word |= (uint32_t)(uint8_t)v << (8 * b);
          }
          words[((size_t)m * 256 + c) * wps + w] = word;
        }
    ANN_TRY(cudaMalloc(&ix->cb_words, words.size() * 4), "cudaMalloc codebook");
    ANN_TRY(cudaMemcpy(ix->cb_words, words.data(), words.size() * 4, cudaMemcpyHostToDevice), "upload codebook");
  } else {
    const size_t vbytes = (size_t)n * d * elt_size(g->dtype);
    ANN_TRY(cudaMalloc(&ix->vectors, vbytes), "cudaMalloc vectors");
    ANN_TRY(cudaMemcpy(ix->vectors, g->vectors, vbytes, cudaMemcpyHostToDevice), "upload vectors");
    ix->adj_stride = align_up(R, 4);
    ix->block_bytes = ix->adj_stride * 4;
    ix->slot_bytes = ix->block_bytes;
    std::vector<int32_t> rows((size_t)n * ix->adj_stride, -1);
    host_parallel(n, [&](int64_t lo, int64_t hi) {
      for (int64_t i = lo; i < hi; ++i)
        for (int j = 0; j < R; ++j) {
          const int32_t v = g->adj[(size_t)i * R + j];
          if (v < 0) break;
          rows[(size_t)i * ix->adj_stride + j] = v;
        }
    });
    ANN_TRY(cudaMalloc(&ix->adj, rows.size() * 4), "cudaMalloc adjacency");
    ANN_TRY(cudaMemcpy(ix->adj, rows.data(), rows.size() * 4, cudaMemcpyHostToDevice), "upload adjacency");
    const float* fv = static_cast<const float*>(g->vectors);
    if (ix->mode == kModeBF16) {
      std::vector<uint16_t> b((size_t)n * d);
      ann_encode_bf16(fv, (int64_t)b.size(), b.data());
      ANN_TRY(cudaMalloc(&ix->nav, b.size() * 2), "cudaMalloc navigation copy");
      ANN_TRY(cudaMemcpy(ix->nav, b.data(), b.size() * 2, cudaMemcpyHostToDevice), "upload navigation copy");
    } else if (ix->mode == kModeFP8) {
      std::vector<uint8_t> b((size_t)n * d);
      ann_encode_fp8e4m3(fv, (int64_t)b.size(), g->nav_scale, b.data());
      ix->nav_inv_scale = 1.0f / g->nav_scale;
      ANN_TRY(cudaMalloc(&ix->nav, b.size()), "cudaMalloc navigation copy");
      ANN_TRY(cudaMemcpy(ix->nav, b.data(), b.size(), cudaMemcpyHostToDevice), "upload navigation copy");
    } else if (ix->mode == kModePqF32) {
      const size_t ncb = (size_t)g->M * 256 * (d / g->M);
      ANN_TRY(cudaMalloc(&ix->cb_f32, ncb * 4), "cudaMalloc codebook");
      ANN_TRY(cudaMemcpy(ix->cb_f32, g->codebook, ncb * 4, cudaMemcpyHostToDevice), "upload codebook");
      ANN_TRY(cudaMalloc(&ix->codes, (size_t)n * g->M), "cudaMalloc codes");
      ANN_TRY(cudaMemcpy(ix->codes, g->codes, (size_t)n * g->M, cudaMemcpyHostToDevice), "upload codes");
    }
  }
#undef ANN_TRY
  *out = ix;
  return ANN_OK;
}

}  // extern "C"

namespace {

int validate_search(const ann_index* ix, const void* q, int64_t nq, int k, int L, int depth,
                    const void* ids, const void* dists) {
  if (!ix) return set_error(ANN_EINVAL, "index is NULL");
  if (nq < 0 || nq >= INT32_MAX) return set_error(ANN_EINVAL, "nq=%lld out of range", (long long)nq);
  if (k < 1 || L < k || L > kMaxL) return set_error(ANN_EINVAL, "need 1 <= k <= L <= %d (k=%d, L=%d)", kMaxL, k, L);
  if (k > 256) return set_error(ANN_EINVAL, "k=%d > 256", k);
  if (depth < 0 || depth > kMaxDepth) return set_error(ANN_EINVAL, "depth=%d out of range [0,%d]", depth, kMaxDepth);
  if (nq > 0 && (!q || !ids || !dists)) return set_error(ANN_EINVAL, "queries, ids and dists are required");
  return ANN_OK;
}

// Enqueue one search of nq device-resident queries on `st`.
bool rerank_mode(int mode) { return mode == kModeBF16 || mode == kModeFP8 || mode == kModePqF32; }

// Device-visible buffers of the CPU-agent I/O ablation (see SearchArgs).
struct AgentBufs {
  AgentReq* req;
  const unsigned* done;
  const uint8_t* stage;
  unsigned* seq;
  int64_t wait_ns;
};

int enqueue_search(ann_index* ix, const void* q, int64_t nq, int k, int L, int depth, int32_t* ids,
                   float* dists, const ann_trace* tr, cudaStream_t st, bool timed,
                   bool kernel_grained = false, const AgentBufs* agent = nullptr) {
  if (nq == 0) return ANN_OK;
  const int slot_bytes = ix->slot_bytes;
  // precision variants: keep the top rerank_mult*k expanded by navigation
  // distance, then rerank them exactly in FP32
  const bool rr = rerank_mode(ix->mode);
  const int k_out = k;
  int32_t* ids_out = ids;
  float* dists_out = dists;
  if (rr) {
    k = std::min(L, std::min(512, std::max(k, ix->rerank_mult * k)));
    cudaError_t e1 = ix->rr_ids.ensure((size_t)nq * k * 4);
    if (e1 == cudaSuccess) e1 = ix->rr_d.ensure((size_t)nq * k * 4);
    if (e1 != cudaSuccess) return cuda_error(e1, "rerank buffers");
    ids = static_cast<int32_t*>(ix->rr_ids.p);
    dists = static_cast<float*>(ix->rr_d.p);
  }
  SearchPlan plan;
  cudaError_t e = plan_search(ix->mode, ix->R, ix->M, ix->d, slot_bytes, depth, L, k, nq, &plan, ix->n,
                              (kernel_grained || agent) ? 1 : ix->wpq);
  if (e != cudaSuccess) return cuda_error(e, "plan search");
  const size_t want = (size_t)plan.tables * (size_t)plan.vis_words;
  if (want > ix->vis_words) {
    // tables must start all-zero; the kernel clears after each query
    cudaError_t s = cudaStreamSynchronize(st);
    if (s != cudaSuccess) return cuda_error(s, "sync before scratch growth");
    cudaFree(ix->vis);
    ix->vis = nullptr;
    ix->vis_words = 0;
    e = cudaMalloc(&ix->vis, want * 4);
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc visited tables");
    e = cudaMemset(ix->vis, 0, want * 4);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemset visited tables");
    ix->vis_words = want;
  }
  const size_t log_bytes = (size_t)plan.tables * plan.vis_log_cap * 4;
  if (log_bytes > ix->vis_log.cap) {
    cudaError_t s = cudaStreamSynchronize(st);
    if (s != cudaSuccess) return cuda_error(s, "sync before scratch growth");
    e = ix->vis_log.ensure(log_bytes);
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc visited log");
  }
  SearchArgs a{};
  a.n = (int32_t)ix->n;
  a.d = ix->d;
  a.R = ix->R;
  a.entry = ix->entry;
  a.M = ix->M;
  a.dsub = ix->dsub;
  a.blocks = ix->blocks_dev;
  a.block_bytes = ix->block_bytes;
  a.ids_off = ix->ids_off;
  a.deg_off = ix->deg_off;
  a.slot_bytes = ix->slot_bytes;
  a.codes = ix->codes;
  a.cb_words = ix->cb_words;
  a.cb_f32 = ix->cb_f32;
  a.nav = ix->nav;
  a.nav_inv_scale = ix->nav_inv_scale;
  a.vectors = ix->vectors;
  a.adj = ix->adj;
  a.adj_stride = ix->adj_stride;
  a.id_map = rr ? nullptr : ix->id_map;  // with a rerank, the rerank maps the final ids
  a.grid_bar = nullptr;
  if (kernel_grained) {
    e = ix->grid_bar.ensure(4 * sizeof(unsigned));
    if (e != cudaSuccess) return cuda_error(e, "grid barrier state");
    const unsigned warps = static_cast<unsigned>(plan.blocks * plan.warps_per_block);
    // Test hook for the bounded waits: ANN_TEST_STALL_ROUNDS=1 presets the
    // arrival count past the last arrival, so no round can complete and
    // every warp must give up (the call then reports ANN_ETIMEOUT).
    const char* stall = std::getenv("ANN_TEST_STALL_ROUNDS");
    const unsigned arrivals = (stall && stall[0] == '1') ? warps : 0u;
    const unsigned init[4] = {arrivals, 0u, warps, 0u};
    e = cudaMemcpyAsync(ix->grid_bar.p, init, sizeof(init), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_error(e, "grid barrier state");
    a.grid_bar = static_cast<unsigned*>(ix->grid_bar.p);
  }
  if (agent) {
    a.agent_req = agent->req;
    a.agent_done = agent->done;
    a.agent_stage = agent->stage;
    a.agent_seq = agent->seq;
    a.agent_wait_ns = agent->wait_ns;
  }
  a.queries = q;
  a.nq = (int32_t)nq;
  a.k = k;
  a.L = L;
  a.depth = depth;
  a.ids = ids;
  a.dists = dists;
  a.steps = tr ? tr->steps : nullptr;
  a.status = tr ? tr->status : nullptr;
  a.t_begin = tr ? tr->t_begin : nullptr;
  a.t_end = tr ? tr->t_end : nullptr;
  a.vis = ix->vis;
  a.vis_words = plan.vis_words;
  a.vis_log = static_cast<uint32_t*>(ix->vis_log.p);
  a.vis_log_cap = plan.vis_log_cap;
  a.counters = ix->counters;
  a.expansions = ix->expansions;
  e = cudaMemsetAsync(ix->counters, 0, sizeof(int32_t), st);  // next-query counter
  if (e != cudaSuccess) return cuda_error(e, "reset work counter");
  if (timed) cudaEventRecord(ix->ev0, st);
  e = kernel_grained ? launch_search_coop(a, plan, st) : launch_search(a, plan, st);
  if (e != cudaSuccess) return cuda_error(e, "search kernel launch");
  if (rr) {
    e = launch_rerank(static_cast<const float*>(ix->vectors), ix->d, static_cast<const float*>(q), (int)nq,
                      ids, ix->id_map, k, k_out, ids_out, dists_out, st);
    if (e != cudaSuccess) return cuda_error(e, "rerank kernel launch");
  }
  if (timed) cudaEventRecord(ix->ev1, st);
  return ANN_OK;
}

// Read and reset the device-side failure counters and expansion total.
int collect(ann_index* ix, cudaStream_t st, int64_t queries, ann_search_stats* stats, bool timed) {
  int32_t c[4];
  unsigned long long ex = 0;
  cudaError_t e = cudaMemcpyAsync(c, ix->counters, sizeof(c), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ex, ix->expansions, sizeof(ex), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "search");
  const int32_t init[4] = {0, 0, INT32_MAX, 0};
  e = cudaMemcpyAsync(ix->counters, init, sizeof(init), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ix->expansions, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "reset counters");
  float ms = 0.f;
  if (timed) cudaEventElapsedTime(&ms, ix->ev0, ix->ev1);
  if (stats) {
    stats->queries = queries;
    stats->expansions = (int64_t)ex;
    stats->bytes_per_expansion = ix->slot_bytes;
    stats->n_failed = c[1];
    stats->first_failed = c[1] > 0 ? c[2] : -1;
    stats->kernel_ms = ms;
  }
  if (c[3] != 0)
    return set_error(ANN_ETIMEOUT, "a kernel-grained round barrier timed out (%d queries failed)", c[1]);
  if (c[1] > 0)
    return set_error(ANN_ENOMEM, "%d queries stopped early (first: query %d)", c[1], c[2]);
  return ANN_OK;
}

struct BusyGuard {
  ann_index* ix;
  bool ok;
  explicit BusyGuard(ann_index* i) : ix(i) {
    int z = 0;
    ok = ix->busy.compare_exchange_strong(z, 1);
  }
  ~BusyGuard() {
    if (ok) ix->busy.store(0);
  }
};

}  // namespace

extern "C" {

int ann_search(ann_index* ix, const void* queries, int64_t nq, int32_t k, int32_t L, int32_t depth,
               int32_t* ids, float* dists, const ann_trace* trace, ann_search_stats* stats) {
  int rc = validate_search(ix, queries, nq, k, L, depth, ids, dists);
  if (rc != ANN_OK) return rc;
  BusyGuard guard(ix);
  if (!guard.ok) return set_error(ANN_EBUSY, "index is busy with another search");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (nq == 0) return ANN_OK;
  cudaStream_t st = ix->stream;
  const size_t qbytes = (size_t)nq * ix->d * elt_size(ix->dtype);  // float32 for the precision variants
  cudaError_t e = ix->q_stage.ensure(qbytes);
  if (e == cudaSuccess) e = ix->ids_stage.ensure((size_t)nq * k * 4);
  if (e == cudaSuccess) e = ix->dists_stage.ensure((size_t)nq * k * 4);
  if (e == cudaSuccess && trace) {
    e = ix->steps_stage.ensure((size_t)nq * 4);
    if (e == cudaSuccess) e = ix->status_stage.ensure((size_t)nq * 4);
    if (e == cudaSuccess) e = ix->tb_stage.ensure((size_t)nq * 8);
    if (e == cudaSuccess) e = ix->te_stage.ensure((size_t)nq * 8);
  }
  if (e != cudaSuccess) return cuda_error(e, "staging buffers");
  e = cudaMemcpyAsync(ix->q_stage.p, queries, qbytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_error(e, "copy queries");
  ann_trace dtr{};
  if (trace) {
    dtr.steps = trace->steps ? static_cast<int32_t*>(ix->steps_stage.p) : nullptr;
    dtr.status = trace->status ? static_cast<int32_t*>(ix->status_stage.p) : nullptr;
    dtr.t_begin = trace->t_begin ? static_cast<int64_t*>(ix->tb_stage.p) : nullptr;
    dtr.t_end = trace->t_end ? static_cast<int64_t*>(ix->te_stage.p) : nullptr;
  }
  int32_t* ids_d = static_cast<int32_t*>(ix->ids_stage.p);
  float* dists_d = static_cast<float*>(ix->dists_stage.p);
  rc = enqueue_search(ix, ix->q_stage.p, nq, k, L, depth, ids_d, dists_d, trace ? &dtr : nullptr,
                      st, true);
  if (rc != ANN_OK) return rc;
  e = cudaMemcpyAsync(ids, ids_d, (size_t)nq * k * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dists, dists_d, (size_t)nq * k * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && trace) {
    if (trace->steps) e = cudaMemcpyAsync(trace->steps, dtr.steps, nq * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && trace->status) e = cudaMemcpyAsync(trace->status, dtr.status, nq * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && trace->t_begin) e = cudaMemcpyAsync(trace->t_begin, dtr.t_begin, nq * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && trace->t_end) e = cudaMemcpyAsync(trace->t_end, dtr.t_end, nq * 8, cudaMemcpyDeviceToHost, st);
  }
  if (e != cudaSuccess) return cuda_error(e, "copy results");
  return collect(ix, st, nq, stats, true);
}

int ann_search_dev(ann_index* ix, const void* queries, int64_t nq, int32_t k, int32_t L, int32_t depth,
                   int32_t* ids, float* dists, const ann_trace* trace, void* stream) {
  int rc = validate_search(ix, queries, nq, k, L, depth, ids, dists);
  if (rc != ANN_OK) return rc;
  if (reinterpret_cast<uintptr_t>(queries) % 16)
    return set_error(ANN_EINVAL, "queries must be 16-byte aligned");
  BusyGuard guard(ix);
  if (!guard.ok) return set_error(ANN_EBUSY, "index is busy with another search");
  rc = enqueue_search(ix, queries, nq, k, L, depth, ids, dists, trace,
                      static_cast<cudaStream_t>(stream), false);
  if (rc == ANN_OK) ix->pending_queries += nq;
  return rc;
}

int ann_search_dev_kernel_grained(ann_index* ix, const void* queries, int64_t nq, int32_t k, int32_t L,
                                  int32_t depth, int32_t* ids, float* dists, const ann_trace* trace,
                                  void* stream) {
  int rc = validate_search(ix, queries, nq, k, L, depth, ids, dists);
  if (rc != ANN_OK) return rc;
  if (reinterpret_cast<uintptr_t>(queries) % 16)
    return set_error(ANN_EINVAL, "queries must be 16-byte aligned");
  BusyGuard guard(ix);
  if (!guard.ok) return set_error(ANN_EBUSY, "index is busy with another search");
  rc = enqueue_search(ix, queries, nq, k, L, depth, ids, dists, trace,
                      static_cast<cudaStream_t>(stream), false, true);
  if (rc == ANN_OK) ix->pending_queries += nq;
  return rc;
}

// One host agent thread: serve the request entries [lo, hi) until *stop.
// A new sequence number in an entry is a request: copy the node's block
// into the entry's staging slot, then publish the number in `done` (release
// order: the GPU that reads the number reads the bytes after it).
void agent_serve(AgentReq* req, unsigned* done, uint8_t* stage, const uint8_t* blocks, int block_bytes,
                 int slot_bytes, int64_t n, size_t lo, size_t hi, const std::atomic<bool>* stop) {
  std::vector<unsigned> last(hi - lo, 0u);
  while (!stop->load(std::memory_order_acquire)) {
    bool any = false;
    for (size_t e = lo; e < hi; ++e) {
      const unsigned sq = __atomic_load_n(&req[e].seq, __ATOMIC_ACQUIRE);
      if (sq == last[e - lo]) continue;
      const int32_t node = __atomic_load_n(&req[e].node, __ATOMIC_RELAXED);
      if (node >= 0 && node < n)
        std::memcpy(stage + e * slot_bytes, blocks + static_cast<size_t>(node) * block_bytes, slot_bytes);
      __atomic_store_n(&done[e], sq, __ATOMIC_RELEASE);
      last[e - lo] = sq;
      any = true;
    }
    if (!any) std::this_thread::yield();
  }
}

int ann_search_cpu_agent(ann_index* ix, const void* queries, int64_t nq, int32_t k, int32_t L, int32_t depth,
                         int32_t agent_threads, int64_t wait_us, int32_t* ids, float* dists,
                         ann_search_stats* stats, double* seconds) {
  int rc = validate_search(ix, queries, nq, k, L, depth, ids, dists);
  if (rc != ANN_OK) return rc;
  if (ix->mode != kModePqU8 || ix->blocks_in_hbm || !ix->blocks_host)
    return set_error(ANN_EINVAL, "cpu agent: needs a PQ index with its node blocks in host pinned memory");
  if (agent_threads < 0 || agent_threads > 64 || wait_us < 1 || wait_us > 60000000)
    return set_error(ANN_EINVAL, "cpu agent: need 0 <= agent_threads <= 64 and 1 <= wait_us <= 6e7");
  BusyGuard guard(ix);
  if (!guard.ok) return set_error(ANN_EBUSY, "index is busy with another search");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (seconds) *seconds = 0.0;
  if (nq == 0) return ANN_OK;
  cudaStream_t st = ix->stream;
  SearchPlan plan;
  cudaError_t e = plan_search(ix->mode, ix->R, ix->M, ix->d, ix->slot_bytes, depth, L, k, nq, &plan, ix->n, 1);
  if (e != cudaSuccess) return cuda_error(e, "plan search");
  const size_t entries = static_cast<size_t>(plan.blocks) * plan.warps_per_block * (depth + 1);
  AgentReq* req = nullptr;
  unsigned* done = nullptr;
  uint8_t* stage = nullptr;
  unsigned* seq = nullptr;
  auto free_all = [&] {
    if (req) cudaFreeHost(req);
    if (done) cudaFreeHost(done);
    if (stage) cudaFreeHost(stage);
    cudaFree(seq);
  };
  e = cudaHostAlloc(reinterpret_cast<void**>(&req), entries * sizeof(AgentReq), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&done), entries * 4, cudaHostAllocMapped);
  if (e == cudaSuccess)
    e = cudaHostAlloc(reinterpret_cast<void**>(&stage), entries * ix->slot_bytes, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaMalloc(&seq, entries * 4);
  if (e == cudaSuccess) e = cudaMemset(seq, 0, entries * 4);
  const size_t qbytes = (size_t)nq * ix->d;
  if (e == cudaSuccess) e = ix->q_stage.ensure(qbytes);
  if (e == cudaSuccess) e = ix->ids_stage.ensure((size_t)nq * k * 4);
  if (e == cudaSuccess) e = ix->dists_stage.ensure((size_t)nq * k * 4);
  if (e != cudaSuccess) {
    free_all();
    return cuda_error(e, "cpu agent buffers");
  }
  std::memset(req, 0, entries * sizeof(AgentReq));
  std::memset(done, 0, entries * 4);
  AgentBufs ab;
  void* dp = nullptr;
  e = cudaHostGetDevicePointer(&dp, req, 0);
  ab.req = static_cast<AgentReq*>(dp);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&dp, done, 0);
  ab.done = static_cast<const unsigned*>(dp);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&dp, stage, 0);
  ab.stage = static_cast<const uint8_t*>(dp);
  ab.seq = seq;
  ab.wait_ns = wait_us * 1000;
  if (e == cudaSuccess) e = cudaMemcpyAsync(ix->q_stage.p, queries, qbytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    free_all();
    return cuda_error(e, "cpu agent set-up");
  }
  std::atomic<bool> stop{false};
  std::vector<std::thread> agents;
  for (int t = 0; t < agent_threads; ++t)
    agents.emplace_back(agent_serve, req, done, stage, ix->blocks_host, ix->block_bytes, ix->slot_bytes, ix->n,
                        entries * t / agent_threads, entries * (t + 1) / agent_threads, &stop);
  int32_t* ids_d = static_cast<int32_t*>(ix->ids_stage.p);
  float* dists_d = static_cast<float*>(ix->dists_stage.p);
  const auto t0 = std::chrono::steady_clock::now();
  rc = enqueue_search(ix, ix->q_stage.p, nq, k, L, depth, ids_d, dists_d, nullptr, st, true, false, &ab);
  if (rc == ANN_OK) {
    e = cudaStreamSynchronize(st);  // the agents serve requests until the kernel is done
    if (seconds) *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  stop.store(true, std::memory_order_release);
  for (auto& t : agents) t.join();
  if (rc == ANN_OK && e != cudaSuccess) rc = cuda_error(e, "cpu agent search");
  if (rc == ANN_OK) {
    e = cudaMemcpyAsync(ids, ids_d, (size_t)nq * k * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dists, dists_d, (size_t)nq * k * 4, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) rc = cuda_error(e, "copy results");
  }
  if (rc == ANN_OK) {
    ann_search_stats local{};
    ann_search_stats* sp = stats ? stats : &local;
    rc = collect(ix, st, nq, sp, true);
    // the one way a query stops early here: a wait for the agent ran out
    if (rc == ANN_ENOMEM)
      rc = set_error(ANN_ETIMEOUT, "cpu agent: a wait for the host agent ran out (%lld queries failed)",
                     (long long)sp->n_failed);
  } else {
    cudaStreamSynchronize(st);
  }
  free_all();
  return rc;
}

int ann_sync(ann_index* ix, void* stream, ann_search_stats* stats) {
  if (!ix) return set_error(ANN_EINVAL, "index is NULL");
  BusyGuard guard(ix);
  if (!guard.ok) return set_error(ANN_EBUSY, "index is busy with another search");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  const int64_t q = ix->pending_queries;
  ix->pending_queries = 0;
  return collect(ix, static_cast<cudaStream_t>(stream), q, stats, false);
}

int ann_knn_exact_ex(const void* base, int32_t dtype, int64_t n, int32_t d, const void* queries,
                     int64_t nq, int32_t k, int32_t engine, int32_t* ids, float* dists, float* kernel_ms) {
  if (!base || !queries || !ids || !dists) return set_error(ANN_EINVAL, "NULL buffer");
  if (dtype != ANN_U8 && dtype != ANN_F32) return set_error(ANN_EINVAL, "unknown dtype");
  if (n < 1 || n >= (1ll << 31) || nq < 0 || k < 1 || k > 128 || d < 4 || d % 4 ||
      d > (dtype == ANN_U8 ? 512 : 256))
    return set_error(ANN_EINVAL, "knn: bad sizes (n=%lld d=%d k=%d)", (long long)n, d, k);
  if (engine < ANN_KNN_AUTO || engine > ANN_KNN_CUDA_CORES)
    return set_error(ANN_EINVAL, "knn: unknown engine %d", engine);
  if (engine == ANN_KNN_TENSOR_CORES && (dtype != ANN_U8 || d > 128))
    return set_error(ANN_EINVAL, "knn: the tensor-core engine needs uint8 data with d <= 128 (d=%d)", d);
  if (kernel_ms) *kernel_ms = 0.f;
  if (nq == 0) return ANN_OK;
  const size_t es = elt_size(dtype);
  void *db = nullptr, *dq = nullptr;
  int32_t* di = nullptr;
  float* dd = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int timed_out = 0;
  cudaError_t e = cudaMalloc(&db, (size_t)n * d * es);
  if (e == cudaSuccess) e = cudaMalloc(&dq, (size_t)nq * d * es);
  if (e == cudaSuccess) e = cudaMalloc(&di, (size_t)nq * k * 4);
  if (e == cudaSuccess) e = cudaMalloc(&dd, (size_t)nq * k * 4);
  if (e == cudaSuccess) e = cudaEventCreate(&ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&ev1);
  if (e == cudaSuccess) e = cudaMemcpy(db, base, (size_t)n * d * es, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dq, queries, (size_t)nq * d * es, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaEventRecord(ev0, 0);
  if (e == cudaSuccess) e = knn_exact_device(db, dtype, n, d, dq, nq, k, di, dd, 0, engine, &timed_out);
  if (e == cudaSuccess) e = cudaEventRecord(ev1, 0);
  if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
  if (e == cudaSuccess && kernel_ms) e = cudaEventElapsedTime(kernel_ms, ev0, ev1);
  if (e == cudaSuccess) e = cudaMemcpy(ids, di, (size_t)nq * k * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(dists, dd, (size_t)nq * k * 4, cudaMemcpyDeviceToHost);
  cudaFree(db);
  cudaFree(dq);
  cudaFree(di);
  cudaFree(dd);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (e != cudaSuccess) return cuda_error(e, "knn");
  if (timed_out) return set_error(ANN_ETIMEOUT, "knn: a bounded wait of the tensor-core kernel ran out");
  return ANN_OK;
}

int ann_knn_exact(const void* base, int32_t dtype, int64_t n, int32_t d, const void* queries,
                  int64_t nq, int32_t k, int32_t* ids, float* dists) {
  return ann_knn_exact_ex(base, dtype, n, d, queries, nq, k, ANN_KNN_AUTO, ids, dists, nullptr);
}

int ann_probe_read_bandwidth(int64_t bytes, int32_t block_bytes, int32_t tier, int32_t iters,
                             double* gbps_out) {
  if (!gbps_out || bytes < block_bytes || block_bytes < 16 || block_bytes % 16 || block_bytes > 4096 ||
      iters < 1 || (tier != ANN_TIER_HOST_PINNED && tier != ANN_TIER_HBM))
    return set_error(ANN_EINVAL, "probe: bad arguments");
  const int64_t nblocks = bytes / block_bytes;
  uint8_t* host = nullptr;
  uint8_t* dev = nullptr;
  unsigned long long* sink = nullptr;
  cudaError_t e;
  if (tier == ANN_TIER_HOST_PINNED) {
    e = cudaHostAlloc(reinterpret_cast<void**>(&host), (size_t)nblocks * block_bytes,
                      cudaHostAllocMapped | cudaHostAllocPortable);
    if (e == cudaSuccess) {
      std::memset(host, 1, (size_t)nblocks * block_bytes);
      e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&dev), host, 0);
    }
  } else {
    e = cudaMalloc(&dev, (size_t)nblocks * block_bytes);
    if (e == cudaSuccess) e = cudaMemset(dev, 1, (size_t)nblocks * block_bytes);
  }
  if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(unsigned long long));
  float ms = 0.f;
  int64_t moved = 0;
  if (e == cudaSuccess) e = launch_read_probe(dev, nblocks, block_bytes, iters, sink, 0, &ms, &moved);
  if (host) cudaFreeHost(host);
  else cudaFree(dev);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_error(e, "probe");
  *gbps_out = ms > 0.f ? (double)moved / (ms * 1e-3) / 1e9 : 0.0;
  return ANN_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Index files: "ANNIDX01", int64 n, int32 d, dtype, R, entry, M, 0, then the
// vectors, the adjacency, and (M > 0) the codebook and the codes.
// ---------------------------------------------------------------------------
namespace {

struct FileHeader {
  char magic[8];
  int64_t n;
  int32_t d, dtype, R, entry, M, flags;  // flags: bit 0 = an id map follows the codes
};

bool write_all(FILE* f, const void* p, size_t bytes) { return bytes == 0 || fwrite(p, 1, bytes, f) == bytes; }
bool read_all(FILE* f, void* p, size_t bytes) { return bytes == 0 || fread(p, 1, bytes, f) == bytes; }

}  // namespace

extern "C" {

int ann_save_graph_file(const char* path, const ann_graph_desc* g) {
  if (!path) return set_error(ANN_EINVAL, "path is NULL");
  ann_graph_desc chk = *g;
  chk.tier = ANN_TIER_HBM;
  int rc = validate_desc(&chk);
  if (rc != ANN_OK) return rc;
  FILE* f = fopen(path, "wb");
  if (!f) return set_error(ANN_EIO, "cannot open %s for writing", path);
  FileHeader h;
  std::memcpy(h.magic, "ANNIDX01", 8);
  h.n = g->n;
  h.d = g->d;
  h.dtype = g->dtype;
  h.R = g->R;
  h.entry = g->entry;
  h.M = g->M;
  h.flags = g->id_map ? 1 : 0;
  bool ok = write_all(f, &h, sizeof(h)) &&
            write_all(f, g->vectors, (size_t)g->n * g->d * elt_size(g->dtype)) &&
            write_all(f, g->adj, (size_t)g->n * g->R * 4);
  if (ok && g->M > 0)
    ok = write_all(f, g->codebook, (size_t)g->M * 256 * (g->d / g->M) * 4) &&
         write_all(f, g->codes, (size_t)g->n * g->M);
  if (ok && g->id_map) ok = write_all(f, g->id_map, (size_t)g->n * 4);
  ok = (fclose(f) == 0) && ok;
  return ok ? ANN_OK : set_error(ANN_EIO, "short write to %s", path);
}

int ann_load_graph_file(ann_index** out, const char* path, int32_t tier) {
  if (!out || !path) return set_error(ANN_EINVAL, "NULL argument");
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return set_error(ANN_EIO, "cannot open %s", path);
  FileHeader h;
  if (!read_all(f, &h, sizeof(h)) || std::memcmp(h.magic, "ANNIDX01", 8) != 0) {
    fclose(f);
    return set_error(ANN_EIO, "%s is not an index file", path);
  }
  if (h.n < 1 || h.n >= INT32_MAX || h.d < 4 || h.d > kMaxD || h.R < 1 || h.R > kMaxR ||
      h.M < 0 || h.M > kMaxM || (h.M > 0 && h.d % h.M) || (h.dtype != ANN_U8 && h.dtype != ANN_F32) ||
      (h.flags & ~1)) {
    fclose(f);
    return set_error(ANN_EIO, "%s: corrupt header", path);
  }
  std::vector<uint8_t> vec((size_t)h.n * h.d * elt_size(h.dtype));
  std::vector<int32_t> adj((size_t)h.n * h.R);
  std::vector<float> cb;
  std::vector<uint8_t> codes;
  bool ok = read_all(f, vec.data(), vec.size()) && read_all(f, adj.data(), adj.size() * 4);
  if (ok && h.M > 0) {
    cb.resize((size_t)h.M * 256 * (h.d / h.M));
    codes.resize((size_t)h.n * h.M);
    ok = read_all(f, cb.data(), cb.size() * 4) && read_all(f, codes.data(), codes.size());
  }
  std::vector<int32_t> id_map;
  if (ok && (h.flags & 1)) {
    id_map.resize((size_t)h.n);
    ok = read_all(f, id_map.data(), id_map.size() * 4);
  }
  fclose(f);
  if (!ok) return set_error(ANN_EIO, "%s is truncated", path);
  ann_graph_desc g{};
  g.n = h.n;
  g.d = h.d;
  g.dtype = h.dtype;
  g.R = h.R;
  g.entry = h.entry;
  g.vectors = vec.data();
  g.adj = adj.data();
  g.M = h.M;
  g.codebook = h.M > 0 ? cb.data() : nullptr;
  g.codes = h.M > 0 ? codes.data() : nullptr;
  g.tier = tier;
  g.id_map = id_map.empty() ? nullptr : id_map.data();
  return ann_load_graph(out, &g);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Read-only view of an index for other translation units of the library:
// fills the index part of SearchArgs and the plan inputs.
// ---------------------------------------------------------------------------
namespace ann {

int index_search_view(const ann_index* ix, SearchArgs* a, int* mode, int* slot_bytes) {
  if (!ix) return set_error(ANN_EINVAL, "index is NULL");
  *a = SearchArgs{};
  a->n = (int32_t)ix->n;
  a->d = ix->d;
  a->R = ix->R;
  a->entry = ix->entry;
  a->M = ix->M;
  a->dsub = ix->dsub;
  a->blocks = ix->blocks_dev;
  a->block_bytes = ix->block_bytes;
  a->ids_off = ix->ids_off;
  a->deg_off = ix->deg_off;
  a->slot_bytes = ix->slot_bytes;
  a->codes = ix->codes;
  a->cb_words = ix->cb_words;
  a->cb_f32 = ix->cb_f32;
  a->nav = ix->nav;
  a->nav_inv_scale = ix->nav_inv_scale;
  a->vectors = ix->vectors;
  a->adj = ix->adj;
  a->adj_stride = ix->adj_stride;
  a->id_map = ix->id_map;
  *mode = ix->mode;
  *slot_bytes = ix->slot_bytes;
  return ANN_OK;
}

}  // namespace ann
