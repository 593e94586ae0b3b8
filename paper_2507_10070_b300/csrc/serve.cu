// ann_serve_*: a continuous-batching request loop over one index.
//
// Requests (batches of queries with their own k and L) are admitted as work
// items into a ring of `slots` staging entries in mapped pinned host memory;
// admission is by free staging slots (ANN_EBUSY when full).  A persistent
// serving kernel (serve_kernel in search.cu) keeps one query per resident
// warp: a warp that finishes a query claims the next published item, whatever
// request it belongs to, so requests that arrive while others run start as
// soon as a warp frees up and overlap on the device.  Results go straight to
// mapped host memory, followed by a per-item done word that ann_serve_poll
// waits on.  Each query's search is independent of the others, so a query's
// results are the same alone and in any mix.
//
// A host thread owns the kernel's life: it launches it when items are
// pending and it is not running; the kernel returns on its own after
// `idle_exit_us` without work (bounded polling), or when asked to stop.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ann_internal.h"

namespace ann {
int index_search_view(const ann_index* ix, SearchArgs* a, int* mode, int* slot_bytes);
}

using namespace ann;

struct ann_server {
  ann_index* ix = nullptr;
  ann_serve_cfg cfg{};
  int device = 0;
  int mode = 0, slot_bytes = 0, qbytes = 0;
  SearchArgs args{};
  SearchPlan plan{};
  ServeArgs sa{};
  // mapped pinned host region and its parts
  void* host = nullptr;
  volatile unsigned long long* tail = nullptr;
  volatile int* stop_flag = nullptr;
  int32_t* item_kL = nullptr;
  uint8_t* qbuf = nullptr;
  int32_t* rids = nullptr;
  float* rdists = nullptr;
  int32_t* rsteps = nullptr;
  int32_t* rstatus = nullptr;
  int64_t* rtimes = nullptr;
  volatile unsigned long long* done = nullptr;
  // device memory
  unsigned long long* head_d = nullptr;  // [0] head, [1] tail mirror, [2] last claim time
  uint32_t* vis_d = nullptr;
  uint32_t* vlog_d = nullptr;
  int32_t* counters_d = nullptr;
  unsigned long long* exp_d = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t finished = nullptr;
  // bookkeeping (under mu)
  std::mutex mu;
  std::condition_variable cv;
  uint64_t published = 0, retired = 0, claimed = 0;
  std::vector<uint8_t> consumed;
  struct Req {
    uint64_t first;
    int64_t nq;
    int32_t k;
    int64_t ready;  // leading queries known to be done
  };
  std::unordered_map<uint64_t, Req> reqs;
  uint64_t next_req = 1;
  bool running = false, quit = false;
  int64_t launches = 0;
  cudaError_t launch_error = cudaSuccess;
  std::thread launcher;
};

namespace {

void launcher_loop(ann_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->quit) {
    if (s->running) {
      // Any answer but "not ready" ends the run; an error (a failed kernel)
      // is kept and returned by every later submit and poll.
      const cudaError_t q = cudaEventQuery(s->finished);
      if (q == cudaSuccess) {
        s->running = false;
        unsigned long long h = 0;
        cudaError_t e = cudaMemcpyAsync(&h, s->head_d, sizeof(h), cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e == cudaSuccess) s->claimed = h;
        else s->launch_error = e;
      } else if (q != cudaErrorNotReady) {
        s->running = false;
        s->launch_error = q;
      }
    }
    if (!s->running && s->published > s->claimed && s->launch_error == cudaSuccess) {
      cudaError_t e = launch_serve(s->args, s->sa, s->plan, s->stream);
      if (e == cudaSuccess) e = cudaEventRecord(s->finished, s->stream);
      if (e != cudaSuccess) {
        s->launch_error = e;
      } else {
        s->running = true;
        ++s->launches;
      }
    }
    s->cv.wait_for(lk, std::chrono::microseconds(s->running ? 200 : 50));
  }
}

void destroy(ann_server* s) {
  if (!s) return;
  if (s->launcher.joinable()) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->quit = true;
    }
    s->cv.notify_all();
    s->launcher.join();
  }
  if (s->stop_flag) *s->stop_flag = 1;
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->host) cudaFreeHost(s->host);
  cudaFree(s->head_d);
  cudaFree(s->vis_d);
  cudaFree(s->vlog_d);
  cudaFree(s->counters_d);
  cudaFree(s->exp_d);
  if (s->finished) cudaEventDestroy(s->finished);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

size_t align_to(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

extern "C" {

int ann_serve_create(ann_index* ix, const ann_serve_cfg* cfg, ann_server** out) {
  if (!ix || !cfg || !out) return set_error(ANN_EINVAL, "ann_serve_create: NULL argument");
  *out = nullptr;
  if (cfg->max_L < 1 || cfg->max_L > kMaxL || cfg->max_k < 1 || cfg->max_k > 256 ||
      cfg->max_k > cfg->max_L)
    return set_error(ANN_EINVAL, "need 1 <= max_k <= min(max_L, 256), max_L <= %d", kMaxL);
  if (cfg->depth < 0 || cfg->depth > kMaxDepth) return set_error(ANN_EINVAL, "depth out of range");
  if (cfg->slots < 1 || cfg->slots > (1 << 24)) return set_error(ANN_EINVAL, "slots out of range");
  if (cfg->idle_exit_us < 1) return set_error(ANN_EINVAL, "idle_exit_us must be positive");
  ann_server* s = new ann_server();
  s->ix = ix;
  s->cfg = *cfg;
  int rc = index_search_view(ix, &s->args, &s->mode, &s->slot_bytes);
  if (rc != ANN_OK) {
    delete s;
    return rc;
  }
  if (s->mode == kModeBF16 || s->mode == kModeFP8 || s->mode == kModePqF32) {
    delete s;
    return set_error(ANN_EINVAL, "compressed-navigation indexes need the rerank pass: serve a PQ-u8 or exact index");
  }
  cudaError_t e = cudaGetDevice(&s->device);
  if (e != cudaSuccess) {
    delete s;
    return cuda_error(e, "cudaGetDevice");
  }
  s->qbytes = s->args.d * (s->mode == kModeExactF32 ? 4 : 1);
  e = plan_search(s->mode, s->args.R, s->args.M, s->args.d, s->slot_bytes, cfg->depth,
                  cfg->max_L, cfg->max_k, INT32_MAX, &s->plan, s->args.n);
  if (e != cudaSuccess) {
    delete s;
    return cuda_error(e, "plan serving kernel");
  }
  const size_t slots = (size_t)cfg->slots;
  // one mapped host region: control words, items, queries, results
  size_t off = 0;
  const size_t o_ctrl = off;
  off += 256;
  const size_t o_kL = off;
  off = align_to(off + slots * 8, 256);
  const size_t o_q = off;
  off = align_to(off + slots * s->qbytes, 256);
  const size_t o_ids = off;
  off = align_to(off + slots * cfg->max_k * 4, 256);
  const size_t o_d = off;
  off = align_to(off + slots * cfg->max_k * 4, 256);
  const size_t o_steps = off;
  off = align_to(off + slots * 4, 256);
  const size_t o_status = off;
  off = align_to(off + slots * 4, 256);
  const size_t o_times = off;
  off = align_to(off + slots * 16, 256);
  const size_t o_done = off;
  off = align_to(off + slots * 8, 256);
#define SV_TRY(call, what)          \
  do {                              \
    e = (call);                     \
    if (e != cudaSuccess) {         \
      destroy(s);                   \
      return cuda_error(e, what);   \
    }                               \
  } while (0)
  SV_TRY(cudaHostAlloc(&s->host, off, cudaHostAllocMapped | cudaHostAllocPortable), "cudaHostAlloc serving ring");
  std::memset(s->host, 0, off);
  uint8_t* h = static_cast<uint8_t*>(s->host);
  s->tail = reinterpret_cast<volatile unsigned long long*>(h + o_ctrl);
  s->stop_flag = reinterpret_cast<volatile int*>(h + o_ctrl + 64);
  s->item_kL = reinterpret_cast<int32_t*>(h + o_kL);
  s->qbuf = h + o_q;
  s->rids = reinterpret_cast<int32_t*>(h + o_ids);
  s->rdists = reinterpret_cast<float*>(h + o_d);
  s->rsteps = reinterpret_cast<int32_t*>(h + o_steps);
  s->rstatus = reinterpret_cast<int32_t*>(h + o_status);
  s->rtimes = reinterpret_cast<int64_t*>(h + o_times);
  s->done = reinterpret_cast<volatile unsigned long long*>(h + o_done);
  uint8_t* hd = nullptr;
  SV_TRY(cudaHostGetDevicePointer(reinterpret_cast<void**>(&hd), s->host, 0), "cudaHostGetDevicePointer");
  const size_t nwarps = (size_t)s->plan.blocks * s->plan.warps_per_block;
  SV_TRY(cudaMalloc(&s->head_d, 3 * sizeof(unsigned long long)), "cudaMalloc serving head");
  SV_TRY(cudaMemset(s->head_d, 0, 3 * sizeof(unsigned long long)), "cudaMemset");
  SV_TRY(cudaMalloc(&s->vis_d, nwarps * s->plan.vis_words * 4), "cudaMalloc visited sets");
  SV_TRY(cudaMemset(s->vis_d, 0, nwarps * s->plan.vis_words * 4), "cudaMemset");
  SV_TRY(cudaMalloc(&s->vlog_d, nwarps * s->plan.vis_log_cap * 4), "cudaMalloc visited logs");
  SV_TRY(cudaMalloc(&s->counters_d, 4 * sizeof(int32_t)), "cudaMalloc counters");
  SV_TRY(cudaMemset(s->counters_d, 0, 4 * sizeof(int32_t)), "cudaMemset");
  SV_TRY(cudaMalloc(&s->exp_d, sizeof(unsigned long long)), "cudaMalloc counters");
  SV_TRY(cudaMemset(s->exp_d, 0, sizeof(unsigned long long)), "cudaMemset");
  SV_TRY(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking), "cudaStreamCreate");
  SV_TRY(cudaEventCreateWithFlags(&s->finished, cudaEventDisableTiming), "cudaEventCreate");
#undef SV_TRY
  s->args.L = cfg->max_L;
  s->args.k = cfg->max_k;
  s->args.depth = cfg->depth;
  s->args.vis = s->vis_d;
  s->args.vis_words = s->plan.vis_words;
  s->args.vis_log = s->vlog_d;
  s->args.vis_log_cap = s->plan.vis_log_cap;
  s->args.counters = s->counters_d;
  s->args.expansions = s->exp_d;
  ServeArgs& a = s->sa;
  a.tail = reinterpret_cast<const unsigned long long*>(hd + o_ctrl);
  a.stop = reinterpret_cast<const int*>(hd + o_ctrl + 64);
  a.head = s->head_d;
  a.tail_mirror = s->head_d + 1;
  a.last_claim = s->head_d + 2;
  a.item_kL = reinterpret_cast<const int32_t*>(hd + o_kL);
  a.qbuf = hd + o_q;
  a.rids = reinterpret_cast<int32_t*>(hd + o_ids);
  a.rdists = reinterpret_cast<float*>(hd + o_d);
  a.rsteps = reinterpret_cast<int32_t*>(hd + o_steps);
  a.rstatus = reinterpret_cast<int32_t*>(hd + o_status);
  a.rtimes = reinterpret_cast<int64_t*>(hd + o_times);
  a.done = reinterpret_cast<unsigned long long*>(hd + o_done);
  a.slots = cfg->slots;
  a.qbytes = s->qbytes;
  a.max_k = cfg->max_k;
  a.idle_ns = (long long)cfg->idle_exit_us * 1000;
  s->consumed.assign(slots, 1);
  s->launcher = std::thread(launcher_loop, s);
  *out = s;
  return ANN_OK;
}

int ann_serve_submit(ann_server* s, const void* queries, int64_t nq, int32_t k, int32_t L,
                     uint64_t* req_id) {
  if (!s || !queries || !req_id) return set_error(ANN_EINVAL, "ann_serve_submit: NULL argument");
  if (nq < 1 || nq > s->cfg.slots) return set_error(ANN_EINVAL, "nq=%lld out of range [1, %d]", (long long)nq, s->cfg.slots);
  if (k < 1 || k > s->cfg.max_k || L < k || L > s->cfg.max_L)
    return set_error(ANN_EINVAL, "need 1 <= k <= %d, k <= L <= %d (k=%d, L=%d)", s->cfg.max_k, s->cfg.max_L, k, L);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->launch_error != cudaSuccess) return cuda_error(s->launch_error, "serving kernel launch");
  const uint64_t in_use = s->published - s->retired;
  if ((uint64_t)nq > (uint64_t)s->cfg.slots - in_use)
    return set_error(ANN_EBUSY, "%lld queries do not fit: %llu of %d staging slots free",
                     (long long)nq, (unsigned long long)(s->cfg.slots - in_use), s->cfg.slots);
  const uint8_t* q = static_cast<const uint8_t*>(queries);
  for (int64_t i = 0; i < nq; ++i) {
    const uint64_t item = s->published + i;
    const size_t slot = item % s->cfg.slots;
    std::memcpy(s->qbuf + slot * s->qbytes, q + i * s->qbytes, s->qbytes);
    s->item_kL[2 * slot] = k;
    s->item_kL[2 * slot + 1] = L;
    s->consumed[slot] = 0;
  }
  const uint64_t first = s->published;
  s->published += nq;
  std::atomic_thread_fence(std::memory_order_release);
  *s->tail = s->published;  // publish: the kernel reads it with acquire semantics
  *req_id = s->next_req++;
  s->reqs[*req_id] = {first, nq, k, 0};
  s->cv.notify_all();
  return ANN_OK;
}

int ann_serve_poll(ann_server* s, uint64_t req_id, int32_t* ids, float* dists, int64_t timeout_us,
                   ann_serve_result* info) {
  if (!s || !ids || !dists) return set_error(ANN_EINVAL, "ann_serve_poll: NULL argument");
  ann_server::Req r;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return set_error(ANN_EINVAL, "unknown request %llu", (unsigned long long)req_id);
    r = it->second;
    if (s->launch_error != cudaSuccess) return cuda_error(s->launch_error, "serving kernel launch");
  }
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us > 0 ? timeout_us : 0);
  int64_t ready = 0;
  for (;;) {
    while (ready < r.nq && s->done[(r.first + ready) % s->cfg.slots] == r.first + ready + 1) ++ready;
    if (ready == r.nq) break;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->launch_error != cudaSuccess) return cuda_error(s->launch_error, "serving kernel");
    }
    if (std::chrono::steady_clock::now() >= deadline)
      return set_error(ANN_ETIMEOUT, "request %llu: %lld of %lld queries done", (unsigned long long)req_id,
                       (long long)ready, (long long)r.nq);
    std::this_thread::sleep_for(std::chrono::microseconds(10));
  }
  std::atomic_thread_fence(std::memory_order_acquire);
  int failed = 0;
  int64_t steps = 0, t0 = INT64_MAX, t1 = 0;
  for (int64_t i = 0; i < r.nq; ++i) {
    const size_t slot = (r.first + i) % s->cfg.slots;
    std::memcpy(ids + i * r.k, s->rids + slot * s->cfg.max_k, r.k * 4);
    std::memcpy(dists + i * r.k, s->rdists + slot * s->cfg.max_k, r.k * 4);
    if (s->rstatus[slot] != ANN_OK) ++failed;
    steps += s->rsteps[slot];
    t0 = std::min<int64_t>(t0, s->rtimes[2 * slot]);
    t1 = std::max<int64_t>(t1, s->rtimes[2 * slot + 1]);
  }
  if (info) {
    info->queries = r.nq;
    info->expansions = steps;
    info->n_failed = failed;
    info->device_ns = t1 - t0;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (int64_t i = 0; i < r.nq; ++i) s->consumed[(r.first + i) % s->cfg.slots] = 1;
    while (s->retired < s->published && s->consumed[s->retired % s->cfg.slots]) ++s->retired;
    s->reqs.erase(req_id);
  }
  if (failed) return set_error(ANN_ENOMEM, "request %llu: %d queries stopped early",
                               (unsigned long long)req_id, failed);
  return ANN_OK;
}

int ann_serve_poll_any(ann_server* s, uint64_t* req_ids, int32_t max, int64_t timeout_us,
                       int32_t* n_ready) {
  if (!s || !req_ids || !n_ready || max < 1) return set_error(ANN_EINVAL, "ann_serve_poll_any: bad argument");
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us > 0 ? timeout_us : 0);
  for (;;) {
    int32_t n = 0;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->launch_error != cudaSuccess) return cuda_error(s->launch_error, "serving kernel launch");
      for (auto& kv : s->reqs) {
        ann_server::Req& r = kv.second;
        while (r.ready < r.nq && s->done[(r.first + r.ready) % s->cfg.slots] == r.first + r.ready + 1) ++r.ready;
        if (r.ready == r.nq) {
          req_ids[n++] = kv.first;
          if (n == max) break;
        }
      }
    }
    if (n > 0 || std::chrono::steady_clock::now() >= deadline) {
      *n_ready = n;
      return ANN_OK;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(10));
  }
}

int ann_serve_stats(ann_server* s, ann_serve_counters* out) {
  if (!s || !out) return set_error(ANN_EINVAL, "ann_serve_stats: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  out->launches = s->launches;
  out->published = (int64_t)s->published;
  out->retired = (int64_t)s->retired;
  out->resident_warps = (int64_t)s->plan.blocks * s->plan.warps_per_block;
  out->running = s->running ? 1 : 0;
  return ANN_OK;
}

void ann_serve_destroy(ann_server* s) { destroy(s); }

}  // extern "C"
