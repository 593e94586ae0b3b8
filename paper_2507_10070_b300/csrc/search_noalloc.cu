// ann_search_dev_noalloc: the device-buffer search with no allocation at call
// time.
//
// Some callers cannot call cudaMalloc while they search: a serving thread
// with a hard latency budget (cudaMalloc can synchronise the device and take
// milliseconds), a process whose device memory is fully reserved up front by
// its own pool, or code that must not grow its footprint after start-up.  For
// them this entry point runs the same search kernel with its scratch -- the
// per-warp visited tables, their clear logs and the work counters -- in one
// file-scope device array of fixed size that every GPU loading the library
// holds until the process exits.  The caller still owns queries and outputs.
//
// Host code cannot use the array's name as a device address (on the host it
// names a stand-in object: a kernel handed it would fault, or silently touch
// the wrong memory where the GPU can reach host memory), so the first call on
// each device looks the address up with cudaGetSymbolAddress while that
// device is current and keeps it.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "ann_internal.h"

namespace ann {

int index_search_view(const ann_index* ix, SearchArgs* a, int* mode, int* slot_bytes);

namespace {

constexpr size_t kScratchBytes = 16ull << 20;  // 16 MiB per device
constexpr int kMinWarps = 32;                  // a call must fit at least 32 warps
constexpr int kMaxDevices = 64;
constexpr size_t kHeader = 256;                // counters + expansions, padded

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once).
int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_error(ANN_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(static scratch)");
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return ANN_OK;
}

}  // namespace
}  // namespace ann

using namespace ann;

extern "C" int ann_search_dev_noalloc(ann_index* ix, const void* queries, int64_t nq, int32_t k,
                                      int32_t L, int32_t depth, int32_t* ids, float* dists,
                                      const ann_trace* trace, void* stream) {
  if (!ix) return set_error(ANN_EINVAL, "index is NULL");
  if (nq < 0 || nq >= INT32_MAX) return set_error(ANN_EINVAL, "nq=%lld out of range", (long long)nq);
  if (k < 1 || L < k || L > kMaxL || k > 256)
    return set_error(ANN_EINVAL, "need 1 <= k <= min(L, 256), L <= %d (k=%d, L=%d)", kMaxL, k, L);
  if (depth < 0 || depth > kMaxDepth) return set_error(ANN_EINVAL, "depth=%d out of range", depth);
  if (nq > 0 && (!queries || !ids || !dists)) return set_error(ANN_EINVAL, "queries, ids and dists are required");
  if (reinterpret_cast<uintptr_t>(queries) % 16) return set_error(ANN_EINVAL, "queries must be 16-byte aligned");
  SearchArgs a{};
  int mode = 0, slot_bytes = 0;
  int rc = index_search_view(ix, &a, &mode, &slot_bytes);
  if (rc != ANN_OK) return rc;
  if (mode == kModeBF16 || mode == kModeFP8 || mode == kModePqF32)
    return set_error(ANN_EINVAL, "compressed-navigation indexes need the rerank pass: use ann_search_dev");
  void* base = nullptr;
  rc = scratch_address(&base);  // first call on a device: symbol lookup
  if (rc != ANN_OK) return rc;
  if (nq == 0) return ANN_OK;
  SearchPlan plan;
  cudaError_t e = plan_search(mode, a.R, a.M, a.d, slot_bytes, depth, L, k, nq, &plan, a.n);
  if (e != cudaSuccess) return cuda_error(e, "plan search");
  const size_t table_bytes = (size_t)plan.vis_words * 4;
  const size_t log_bytes = (size_t)plan.vis_log_cap * 4;
  const size_t per_warp = table_bytes + log_bytes;
  const size_t fit = (kScratchBytes - kHeader) / per_warp;
  if (fit < (size_t)kMinWarps)
    return set_error(ANN_EINVAL,
                     "an index of %d nodes needs %zu bytes of scratch per warp; the %zu MiB static "
                     "scratch must hold at least %d warps (use ann_search_dev)",
                     a.n, per_warp, kScratchBytes >> 20, kMinWarps);
  const int64_t warps = (int64_t)plan.blocks * plan.warps_per_block;
  if (warps > (int64_t)fit) plan.blocks = (int)(fit / plan.warps_per_block);
  const size_t nwarps = (size_t)plan.blocks * plan.warps_per_block;
  unsigned char* sb = static_cast<unsigned char*>(base);
  a.counters = reinterpret_cast<int32_t*>(sb);
  a.expansions = reinterpret_cast<unsigned long long*>(sb + 64);
  a.vis = reinterpret_cast<uint32_t*>(sb + kHeader);
  a.vis_words = plan.vis_words;
  a.vis_log = reinterpret_cast<uint32_t*>(sb + kHeader + nwarps * table_bytes);
  a.vis_log_cap = plan.vis_log_cap;
  a.queries = queries;
  a.nq = (int32_t)nq;
  a.k = k;
  a.L = L;
  a.depth = depth;
  a.ids = ids;
  a.dists = dists;
  a.steps = trace ? trace->steps : nullptr;
  a.status = trace ? trace->status : nullptr;
  a.t_begin = trace ? trace->t_begin : nullptr;
  a.t_end = trace ? trace->t_end : nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // The array keeps whatever the last call left: zero the counters and the
  // visited tables this call uses (the kernel needs all-zero tables), then
  // start counters[2] (lowest failed query, kept by atomicMin) at INT32_MAX,
  // as the other entry points do.
  static const int32_t kNoFailure = INT32_MAX;
  e = cudaMemsetAsync(sb, 0, kHeader, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sb + 2 * sizeof(int32_t), &kNoFailure, sizeof(kNoFailure),
                                            cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.vis, 0, nwarps * table_bytes, st);
  if (e != cudaSuccess) return cuda_error(e, "clear static scratch");
  e = launch_search(a, plan, st);
  if (e != cudaSuccess) return cuda_error(e, "search kernel launch");
  return ANN_OK;
}
