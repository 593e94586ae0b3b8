// ann_reorder_graph: breadth-first storage order of the node blocks
// (index-construction tooling, host threads).
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/ann.h"

namespace ann {
int set_error(int status, const char* fmt, ...);
}

namespace {

template <class F>
void parallel_rows(int64_t n, F&& fn) {
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

}  // namespace

extern "C" int ann_reorder_graph(const void* base, int32_t dtype, int64_t n, int32_t d, int32_t R,
                                 const int32_t* adj, int32_t entry, const uint8_t* codes, int32_t M,
                                 void* base_out, int32_t* adj_out, uint8_t* codes_out,
                                 int32_t* old_of_new, int32_t* entry_out) {
  using ann::set_error;
  if (!base || !adj || !base_out || !adj_out || !old_of_new || !entry_out)
    return set_error(ANN_EINVAL, "ann_reorder_graph: NULL buffer");
  if (dtype != ANN_U8 && dtype != ANN_F32) return set_error(ANN_EINVAL, "ann_reorder_graph: unknown dtype");
  if (n < 1 || n >= INT32_MAX || d < 1 || R < 1 || entry < 0 || entry >= n || M < 0 ||
      (M > 0 && (!codes || !codes_out)))
    return set_error(ANN_EINVAL, "ann_reorder_graph: bad sizes (n=%lld d=%d R=%d entry=%d M=%d)",
                     (long long)n, d, R, entry, M);
  std::atomic<int64_t> bad{-1};
  parallel_rows(n * R, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i)
      if (adj[i] < -1 || adj[i] >= n) {
        int64_t expect = -1;
        bad.compare_exchange_strong(expect, i);
        return;
      }
  });
  if (bad.load() >= 0)
    return set_error(ANN_EINVAL, "ann_reorder_graph: id %d in row %lld out of range", adj[bad.load()],
                     (long long)(bad.load() / R));
  // breadth-first order: old_of_new doubles as the queue
  std::vector<int32_t> pos(n, -1);  // new position of each node
  int64_t head = 0, tail = 0;
  old_of_new[tail] = entry;
  pos[entry] = static_cast<int32_t>(tail++);
  int64_t next_unreached = 0;
  while (tail < n) {
    if (head == tail) {  // the rest of the graph is not reachable from what is queued
      while (pos[next_unreached] >= 0) ++next_unreached;
      old_of_new[tail] = static_cast<int32_t>(next_unreached);
      pos[next_unreached] = static_cast<int32_t>(tail++);
    }
    const int32_t* row = adj + static_cast<size_t>(old_of_new[head++]) * R;
    for (int j = 0; j < R && row[j] >= 0; ++j)
      if (pos[row[j]] < 0) {
        old_of_new[tail] = row[j];
        pos[row[j]] = static_cast<int32_t>(tail++);
      }
  }
  // the rows in their new order
  const size_t row_bytes = static_cast<size_t>(d) * (dtype == ANN_U8 ? 1 : 4);
  parallel_rows(n, [&](int64_t lo, int64_t hi) {
    for (int64_t i = lo; i < hi; ++i) {
      const int64_t o = old_of_new[i];
      std::memcpy(static_cast<uint8_t*>(base_out) + i * row_bytes,
                  static_cast<const uint8_t*>(base) + o * row_bytes, row_bytes);
      if (M > 0) std::memcpy(codes_out + i * M, codes + o * M, static_cast<size_t>(M));
      const int32_t* src = adj + o * R;
      int32_t* dst = adj_out + i * R;
      for (int j = 0; j < R; ++j) dst[j] = src[j] >= 0 ? pos[src[j]] : -1;
    }
  });
  *entry_out = pos[entry];
  return ANN_OK;
}
