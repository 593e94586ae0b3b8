// ann_reorder_graph(_ex): storage order of the node blocks, breadth-first
// or spatial (index-construction tooling, host threads).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <utility>
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

uint64_t mix64(uint64_t z) {  // splitmix64's output function
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Spatial order: a tree of 2-means bisections.  A node [lo, hi) of `perm`
// splits into two parts of h and cnt - h points, h a multiple of the leaf
// size near cnt / 2, so that every leaf after the first starts at a multiple
// of `leaf` (one translation granule of node blocks).  The split direction
// comes from two seed points (a deterministic hash of the range) refined by
// three rounds of 2-means: the side of a point is its margin
// x.(a - b) - (|a|^2 - |b|^2) / 2, the h largest margins go first (ties by
// id), and a, b become the means of the two parts.  The leaves, in the order
// the in-place partition leaves them, are the storage order, so points that
// are close in space share granules.  Deterministic for any thread count.
struct Spatial {
  const void* base;
  bool u8;
  int d;
  int64_t leaf;

  float coord(int32_t id, int j) const {
    return u8 ? static_cast<float>(static_cast<const uint8_t*>(base)[static_cast<size_t>(id) * d + j])
              : static_cast<const float*>(base)[static_cast<size_t>(id) * d + j];
  }

  void split(int32_t* perm, int64_t lo, int64_t hi, int depth) const {
    const int64_t cnt = hi - lo;
    if (cnt <= leaf) return;
    int64_t h = ((cnt / 2 + leaf / 2) / leaf) * leaf;
    if (h < leaf) h = leaf;
    if (h >= cnt) h = cnt - 1;  // cannot happen for cnt > leaf, kept as a guard
    const uint64_t hs = mix64(static_cast<uint64_t>(lo) * 0x9e3779b97f4a7c15ull ^ static_cast<uint64_t>(hi));
    const int64_t i1 = static_cast<int64_t>(hs % static_cast<uint64_t>(cnt));
    int64_t i2 = static_cast<int64_t>((hs >> 32) % static_cast<uint64_t>(cnt));
    if (i2 == i1) i2 = (i1 + 1) % cnt;
    std::vector<float> a(d), b(d), w(d);
    for (int j = 0; j < d; ++j) {
      a[j] = coord(perm[lo + i1], j);
      b[j] = coord(perm[lo + i2], j);
    }
    std::vector<std::pair<float, int32_t>> m(static_cast<size_t>(cnt));
    const bool big = cnt > (1 << 20);
    for (int it = 0; it < 4; ++it) {
      double na = 0, nb = 0;
      for (int j = 0; j < d; ++j) {
        w[j] = a[j] - b[j];
        na += static_cast<double>(a[j]) * a[j];
        nb += static_cast<double>(b[j]) * b[j];
      }
      const float bias = static_cast<float>(0.5 * (na - nb));
      auto margins = [&](int64_t s, int64_t e) {
        for (int64_t i = s; i < e; ++i) {
          const int32_t id = perm[lo + i];
          float acc = 0.f;
          for (int j = 0; j < d; ++j) acc += coord(id, j) * w[j];
          m[i] = {acc - bias, id};
        }
      };
      if (big) parallel_rows(cnt, margins); else margins(0, cnt);
      std::nth_element(m.begin(), m.begin() + h, m.end(), [](const std::pair<float, int32_t>& x,
                                                             const std::pair<float, int32_t>& y) {
        return x.first > y.first || (x.first == y.first && x.second < y.second);
      });
      if (it == 3) break;
      // the means of the two parts (fixed chunks summed in order: deterministic)
      auto mean_of = [&](int64_t s, int64_t e, std::vector<float>& out) {
        const int64_t chunk = 1 << 16;
        const int64_t nchunks = (e - s + chunk - 1) / chunk;
        std::vector<double> part(static_cast<size_t>(nchunks) * d, 0.0);
        auto sum = [&](int64_t c0, int64_t c1) {
          for (int64_t c = c0; c < c1; ++c)
            for (int64_t i = s + c * chunk; i < std::min(e, s + (c + 1) * chunk); ++i)
              for (int j = 0; j < d; ++j) part[c * d + j] += coord(m[i].second, j);
        };
        if (big) parallel_rows(nchunks, sum); else sum(0, nchunks);
        for (int j = 0; j < d; ++j) {
          double t = 0;
          for (int64_t c = 0; c < nchunks; ++c) t += part[c * d + j];
          out[j] = static_cast<float>(t / static_cast<double>(e - s));
        }
      };
      mean_of(0, h, a);
      mean_of(h, cnt, b);
    }
    for (int64_t i = 0; i < cnt; ++i) perm[lo + i] = m[i].second;
    std::vector<std::pair<float, int32_t>>().swap(m);
    if (cnt > (1 << 20) && depth < 4) {
      std::thread t([&] { split(perm, lo, lo + h, depth + 1); });
      split(perm, lo + h, hi, depth + 1);
      t.join();
    } else {
      split(perm, lo, lo + h, depth + 1);
      split(perm, lo + h, hi, depth + 1);
    }
  }
};

}  // namespace

extern "C" int ann_reorder_graph_ex(const void* base, int32_t dtype, int64_t n, int32_t d, int32_t R,
                                    const int32_t* adj, int32_t entry, const uint8_t* codes, int32_t M,
                                    int32_t order, void* base_out, int32_t* adj_out, uint8_t* codes_out,
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
  if (order != ANN_ORDER_BFS && order != ANN_ORDER_SPATIAL)
    return set_error(ANN_EINVAL, "ann_reorder_graph: unknown order %d", order);
  std::vector<int32_t> pos(n, -1);  // new position of each node
  if (order == ANN_ORDER_SPATIAL) {
    for (int64_t i = 0; i < n; ++i) old_of_new[i] = static_cast<int32_t>(i);
    const Spatial sp{base, dtype == ANN_U8, d, 128};
    sp.split(old_of_new, 0, n, 0);
    for (int64_t i = 0; i < n; ++i) pos[old_of_new[i]] = static_cast<int32_t>(i);
  } else {
  // breadth-first order: old_of_new doubles as the queue
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

extern "C" int ann_reorder_graph(const void* base, int32_t dtype, int64_t n, int32_t d, int32_t R,
                                 const int32_t* adj, int32_t entry, const uint8_t* codes, int32_t M,
                                 void* base_out, int32_t* adj_out, uint8_t* codes_out,
                                 int32_t* old_of_new, int32_t* entry_out) {
  return ann_reorder_graph_ex(base, dtype, n, d, R, adj, entry, codes, M, ANN_ORDER_BFS, base_out, adj_out,
                              codes_out, old_of_new, entry_out);
}
