// ann_build_graph: Vamana graph construction on host threads (index-build
// tooling, off the search path).  The paper searches DiskANN's Vamana index;
// this follows the published Vamana algorithm (Subramanya et al., NeurIPS'19):
// random start graph, GreedySearch + RobustPrune + back edges, one pass with
// alpha = 1 and one with the given alpha.  Nodes are inserted in batches that
// grow geometrically up to 2% of n: all searches of a batch read the graph as
// it stood before the batch, then the batch's edges and back edges are applied
// in a fixed order -- so the graph is independent of the thread count.
// alpha is compared with squared distances (DiskANN's own convention).
#include <algorithm>
#include <cmath>
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
void parallel_for(int64_t n, int threads, F&& fn) {
  if (threads <= 1 || n <= 1) {
    for (int64_t i = 0; i < n; ++i) fn(i, 0);
    return;
  }
  std::vector<std::thread> pool;
  const int t = static_cast<int>(std::min<int64_t>(threads, n));
  std::vector<int64_t> next(1, 0);
  for (int w = 0; w < t; ++w)
    pool.emplace_back([&, w] {
      for (int64_t i = w; i < n; i += t) fn(i, w);
    });
  for (auto& th : pool) th.join();
}

uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

struct Data {
  int dtype, d;
  const uint8_t* u8;
  const float* f32;
  float dist(int64_t a, int64_t b) const {
    if (dtype == ANN_U8) {
      const uint8_t* x = u8 + a * d;
      const uint8_t* y = u8 + b * d;
      uint32_t s = 0;
      for (int i = 0; i < d; ++i) {
        const int t = static_cast<int>(x[i]) - static_cast<int>(y[i]);
        s += static_cast<uint32_t>(t * t);
      }
      return static_cast<float>(s);
    }
    const float* x = f32 + a * d;
    const float* y = f32 + b * d;
    float s = 0.f;
    for (int i = 0; i < d; ++i) {
      const float t = x[i] - y[i];
      s += t * t;
    }
    return s;
  }
};

struct Cand {
  float dist;
  int32_t id;
  bool operator<(const Cand& o) const { return dist < o.dist || (dist == o.dist && id < o.id); }
};

// Per-thread scratch for GreedySearch.
struct Scratch {
  std::vector<uint64_t> seen;     // n-bit visited set
  std::vector<int32_t> touched;   // words to clear
  std::vector<Cand> list;         // sorted candidates, <= L
  std::vector<uint8_t> expanded;  // parallel to list
  std::vector<Cand> visited;      // expanded nodes with their distance
  void init(int64_t n, int L) {
    seen.assign((n + 63) / 64, 0);
    list.reserve(L + 1);
    expanded.reserve(L + 1);
  }
  bool test_set(int32_t v) {
    uint64_t& w = seen[v >> 6];
    const uint64_t bit = 1ull << (v & 63);
    if (w & bit) return true;
    if (w == 0) touched.push_back(v >> 6);
    w |= bit;
    return false;
  }
  void clear() {
    for (int32_t w : touched) seen[w] = 0;
    touched.clear();
  }
};

struct Graph {
  int R;
  std::vector<int32_t> nbr;  // n*R
  std::vector<int32_t> deg;  // n
};

// GreedySearch(entry, x_p, L): returns the expanded nodes with their distance to p.
void greedy_search(const Data& D, const Graph& G, int32_t entry, int64_t p, int L, Scratch& s) {
  s.list.clear();
  s.expanded.clear();
  s.visited.clear();
  s.test_set(entry);
  s.list.push_back({D.dist(entry, p), entry});
  s.expanded.push_back(0);
  for (;;) {
    size_t i = 0;
    while (i < s.list.size() && s.expanded[i]) ++i;
    if (i == s.list.size()) break;
    s.expanded[i] = 1;
    const Cand u = s.list[i];
    s.visited.push_back(u);
    const int32_t* nb = &G.nbr[(size_t)u.id * G.R];
    for (int j = 0; j < G.deg[u.id]; ++j) {
      const int32_t w = nb[j];
      if (s.test_set(w)) continue;
      const Cand c{D.dist(w, p), w};
      if (s.list.size() == static_cast<size_t>(L) && !(c < s.list.back())) continue;
      const size_t pos = std::upper_bound(s.list.begin(), s.list.end(), c) - s.list.begin();
      s.list.insert(s.list.begin() + pos, c);
      s.expanded.insert(s.expanded.begin() + pos, 0);
      if (s.list.size() > static_cast<size_t>(L)) {
        s.list.pop_back();
        s.expanded.pop_back();
      }
    }
  }
  s.clear();
}

// RobustPrune: cand holds (d2(p, c), c); keeps <= R ids in `out`.
void robust_prune(const Data& D, int64_t p, std::vector<Cand>& cand, float alpha, int R,
                  std::vector<int32_t>& out) {
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end(),
                         [](const Cand& a, const Cand& b) { return a.id == b.id; }),
             cand.end());
  out.clear();
  std::vector<uint8_t> gone(cand.size(), 0);
  for (size_t i = 0; i < cand.size() && static_cast<int>(out.size()) < R; ++i) {
    if (gone[i] || cand[i].id == p) continue;
    out.push_back(cand[i].id);
    for (size_t j = i + 1; j < cand.size(); ++j) {
      if (gone[j]) continue;
      if (alpha * D.dist(cand[i].id, cand[j].id) <= cand[j].dist) gone[j] = 1;
    }
  }
}

}  // namespace

extern "C" int ann_build_graph(const void* base, int32_t dtype, int64_t n, int32_t d, int32_t R,
                               float alpha, int32_t L_build, uint64_t seed, int32_t nthreads,
                               int32_t* adj_out, int32_t* entry_out) {
  using ann::set_error;
  if (!base || !adj_out) return set_error(ANN_EINVAL, "ann_build_graph: NULL buffer");
  if (dtype != ANN_U8 && dtype != ANN_F32) return set_error(ANN_EINVAL, "ann_build_graph: unknown dtype");
  if (n < 2 || n >= INT32_MAX || d < 1 || R < 1 || L_build < 1 || !(alpha >= 1.0f))
    return set_error(ANN_EINVAL, "ann_build_graph: bad sizes (n=%lld d=%d R=%d L=%d alpha=%g)",
                     (long long)n, d, R, L_build, alpha);
  const int threads = nthreads > 0 ? nthreads : static_cast<int>(std::max(1u, std::thread::hardware_concurrency()));
  Data D{dtype, d, static_cast<const uint8_t*>(base), static_cast<const float*>(base)};

  // Medoid: closest point to the float64 mean, lowest id on ties.
  std::vector<double> mean(d, 0.0);
  for (int64_t i = 0; i < n; ++i)
    for (int j = 0; j < d; ++j)
      mean[j] += dtype == ANN_U8 ? D.u8[i * d + j] : static_cast<double>(D.f32[i * d + j]);
  for (double& m : mean) m /= static_cast<double>(n);
  std::vector<double> md(threads, INFINITY);
  std::vector<int64_t> mi(threads, -1);
  parallel_for(threads, threads, [&](int64_t t, int) {
    for (int64_t i = t * n / threads; i < (t + 1) * n / threads; ++i) {
      double s = 0.0;
      for (int j = 0; j < d; ++j) {
        const double v = (dtype == ANN_U8 ? D.u8[i * d + j] : static_cast<double>(D.f32[i * d + j])) - mean[j];
        s += v * v;
      }
      if (s < md[t]) {
        md[t] = s;
        mi[t] = i;
      }
    }
  });
  int64_t entry = 0;
  double best = INFINITY;
  for (int t = 0; t < threads; ++t)
    if (mi[t] >= 0 && md[t] < best) {
      best = md[t];
      entry = mi[t];
    }

  // Random start graph and insertion order.
  Graph G;
  G.R = R;
  G.nbr.assign((size_t)n * R, -1);
  G.deg.assign(n, 0);
  uint64_t rs = seed;
  const int init_deg = static_cast<int>(std::min<int64_t>(R, n - 1));
  for (int64_t i = 0; i < n; ++i) {
    int32_t* row = &G.nbr[(size_t)i * R];
    int c = 0;
    while (c < init_deg) {
      const int32_t v = static_cast<int32_t>(splitmix64(rs) % static_cast<uint64_t>(n));
      if (v == i) continue;
      bool dup = false;
      for (int j = 0; j < c; ++j) dup |= row[j] == v;
      if (!dup) row[c++] = v;
    }
    G.deg[i] = c;
  }
  std::vector<int32_t> order(n);
  for (int64_t i = 0; i < n; ++i) order[i] = static_cast<int32_t>(i);
  for (int64_t i = n - 1; i > 0; --i) std::swap(order[i], order[splitmix64(rs) % static_cast<uint64_t>(i + 1)]);

  std::vector<Scratch> scratch(threads);
  for (auto& s : scratch) s.init(n, L_build);
  const int64_t max_batch = std::max<int64_t>(1, n / 50);
  std::vector<std::vector<int32_t>> newn;
  for (int pass = 0; pass < 2; ++pass) {
    const float a = pass == 0 ? 1.0f : alpha;
    int64_t done = 0, batch = 1;
    while (done < n) {
      const int64_t b = std::min(batch, n - done);
      newn.assign(b, {});
      // Searches and prunes of the batch against the frozen graph.
      parallel_for(b, threads, [&](int64_t i, int w) {
        const int64_t p = order[done + i];
        Scratch& s = scratch[w];
        greedy_search(D, G, static_cast<int32_t>(entry), p, L_build, s);
        std::vector<Cand> cand = s.visited;
        for (int j = 0; j < G.deg[p]; ++j) {
          const int32_t v = G.nbr[(size_t)p * R + j];
          cand.push_back({D.dist(v, p), v});
        }
        robust_prune(D, p, cand, a, R, newn[i]);
      });
      // Apply the new out-edges, then the back edges grouped by target.
      std::vector<std::pair<int32_t, int32_t>> back;
      for (int64_t i = 0; i < b; ++i) {
        const int64_t p = order[done + i];
        int32_t* row = &G.nbr[(size_t)p * R];
        std::fill(row, row + R, -1);
        std::copy(newn[i].begin(), newn[i].end(), row);
        G.deg[p] = static_cast<int32_t>(newn[i].size());
        for (int32_t j : newn[i]) back.emplace_back(j, static_cast<int32_t>(p));
      }
      std::sort(back.begin(), back.end());
      std::vector<int64_t> starts;
      for (size_t i = 0; i < back.size(); ++i)
        if (i == 0 || back[i].first != back[i - 1].first) starts.push_back(static_cast<int64_t>(i));
      starts.push_back(static_cast<int64_t>(back.size()));
      parallel_for(static_cast<int64_t>(starts.size()) - 1, threads, [&](int64_t g, int) {
        const int32_t j = back[starts[g]].first;
        int32_t* row = &G.nbr[(size_t)j * R];
        std::vector<int32_t> add;
        for (int64_t t = starts[g]; t < starts[g + 1]; ++t) {
          const int32_t p = back[t].second;
          bool have = false;
          for (int e = 0; e < G.deg[j]; ++e) have |= row[e] == p;
          if (!have) add.push_back(p);
        }
        if (add.empty()) return;
        if (G.deg[j] + static_cast<int>(add.size()) <= R) {
          for (int32_t p : add) row[G.deg[j]++] = p;
          return;
        }
        std::vector<Cand> cand;
        for (int e = 0; e < G.deg[j]; ++e) cand.push_back({D.dist(row[e], j), row[e]});
        for (int32_t p : add) cand.push_back({D.dist(p, j), p});
        std::vector<int32_t> out;
        robust_prune(D, j, cand, a, R, out);
        std::fill(row, row + R, -1);
        std::copy(out.begin(), out.end(), row);
        G.deg[j] = static_cast<int32_t>(out.size());
      });
      done += b;
      batch = std::min(batch * 2, max_batch);
    }
  }
  std::memcpy(adj_out, G.nbr.data(), (size_t)n * R * sizeof(int32_t));
  if (entry_out) *entry_out = static_cast<int32_t>(entry);
  return ANN_OK;
}
