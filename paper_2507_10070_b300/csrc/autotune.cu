// ann_autotune_degree: the computation / I/O balanced degree selector
// (Section "Sampling-Based Graph Degree Selector", workflow and Eq. for d).
//
// For each candidate degree R the selector builds a sample index of random
// links -- the paper builds these instead of true neighbourhoods because only
// the memory and I/O pattern matters -- with the workload's element type and
// dimension, random uint8 vectors, random PQ codes and an integer codebook,
// and runs a batch of random queries through the same search kernel.
//   T_c(R): search time per step with the node blocks in HBM (the fetch is
//           short, so a step is its computation);
//   T_f(R): the extra time per step when the blocks sit in the storage tier
//           (host pinned memory read over PCIe) and every fetch is waited for
//           (depth 0);
// per-step times come from the device timestamps and step counts of every
// query (ann_trace), averaged over the batch.  The degree chosen is
// argmin_R |T_c(R) - T_f(R)|; at that degree the pipeline depth with the
// highest measured throughput is chosen.  Warps per query are fixed at one in
// this kernel and reported as such.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "ann_internal.h"

namespace {

uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

struct Timing {
  double step_us = 0;   // mean per-step time over queries
  double qps = 0;       // queries / kernel time
  double steps = 0;     // mean steps per query
};

int time_search(ann_index* ix, const std::vector<uint8_t>& q, int nq, int k, int L, int depth,
                Timing* out) {
  std::vector<int32_t> ids((size_t)nq * k), steps(nq), status(nq);
  std::vector<float> dists((size_t)nq * k);
  std::vector<int64_t> tb(nq), te(nq);
  ann_trace tr{steps.data(), status.data(), tb.data(), te.data()};
  ann_search_stats st{};
  // warm-up, then the measured call
  int rc = ann_search(ix, q.data(), nq, k, L, depth, ids.data(), dists.data(), &tr, &st);
  if (rc != ANN_OK && rc != ANN_ENOMEM) return rc;
  rc = ann_search(ix, q.data(), nq, k, L, depth, ids.data(), dists.data(), &tr, &st);
  if (rc != ANN_OK && rc != ANN_ENOMEM) return rc;
  double sum = 0, ssum = 0;
  int cnt = 0;
  for (int i = 0; i < nq; ++i) {
    if (steps[i] > 0 && status[i] == ANN_OK) {
      sum += double(te[i] - tb[i]) / 1e3 / steps[i];
      ssum += steps[i];
      ++cnt;
    }
  }
  out->step_us = cnt ? sum / cnt : 0.0;
  out->steps = cnt ? ssum / cnt : 0.0;
  out->qps = st.kernel_ms > 0 ? nq / (st.kernel_ms * 1e-3) : 0.0;
  return ANN_OK;
}

}  // namespace

extern "C" int ann_autotune_degree(const ann_autotune_cfg* cfg, ann_autotune_point* points,
                                   int32_t* best_degree, int32_t* best_depth,
                                   float* depth_qps /* [5], may be NULL */,
                                   int32_t* best_warps, float* warps_qps /* [3], may be NULL */) {
  using ann::set_error;
  if (!cfg || !points || !best_degree || !best_depth || !best_warps)
    return set_error(ANN_EINVAL, "ann_autotune_degree: NULL argument");
  if (cfg->n_sample < 1024 || cfg->d < 16 || cfg->d % 16 || cfg->M < 16 || cfg->M % 16 ||
      cfg->d % cfg->M || (cfg->d / cfg->M) % 4 || cfg->n_degrees < 1 || cfg->nq < 32 ||
      cfg->L < 10 || cfg->L > ann::kMaxL)
    return set_error(ANN_EINVAL, "ann_autotune_degree: bad configuration");
  for (int i = 0; i < cfg->n_degrees; ++i)
    if (cfg->degrees[i] < 1 || cfg->degrees[i] > ann::kMaxR || cfg->degrees[i] >= cfg->n_sample)
      return set_error(ANN_EINVAL, "degree %d out of range", cfg->degrees[i]);
  const int64_t n = cfg->n_sample;
  const int d = cfg->d, M = cfg->M, dsub = d / M, nq = cfg->nq, k = 10;
  uint64_t rs = cfg->seed;
  std::vector<uint8_t> base((size_t)n * d), q((size_t)nq * d), codes((size_t)n * M);
  for (auto& v : base) v = static_cast<uint8_t>(splitmix64(rs));
  for (auto& v : q) v = static_cast<uint8_t>(splitmix64(rs));
  for (auto& v : codes) v = static_cast<uint8_t>(splitmix64(rs));
  std::vector<float> cb((size_t)M * 256 * dsub);
  for (auto& v : cb) v = static_cast<float>(splitmix64(rs) & 0xff);
  double best_gap = INFINITY;
  *best_degree = cfg->degrees[0];
  for (int di = 0; di < cfg->n_degrees; ++di) {
    const int R = cfg->degrees[di];
    std::vector<int32_t> adj((size_t)n * R);
    for (int64_t i = 0; i < n; ++i)
      for (int j = 0; j < R; ++j) {
        int32_t v;
        do {
          v = static_cast<int32_t>(splitmix64(rs) % static_cast<uint64_t>(n));
        } while (v == i);
        adj[(size_t)i * R + j] = v;  // a repeated id is simply seen as visited
      }
    Timing host{}, hbm{};
    for (int tier = 0; tier < 2; ++tier) {
      ann_graph_desc g{};
      g.n = n;
      g.d = d;
      g.dtype = ANN_U8;
      g.R = R;
      g.entry = 0;
      g.vectors = base.data();
      g.adj = adj.data();
      g.M = M;
      g.codebook = cb.data();
      g.codes = codes.data();
      g.tier = tier == 0 ? ANN_TIER_HOST_PINNED : ANN_TIER_HBM;
      ann_index* ix = nullptr;
      int rc = ann_load_graph(&ix, &g);
      if (rc != ANN_OK) return rc;
      rc = time_search(ix, q, nq, k, cfg->L, 0, tier == 0 ? &host : &hbm);
      ann_free(ix);
      if (rc != ANN_OK) return rc;
    }
    ann_autotune_point& p = points[di];
    p.degree = R;
    p.t_compute_us = static_cast<float>(hbm.step_us);
    p.t_fetch_us = static_cast<float>(host.step_us > hbm.step_us ? host.step_us - hbm.step_us : 0.0);
    p.step_us_sync = static_cast<float>(host.step_us);
    p.qps_sync = static_cast<float>(host.qps);
    const double gap = std::fabs(p.t_compute_us - p.t_fetch_us);
    if (gap < best_gap) {
      best_gap = gap;
      *best_degree = R;
    }
  }
  // pipeline depth at the chosen degree: the highest measured throughput
  {
    const int R = *best_degree;
    std::vector<int32_t> adj((size_t)n * R);
    for (int64_t i = 0; i < n; ++i)
      for (int j = 0; j < R; ++j) {
        int32_t v;
        do {
          v = static_cast<int32_t>(splitmix64(rs) % static_cast<uint64_t>(n));
        } while (v == i);
        adj[(size_t)i * R + j] = v;
      }
    ann_graph_desc g{};
    g.n = n;
    g.d = d;
    g.dtype = ANN_U8;
    g.R = R;
    g.entry = 0;
    g.vectors = base.data();
    g.adj = adj.data();
    g.M = M;
    g.codebook = cb.data();
    g.codes = codes.data();
    g.tier = ANN_TIER_HOST_PINNED;
    ann_index* ix = nullptr;
    int rc = ann_load_graph(&ix, &g);
    if (rc != ANN_OK) return rc;
    double best_q = -1;
    const int depths[5] = {0, 1, 2, 3, 4};
    for (int di = 0; di < 5; ++di) {
      Timing t{};
      rc = time_search(ix, q, nq, k, cfg->L, depths[di], &t);
      if (rc != ANN_OK) break;
      if (depth_qps) depth_qps[di] = static_cast<float>(t.qps);
      if (t.qps > best_q) {
        best_q = t.qps;
        *best_depth = depths[di];
      }
    }
    // warps per query at that degree and depth: 1, 2 or 4, the highest
    // measured throughput
    double best_w = -1;
    const int warps[3] = {1, 2, 4};
    *best_warps = 1;
    for (int wi = 0; wi < 3 && rc == ANN_OK; ++wi) {
      rc = ann_set_warps_per_query(ix, warps[wi]);
      if (rc != ANN_OK) break;
      Timing t{};
      rc = time_search(ix, q, nq, k, cfg->L, *best_depth, &t);
      if (rc != ANN_OK) break;
      if (warps_qps) warps_qps[wi] = static_cast<float>(t.qps);
      if (t.qps > best_w) {
        best_w = t.qps;
        *best_warps = warps[wi];
      }
    }
    ann_free(ix);
    if (rc != ANN_OK) return rc;
  }
  return ANN_OK;
}
