// ann_build_pq: product-quantiser training and encoding on host threads
// (index-construction tooling, off the search path).
//
// Per subspace: k-means++ seeding (Arthur & Vassilvitskii 2007) driven by the
// caller's uniforms, then Lloyd iterations; empty clusters take the point
// farthest from its centroid.  The arithmetic is float64 in a fixed order
// per point, so for uint8 data (integer inputs, exact sums) the codebook is a
// deterministic function of the inputs whatever the thread count.
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
    for (int64_t i = 0; i < n; ++i) fn(i);
    return;
  }
  std::vector<std::thread> pool;
  const int t = static_cast<int>(std::min<int64_t>(threads, n));
  for (int w = 0; w < t; ++w)
    pool.emplace_back([&, w] {
      for (int64_t i = w; i < n; i += t) fn(i);
    });
  for (auto& th : pool) th.join();
}

uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

inline double sub_dist(const double* x, const double* c, int dsub) {
  double s = 0.0;
  for (int j = 0; j < dsub; ++j) {
    const double t = x[j] - c[j];
    s += t * t;
  }
  return s;
}

// One subspace: X is ns x dsub (float64), C receives K x dsub.
void train_subspace(const double* X, int64_t ns, int dsub, int K, int iters, const double* u,
                    double* C) {
  std::vector<double> D2(ns), adist(ns), sum((size_t)K * dsub);
  std::vector<int32_t> asg(ns);
  std::vector<int64_t> cnt(K);
  int64_t first = static_cast<int64_t>(u[0] * static_cast<double>(ns));
  if (first >= ns) first = ns - 1;
  std::memcpy(C, X + first * dsub, sizeof(double) * dsub);
  for (int64_t i = 0; i < ns; ++i) D2[i] = sub_dist(X + i * dsub, C, dsub);
  for (int c = 1; c < K; ++c) {
    double total = 0.0;
    for (int64_t i = 0; i < ns; ++i) total += D2[i];
    int64_t pick;
    if (total > 0.0) {
      const double target = u[c] * total;
      double run = 0.0;
      pick = ns - 1;
      for (int64_t i = 0; i < ns; ++i) {
        run += D2[i];
        if (run > target) {
          pick = i;
          break;
        }
      }
    } else {
      pick = static_cast<int64_t>(u[c] * static_cast<double>(ns));
      if (pick >= ns) pick = ns - 1;
    }
    double* cc = C + (size_t)c * dsub;
    std::memcpy(cc, X + pick * dsub, sizeof(double) * dsub);
    for (int64_t i = 0; i < ns; ++i) {
      const double t = sub_dist(X + i * dsub, cc, dsub);
      if (t < D2[i]) D2[i] = t;
    }
  }
  for (int it = 0; it < iters; ++it) {
    for (int64_t i = 0; i < ns; ++i) {
      int best = 0;
      double bd = INFINITY;
      for (int c = 0; c < K; ++c) {
        const double t = sub_dist(X + i * dsub, C + (size_t)c * dsub, dsub);
        if (t < bd) {
          bd = t;
          best = c;
        }
      }
      asg[i] = best;
      adist[i] = bd;
    }
    std::fill(sum.begin(), sum.end(), 0.0);
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int64_t i = 0; i < ns; ++i) {
      cnt[asg[i]] += 1;
      for (int j = 0; j < dsub; ++j) sum[(size_t)asg[i] * dsub + j] += X[i * dsub + j];
    }
    for (int c = 0; c < K; ++c) {
      if (cnt[c] > 0) {
        for (int j = 0; j < dsub; ++j)
          C[(size_t)c * dsub + j] = sum[(size_t)c * dsub + j] / static_cast<double>(cnt[c]);
      } else {
        int64_t far = -1;
        double fd = -1.0;
        for (int64_t i = 0; i < ns; ++i)
          if (adist[i] > fd) {
            fd = adist[i];
            far = i;
          }
        adist[far] = -2.0;
        std::memcpy(C + (size_t)c * dsub, X + far * dsub, sizeof(double) * dsub);
      }
    }
  }
}

}  // namespace

extern "C" int ann_build_pq(const void* base, int32_t dtype, int64_t n, int32_t d, int32_t M,
                            int64_t n_train, int32_t iters, const double* kpp_uniforms,
                            uint64_t seed, float* codebook_out, uint8_t* codes_out,
                            int32_t nthreads) {
  using ann::set_error;
  constexpr int K = 256;
  if (!base || !codebook_out || !codes_out) return set_error(ANN_EINVAL, "ann_build_pq: NULL buffer");
  if (dtype != ANN_U8 && dtype != ANN_F32) return set_error(ANN_EINVAL, "ann_build_pq: unknown dtype");
  if (M < 1 || d < 1 || d % M) return set_error(ANN_EINVAL, "ann_build_pq: d=%d not divisible by M=%d", d, M);
  const int64_t ns = std::min(n, n_train);
  if (ns < K) return set_error(ANN_EINVAL, "ann_build_pq: need at least %d training vectors", K);
  if (iters < 0) return set_error(ANN_EINVAL, "ann_build_pq: iters < 0");
  int threads = nthreads > 0 ? nthreads : static_cast<int>(std::max(1u, std::thread::hardware_concurrency()));
  const int dsub = d / M;
  std::vector<double> u((size_t)M * K);
  if (kpp_uniforms) {
    std::memcpy(u.data(), kpp_uniforms, u.size() * sizeof(double));
  } else {
    uint64_t s = seed;
    for (auto& v : u) v = static_cast<double>(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
  }
  auto elem = [&](int64_t i, int j) -> double {
    return dtype == ANN_U8 ? static_cast<double>(static_cast<const uint8_t*>(base)[i * d + j])
                           : static_cast<double>(static_cast<const float*>(base)[i * d + j]);
  };
  std::vector<double> cbd((size_t)M * K * dsub);
  parallel_for(M, threads, [&](int64_t m) {
    std::vector<double> X((size_t)ns * dsub);
    for (int64_t i = 0; i < ns; ++i)
      for (int j = 0; j < dsub; ++j) X[(size_t)i * dsub + j] = elem(i, static_cast<int>(m) * dsub + j);
    train_subspace(X.data(), ns, dsub, K, iters, u.data() + m * K, cbd.data() + (size_t)m * K * dsub);
  });
  for (size_t i = 0; i < cbd.size(); ++i)
    codebook_out[i] = static_cast<float>(dtype == ANN_U8 ? std::nearbyint(cbd[i]) : cbd[i]);
  // Encode: nearest centroid per subspace, lowest index on ties.
  const int64_t chunk = 4096;
  parallel_for((n + chunk - 1) / chunk, threads, [&](int64_t b) {
    const int64_t lo = b * chunk, hi = std::min(n, lo + chunk);
    if (dtype == ANN_U8) {
      const uint8_t* X = static_cast<const uint8_t*>(base);
      std::vector<int32_t> ci((size_t)K * dsub);
      for (int m = 0; m < M; ++m) {
        for (int c = 0; c < K * dsub; ++c) ci[c] = static_cast<int32_t>(codebook_out[(size_t)m * K * dsub + c]);
        for (int64_t i = lo; i < hi; ++i) {
          const uint8_t* x = X + i * d + m * dsub;
          int best = 0;
          int64_t bd = INT64_MAX;
          for (int c = 0; c < K; ++c) {
            int64_t s = 0;
            for (int j = 0; j < dsub; ++j) {
              const int64_t t = static_cast<int64_t>(x[j]) - ci[(size_t)c * dsub + j];
              s += t * t;
            }
            if (s < bd) {
              bd = s;
              best = c;
            }
          }
          codes_out[i * M + m] = static_cast<uint8_t>(best);
        }
      }
    } else {
      const float* X = static_cast<const float*>(base);
      for (int64_t i = lo; i < hi; ++i)
        for (int m = 0; m < M; ++m) {
          int best = 0;
          double bd = INFINITY;
          for (int c = 0; c < K; ++c) {
            double s = 0.0;
            for (int j = 0; j < dsub; ++j) {
              const double t = static_cast<double>(X[i * d + m * dsub + j]) -
                               static_cast<double>(codebook_out[((size_t)m * K + c) * dsub + j]);
              s += t * t;
            }
            if (s < bd) {
              bd = s;
              best = c;
            }
          }
          codes_out[i * M + m] = static_cast<uint8_t>(best);
        }
    }
  });
  return ANN_OK;
}
