/*
 * CPU oracle for the relaxed-pipeline graph search -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct C.  Only the test-suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it; the product library never does.
 * It shares no code, header or table with the CUDA path.
 *
 * Arithmetic: exact squared L2 in int64 for uint8 data, float64 for float32
 * data.  No blocking, fusion or reordering beyond what the definitions state.
 *
 * Contents (paper = arXiv 2507.10070, "FlashANNS"):
 *   orc_l2_*        squared Euclidean distance (definition).
 *   orc_knn         brute-force exact k nearest neighbours, ties by id
 *                   (ground truth for recall@10, Section "Evaluation Metrics").
 *   orc_medoid      entry node: point closest to the float64 mean (DiskANN's
 *                   medoid; the paper only says "entrance node").
 *   orc_pq_train    product-quantiser codebook: k-means++ seeding + Lloyd
 *                   iterations per subspace (PQ codes "in memory", Section
 *                   "Graph-Based Vector Indexing").  Pinned: K=1 closed
 *                   forms, hand-worked seeding at K=2 and K=3, hand-worked
 *                   empty clusters, and Lloyd's steps against scipy's
 *                   kmeans2 from the same start (float data).
 *   orc_pq_encode   nearest-centroid code per subspace, lowest index on ties.
 *   orc_vamana      Vamana graph (DiskANN's index, which the paper builds on):
 *                   random R-regular start, two passes (alpha=1, then alpha,
 *                   alpha compared with squared distances),
 *                   GreedySearch + RobustPrune + back-edges.  Pinned by
 *                   a closed form (points on a line, complete candidates,
 *                   alpha = 1: the path graph; alpha > 1: the ladder that
 *                   alpha on squared distances gives) and graph invariants.
 *   orc_search      best-first search with a dependency-relaxed fetch
 *                   schedule of depth D (Sections "Data-Dependency in
 *                   Traditional Best-First Search" and "Dependency Relaxed
 *                   Strategy"); D = 0 is the textbook synchronous search.
 *                   Pinned by hand traces at D = 0, 1, 2 and 4.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_U8 = 0, ORC_F32 = 1 };

/* ------------------------------------------------------------------------ */
/* Distances (definition of squared L2).                                     */
/* ------------------------------------------------------------------------ */

int64_t orc_l2_u8(const uint8_t* a, const uint8_t* b, int d) {
  int64_t s = 0;
  for (int i = 0; i < d; ++i) {
    int64_t t = (int64_t)a[i] - (int64_t)b[i];
    s += t * t;
  }
  return s;
}

double orc_l2_f32(const float* a, const float* b, int d) {
  double s = 0.0;
  for (int i = 0; i < d; ++i) {
    double t = (double)a[i] - (double)b[i];
    s += t * t;
  }
  return s;
}

/* Distance between row i of `base` and the vector q (same element type). */
static double dist_row(int dtype, const void* base, int64_t i, const void* q, int d) {
  if (dtype == ORC_U8)
    return (double)orc_l2_u8((const uint8_t*)base + i * d, (const uint8_t*)q, d);
  return orc_l2_f32((const float*)base + i * d, (const float*)q, d);
}

static const void* row_ptr(int dtype, const void* base, int64_t i, int d) {
  if (dtype == ORC_U8) return (const uint8_t*)base + i * d;
  return (const float*)base + i * d;
}

static double elem(int dtype, const void* v, int64_t j) {
  if (dtype == ORC_U8) return (double)((const uint8_t*)v)[j];
  return (double)((const float*)v)[j];
}

/* (dist, id) lexicographic order used everywhere. */
typedef struct {
  double dist;
  int32_t id;
} pair_t;

static int pair_less(pair_t a, pair_t b) {
  return a.dist < b.dist || (a.dist == b.dist && a.id < b.id);
}

static int pair_cmp(const void* x, const void* y) {
  pair_t a = *(const pair_t*)x, b = *(const pair_t*)y;
  if (pair_less(a, b)) return -1;
  if (pair_less(b, a)) return 1;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Simple static work split over threads.                                    */
/* ------------------------------------------------------------------------ */

typedef void (*range_fn)(void* ctx, int64_t lo, int64_t hi);
typedef struct {
  range_fn fn;
  void* ctx;
  int64_t lo, hi;
} range_job;

static void* range_thread(void* p) {
  range_job* j = (range_job*)p;
  j->fn(j->ctx, j->lo, j->hi);
  return NULL;
}

static void parallel_for(int64_t n, int nthreads, range_fn fn, void* ctx) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > n) nthreads = (int)(n > 0 ? n : 1);
  if (nthreads == 1) {
    fn(ctx, 0, n);
    return;
  }
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
  range_job* jobs = (range_job*)malloc(sizeof(range_job) * nthreads);
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].fn = fn;
    jobs[t].ctx = ctx;
    jobs[t].lo = n * t / nthreads;
    jobs[t].hi = n * (t + 1) / nthreads;
    pthread_create(&th[t], NULL, range_thread, &jobs[t]);
  }
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
}

/* ------------------------------------------------------------------------ */
/* Brute-force exact kNN.                                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
  int dtype;
  const void* base;
  int64_t n;
  int d;
  const void* queries;
  int k;
  int32_t* ids;
  double* dists;
} knn_ctx;

static void knn_range(void* p, int64_t lo, int64_t hi) {
  knn_ctx* c = (knn_ctx*)p;
  pair_t* best = (pair_t*)malloc(sizeof(pair_t) * (c->k + 1));
  for (int64_t qi = lo; qi < hi; ++qi) {
    const void* q = row_ptr(c->dtype, c->queries, qi, c->d);
    int cnt = 0;
    for (int64_t i = 0; i < c->n; ++i) {
      pair_t e = {dist_row(c->dtype, c->base, i, q, c->d), (int32_t)i};
      if (cnt == c->k && !pair_less(e, best[cnt - 1])) continue;
      int pos = cnt < c->k ? cnt : c->k - 1;  /* slot freed at the end */
      while (pos > 0 && pair_less(e, best[pos - 1])) {
        best[pos] = best[pos - 1];
        --pos;
      }
      best[pos] = e;
      if (cnt < c->k) ++cnt;
    }
    for (int j = 0; j < c->k; ++j) {
      c->ids[qi * c->k + j] = j < cnt ? best[j].id : -1;
      c->dists[qi * c->k + j] = j < cnt ? best[j].dist : INFINITY;
    }
  }
  free(best);
}

void orc_knn(int dtype, const void* base, int64_t n, int d, const void* queries,
             int64_t nq, int k, int32_t* ids, double* dists, int nthreads) {
  knn_ctx c = {dtype, base, n, d, queries, k, ids, dists};
  parallel_for(nq, nthreads, knn_range, &c);
}

/* ------------------------------------------------------------------------ */
/* Medoid: the point closest to the float64 mean, lowest id on ties.         */
/* ------------------------------------------------------------------------ */

int32_t orc_medoid(int dtype, const void* base, int64_t n, int d) {
  double* mean = (double*)calloc(d, sizeof(double));
  for (int64_t i = 0; i < n; ++i)
    for (int j = 0; j < d; ++j) mean[j] += elem(dtype, base, i * d + j);
  for (int j = 0; j < d; ++j) mean[j] /= (double)n;
  int32_t best = 0;
  double bestd = INFINITY;
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
      double t = elem(dtype, base, i * d + j) - mean[j];
      s += t * t;
    }
    if (s < bestd) {
      bestd = s;
      best = (int32_t)i;
    }
  }
  free(mean);
  return best;
}

/* ------------------------------------------------------------------------ */
/* Product quantisation.                                                     */
/* ------------------------------------------------------------------------ */

/* Squared distance between a dsub-slice of a data row and a centroid. */
static double sub_dist(int dtype, const void* X, int64_t i, int d, int off, int dsub,
                       const double* c) {
  double s = 0.0;
  for (int j = 0; j < dsub; ++j) {
    double t = elem(dtype, X, i * d + off + j) - c[j];
    s += t * t;
  }
  return s;
}

/*
 * k-means per subspace.  Seeding is k-means++ (Arthur & Vassilvitskii 2007):
 * the first centre is point floor(u[0]*ns); centre c is the first point whose
 * running sum of D(x)^2 exceeds u[c] * sum D(x)^2 (D = distance to the
 * nearest chosen centre), or point floor(u[c]*ns) if that sum is zero.
 * Then `iters` Lloyd iterations: assign to the nearest centroid (lowest index
 * on ties), replace each centroid by the mean of its points; an empty
 * cluster takes the point farthest from its own centroid (lowest id on ties;
 * each point is used once per iteration).  With round_int the final
 * centroids are rounded half-to-even to integers.
 * distortion_out (nullable, M x (iters+1)): mean squared quantisation error
 * of the assignment made at each iteration (entry iters = final centroids,
 * before rounding).
 */
void orc_pq_train(int dtype, const void* X, int64_t ns, int d, int M, int K, int iters,
                  const double* kpp_u, int round_int, float* codebook,
                  double* distortion_out) {
  int dsub = d / M;
  double* C = (double*)malloc(sizeof(double) * K * dsub);
  double* D2 = (double*)malloc(sizeof(double) * ns);
  int32_t* asg = (int32_t*)malloc(sizeof(int32_t) * ns);
  double* adist = (double*)malloc(sizeof(double) * ns);
  double* sum = (double*)malloc(sizeof(double) * K * dsub);
  int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * K);
  for (int m = 0; m < M; ++m) {
    int off = m * dsub;
    const double* u = kpp_u + (int64_t)m * K;
    /* k-means++ seeding */
    int64_t first = (int64_t)(u[0] * (double)ns);
    if (first >= ns) first = ns - 1;
    for (int j = 0; j < dsub; ++j) C[j] = elem(dtype, X, first * d + off + j);
    for (int64_t i = 0; i < ns; ++i) D2[i] = sub_dist(dtype, X, i, d, off, dsub, C);
    for (int c = 1; c < K; ++c) {
      double total = 0.0;
      for (int64_t i = 0; i < ns; ++i) total += D2[i];
      int64_t pick;
      if (total > 0.0) {
        double target = u[c] * total, run = 0.0;
        pick = ns - 1;
        for (int64_t i = 0; i < ns; ++i) {
          run += D2[i];
          if (run > target) {
            pick = i;
            break;
          }
        }
      } else {
        pick = (int64_t)(u[c] * (double)ns);
        if (pick >= ns) pick = ns - 1;
      }
      double* cc = C + (int64_t)c * dsub;
      for (int j = 0; j < dsub; ++j) cc[j] = elem(dtype, X, pick * d + off + j);
      for (int64_t i = 0; i < ns; ++i) {
        double t = sub_dist(dtype, X, i, d, off, dsub, cc);
        if (t < D2[i]) D2[i] = t;
      }
    }
    /* Lloyd iterations */
    for (int it = 0; it <= iters; ++it) {
      double tot = 0.0;
      for (int64_t i = 0; i < ns; ++i) {
        int best = 0;
        double bd = INFINITY;
        for (int c = 0; c < K; ++c) {
          double t = sub_dist(dtype, X, i, d, off, dsub, C + (int64_t)c * dsub);
          if (t < bd) {
            bd = t;
            best = c;
          }
        }
        asg[i] = best;
        adist[i] = bd;
        tot += bd;
      }
      if (distortion_out) distortion_out[(int64_t)m * (iters + 1) + it] = tot / (double)ns;
      if (it == iters) break;
      memset(sum, 0, sizeof(double) * K * dsub);
      memset(cnt, 0, sizeof(int64_t) * K);
      for (int64_t i = 0; i < ns; ++i) {
        cnt[asg[i]] += 1;
        for (int j = 0; j < dsub; ++j)
          sum[(int64_t)asg[i] * dsub + j] += elem(dtype, X, i * d + off + j);
      }
      for (int c = 0; c < K; ++c) {
        if (cnt[c] > 0) {
          for (int j = 0; j < dsub; ++j)
            C[(int64_t)c * dsub + j] = sum[(int64_t)c * dsub + j] / (double)cnt[c];
        } else {
          int64_t far = -1;
          double fd = -1.0;
          for (int64_t i = 0; i < ns; ++i)
            if (adist[i] > fd) {
              fd = adist[i];
              far = i;
            }
          adist[far] = -2.0; /* used */
          for (int j = 0; j < dsub; ++j)
            C[(int64_t)c * dsub + j] = elem(dtype, X, far * d + off + j);
        }
      }
    }
    for (int c = 0; c < K; ++c)
      for (int j = 0; j < dsub; ++j) {
        double v = C[(int64_t)c * dsub + j];
        if (round_int) v = nearbyint(v); /* default rounding: half to even */
        codebook[((int64_t)m * K + c) * dsub + j] = (float)v;
      }
  }
  free(C);
  free(D2);
  free(asg);
  free(adist);
  free(sum);
  free(cnt);
}

void orc_pq_encode(int dtype, const void* X, int64_t n, int d, int M, int K,
                   const float* codebook, uint8_t* codes) {
  int dsub = d / M;
  double* c = (double*)malloc(sizeof(double) * dsub);
  for (int64_t i = 0; i < n; ++i)
    for (int m = 0; m < M; ++m) {
      int best = 0;
      double bd = INFINITY;
      for (int k = 0; k < K; ++k) {
        for (int j = 0; j < dsub; ++j) c[j] = codebook[((int64_t)m * K + k) * dsub + j];
        double t = sub_dist(dtype, X, i, d, m * dsub, dsub, c);
        if (t < bd) {
          bd = t;
          best = k;
        }
      }
      codes[i * M + m] = (uint8_t)best;
    }
  free(c);
}

/* ------------------------------------------------------------------------ */
/* Search: best-first search with a dependency-relaxed fetch schedule.       */
/* ------------------------------------------------------------------------ */

typedef struct {
  int dtype;
  const void* base;   /* n x d full-precision vectors ("exact" distance) */
  int64_t n;
  int d;
  int R;
  const int32_t* adj; /* n x R neighbour ids, -1 padded */
  int M;              /* 0: navigate on exact distance; >0: on PQ codes */
  const float* codebook;
  const uint8_t* codes;
  int32_t entry;
  const double* navv;  /* n x d navigation vectors (float64), or NULL */
  int rerank;          /* > 0: results = exact rerank of the `rerank` expanded nodes nearest by nav */
} index_t;

/* Navigation distance of node w: the squared distance between the query and
 * w's vector as the navigating representation stores it -- the decoded PQ
 * reconstruction when M > 0, the full-precision vector otherwise. */
static double nav_dist(const index_t* ix, const void* q, int32_t w) {
  if (ix->navv) {
    double s = 0.0;
    for (int j = 0; j < ix->d; ++j) {
      double t = elem(ix->dtype, q, j) - ix->navv[(int64_t)w * ix->d + j];
      s += t * t;
    }
    return s;
  }
  if (ix->M == 0) return dist_row(ix->dtype, ix->base, w, q, ix->d);
  int dsub = ix->d / ix->M;
  double s = 0.0;
  for (int m = 0; m < ix->M; ++m) {
    const float* c = ix->codebook + ((int64_t)m * 256 + ix->codes[(int64_t)w * ix->M + m]) * dsub;
    for (int j = 0; j < dsub; ++j) {
      double t = elem(ix->dtype, q, m * dsub + j) - (double)c[j];
      s += t * t;
    }
  }
  return s;
}

typedef struct {
  pair_t key;
  int selected; /* chosen for a fetch already (in flight or expanded) */
} cand_t;

/*
 * One query.  The candidate list holds at most L (nav distance, id) entries
 * in ascending order; `selected` marks entries already chosen for a fetch.
 * Each iteration:
 *   select  v = first unselected entry (the heap root), mark it, issue its
 *           fetch (push on a FIFO of in-flight fetches);
 *   expand  if more than D fetches are in flight, or nothing was selectable
 *           and something is in flight: take the oldest fetch u, put
 *           (exact(u), u) in the result set, and insert every neighbour of u
 *           not seen before into the list (by nav distance), keep the L best;
 *   stop    when nothing is selectable and nothing is in flight.
 * With D = 0 each fetch is expanded in the iteration that issued it: the
 * textbook best-first search.  With D = k the node selected at step i has
 * seen the expansions of steps up to i-1-k only.
 * Returns the number of expansions; writes the k best of the result set by
 * (exact distance, id), padded with (-1, +inf).  If `expanded_out` is given
 * it receives the expansion sequence (up to expanded_cap entries).
 */
static int search_one(const index_t* ix, const void* q, int k, int L, int D,
                      unsigned char* visited, cand_t* list, int32_t* fifo,
                      pair_t** results, int64_t* results_cap, int32_t* ids_out,
                      double* dists_out, int32_t* expanded_out, int expanded_cap,
                      int32_t* nvisited_out) {
  int len = 0, fhead = 0, fcount = 0, steps = 0, nvisited = 1;
  int64_t nres = 0;
  memset(visited, 0, (size_t)ix->n);
  list[0].key.dist = nav_dist(ix, q, ix->entry);
  list[0].key.id = ix->entry;
  list[0].selected = 0;
  len = 1;
  visited[ix->entry] = 1;
  for (;;) {
    int v = -1;
    for (int i = 0; i < len; ++i)
      if (!list[i].selected) {
        v = i;
        break;
      }
    if (v >= 0) {
      list[v].selected = 1;
      fifo[(fhead + fcount) % (D + 1)] = list[v].key.id;
      ++fcount;
    }
    if (fcount > D || (v < 0 && fcount > 0)) {
      int32_t u = fifo[fhead];
      fhead = (fhead + 1) % (D + 1);
      --fcount;
      if (expanded_out && steps < expanded_cap) expanded_out[steps] = u;
      ++steps;
      if (nres == *results_cap) {
        *results_cap *= 2;
        *results = (pair_t*)realloc(*results, sizeof(pair_t) * (*results_cap));
      }
      /* with a rerank, the result set first ranks expanded nodes by navigation */
      (*results)[nres].dist = ix->rerank > 0 ? nav_dist(ix, q, u) : dist_row(ix->dtype, ix->base, u, q, ix->d);
      (*results)[nres].id = u;
      ++nres;
      const int32_t* nb = ix->adj + (int64_t)u * ix->R;
      for (int j = 0; j < ix->R; ++j) {
        int32_t w = nb[j];
        if (w < 0) break;
        if (visited[w]) continue;
        visited[w] = 1;
        ++nvisited;
        cand_t e;
        e.key.dist = nav_dist(ix, q, w);
        e.key.id = w;
        e.selected = 0;
        /* sorted insertion; an entry pushed past position L falls off */
        int pos = len;
        while (pos > 0 && pair_less(e.key, list[pos - 1].key)) --pos;
        if (pos >= L) continue;
        int last = len < L ? len : L - 1;
        for (int t = last; t > pos; --t) list[t] = list[t - 1];
        list[pos] = e;
        if (len < L) ++len;
      }
    } else if (v < 0) {
      break;
    }
  }
  qsort(*results, (size_t)nres, sizeof(pair_t), pair_cmp);
  if (ix->rerank > 0) {
    /* exact distances of the `rerank` best by navigation, ranked again */
    if (nres > ix->rerank) nres = ix->rerank;
    for (int64_t i = 0; i < nres; ++i)
      (*results)[i].dist = dist_row(ix->dtype, ix->base, (*results)[i].id, q, ix->d);
    qsort(*results, (size_t)nres, sizeof(pair_t), pair_cmp);
  }
  if (nvisited_out) *nvisited_out = nvisited;
  for (int j = 0; j < k; ++j) {
    ids_out[j] = j < nres ? (*results)[j].id : -1;
    dists_out[j] = j < nres ? (*results)[j].dist : INFINITY;
  }
  return steps;
}

typedef struct {
  const index_t* ix;
  const void* queries;
  int k, L, D;
  int32_t* ids;
  double* dists;
  int32_t* steps;
  int32_t* expanded;
  int expanded_cap;
  int32_t* nvisited;
} search_ctx;

static void search_range(void* p, int64_t lo, int64_t hi) {
  search_ctx* c = (search_ctx*)p;
  const index_t* ix = c->ix;
  unsigned char* visited = (unsigned char*)malloc((size_t)ix->n);
  cand_t* list = (cand_t*)malloc(sizeof(cand_t) * (c->L + 1));
  int32_t* fifo = (int32_t*)malloc(sizeof(int32_t) * (c->D + 1));
  int64_t cap = 1024;
  pair_t* res = (pair_t*)malloc(sizeof(pair_t) * cap);
  for (int64_t qi = lo; qi < hi; ++qi) {
    const void* q = row_ptr(ix->dtype, c->queries, qi, ix->d);
    int s = search_one(ix, q, c->k, c->L, c->D, visited, list, fifo, &res, &cap,
                       c->ids + qi * c->k, c->dists + qi * c->k,
                       c->expanded ? c->expanded + qi * c->expanded_cap : NULL,
                       c->expanded_cap, c->nvisited ? c->nvisited + qi : NULL);
    if (c->steps) c->steps[qi] = s;
  }
  free(visited);
  free(list);
  free(fifo);
  free(res);
}

int orc_search(int dtype, const void* base, int64_t n, int d, int R, const int32_t* adj,
               int M, const float* codebook, const uint8_t* codes, int32_t entry,
               const void* queries, int64_t nq, int k, int L, int D, int32_t* ids,
               double* dists, int32_t* steps, int32_t* expanded, int expanded_cap,
               int32_t* nvisited, const double* navv, int rerank, int nthreads) {
  if (k < 1 || L < k || D < 0 || n < 1 || entry < 0 || entry >= n) return -1;
  if (M > 0 && d % M != 0) return -1;
  index_t ix = {dtype, base, n, d, R, adj, M, codebook, codes, entry, navv, rerank};
  search_ctx c = {&ix, queries, k, L, D, ids, dists, steps, expanded, expanded_cap, nvisited};
  parallel_for(nq, nthreads, search_range, &c);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Vamana graph (DiskANN): GreedySearch + RobustPrune, two passes.           */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t* ids;
  int deg;
} nbrs_t;

/* RobustPrune(p, V, alpha, R): repeatedly keep the candidate p* closest to p
 * and drop every candidate p' with alpha * d2(p*, p') <= d2(p, p'), where d2
 * is the SQUARED distance (the convention of DiskANN's public implementation;
 * on the clustered synthetic workloads alpha on plain distances leaves every
 * cluster an island).  Writes <= R ids. */
static int robust_prune(int dtype, const void* base, int d, int32_t p, int32_t* cand,
                        int ncand, double alpha, int R, int32_t* out) {
  pair_t* v = (pair_t*)malloc(sizeof(pair_t) * (ncand > 0 ? ncand : 1));
  int nv = 0;
  const void* xp = row_ptr(dtype, base, p, d);
  for (int i = 0; i < ncand; ++i) {
    if (cand[i] == p) continue;
    int dup = 0;
    for (int j = 0; j < nv; ++j)
      if (v[j].id == cand[i]) dup = 1;
    if (dup) continue;
    v[nv].id = cand[i];
    v[nv].dist = dist_row(dtype, base, cand[i], xp, d);
    ++nv;
  }
  qsort(v, (size_t)nv, sizeof(pair_t), pair_cmp);
  unsigned char* gone = (unsigned char*)calloc((size_t)(nv > 0 ? nv : 1), 1);
  int nout = 0;
  double a2 = alpha;
  for (int i = 0; i < nv && nout < R; ++i) {
    if (gone[i]) continue;
    out[nout++] = v[i].id;
    const void* xs = row_ptr(dtype, base, v[i].id, d);
    for (int j = i + 1; j < nv; ++j) {
      if (gone[j]) continue;
      double dsj = dist_row(dtype, base, v[j].id, xs, d);
      if (a2 * dsj <= v[j].dist) gone[j] = 1;
    }
  }
  free(v);
  free(gone);
  return nout;
}

/* GreedySearch on the graph under construction: synchronous best-first search
 * on exact distances with list size L; returns the expanded (visited) set. */
static int greedy_visited(int dtype, const void* base, int64_t n, int d, nbrs_t* g,
                          int32_t entry, const void* q, int L, unsigned char* seen,
                          cand_t* list, int32_t* out, int out_cap) {
  int len = 1, nout = 0;
  memset(seen, 0, (size_t)n);
  list[0].key.dist = dist_row(dtype, base, entry, q, d);
  list[0].key.id = entry;
  list[0].selected = 0;
  seen[entry] = 1;
  for (;;) {
    int v = -1;
    for (int i = 0; i < len; ++i)
      if (!list[i].selected) {
        v = i;
        break;
      }
    if (v < 0) break;
    list[v].selected = 1;
    int32_t u = list[v].key.id;
    if (nout < out_cap) out[nout++] = u;
    for (int j = 0; j < g[u].deg; ++j) {
      int32_t w = g[u].ids[j];
      if (seen[w]) continue;
      seen[w] = 1;
      cand_t e;
      e.key.dist = dist_row(dtype, base, w, q, d);
      e.key.id = w;
      e.selected = 0;
      int pos = len;
      while (pos > 0 && pair_less(e.key, list[pos - 1].key)) --pos;
      if (pos >= L) continue;
      int last = len < L ? len : L - 1;
      for (int t = last; t > pos; --t) list[t] = list[t - 1];
      list[pos] = e;
      if (len < L) ++len;
    }
  }
  return nout;
}

/*
 * Sequential Vamana.  init_adj: n x init_deg random start graph; order: the
 * insertion order (a permutation of 0..n-1).  Pass 1 prunes with alpha = 1,
 * pass 2 with `alpha`.  For node p: V = expanded set of GreedySearch(entry,
 * x_p, Lb); N(p) = RobustPrune(p, V u N(p)); for each j in N(p) add the back
 * edge j -> p, pruning N(j) u {p} when it would exceed R.  adj_out: n x R,
 * -1 padded.
 */
int orc_vamana(int dtype, const void* base, int64_t n, int d, int R, double alpha, int Lb,
               int32_t entry, const int32_t* order, const int32_t* init_adj, int init_deg,
               int32_t* adj_out) {
  if (R < 1 || Lb < 1 || n < 2) return -1;
  nbrs_t* g = (nbrs_t*)malloc(sizeof(nbrs_t) * n);
  for (int64_t i = 0; i < n; ++i) {
    g[i].ids = (int32_t*)malloc(sizeof(int32_t) * R);
    g[i].deg = 0;
    for (int j = 0; j < init_deg && g[i].deg < R; ++j) g[i].ids[g[i].deg++] = init_adj[i * init_deg + j];
  }
  unsigned char* seen = (unsigned char*)malloc((size_t)n);
  cand_t* list = (cand_t*)malloc(sizeof(cand_t) * (Lb + 1));
  int vcap = (int)n; /* the expanded set of one search is at most n */
  int32_t* V = (int32_t*)malloc(sizeof(int32_t) * ((int64_t)vcap + R + 1));
  int32_t* pruned = (int32_t*)malloc(sizeof(int32_t) * R);
  for (int pass = 0; pass < 2; ++pass) {
    double a = pass == 0 ? 1.0 : alpha;
    for (int64_t t = 0; t < n; ++t) {
      int32_t p = order[t];
      const void* xp = row_ptr(dtype, base, p, d);
      int nv = greedy_visited(dtype, base, n, d, g, entry, xp, Lb, seen, list, V, vcap);
      for (int j = 0; j < g[p].deg; ++j) V[nv++] = g[p].ids[j];
      int np = robust_prune(dtype, base, d, p, V, nv, a, R, pruned);
      memcpy(g[p].ids, pruned, sizeof(int32_t) * np);
      g[p].deg = np;
      for (int j = 0; j < np; ++j) {
        int32_t q = pruned[j];
        int have = 0;
        for (int t2 = 0; t2 < g[q].deg; ++t2)
          if (g[q].ids[t2] == p) have = 1;
        if (have) continue;
        if (g[q].deg < R) {
          g[q].ids[g[q].deg++] = p;
        } else {
          int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (R + 1));
          int32_t* out = (int32_t*)malloc(sizeof(int32_t) * R);
          memcpy(tmp, g[q].ids, sizeof(int32_t) * R);
          tmp[R] = p;
          int nq2 = robust_prune(dtype, base, d, q, tmp, R + 1, a, R, out);
          memcpy(g[q].ids, out, sizeof(int32_t) * nq2);
          g[q].deg = nq2;
          free(tmp);
          free(out);
        }
      }
    }
  }
  for (int64_t i = 0; i < n; ++i) {
    for (int j = 0; j < R; ++j) adj_out[i * R + j] = j < g[i].deg ? g[i].ids[j] : -1;
    free(g[i].ids);
  }
  free(g);
  free(seen);
  free(list);
  free(V);
  free(pruned);
  return 0;
}
