/*
 * ann.h -- C ABI of the B300 relaxed-pipeline graph search library (libann).
 *
 * The library runs best-first (beam) search over a Vamana-style proximity
 * graph for batches of queries on one GPU (arXiv 2507.10070, "FlashANNS").
 * Navigation distances come from product-quantisation (PQ) codes held in HBM
 * (Section "Graph-Based Vector Indexing", phases 1-2).  The full-precision
 * node blocks -- vector, degree and neighbour ids -- stay in a slower tier,
 * host pinned memory by default, which the GPU reads over PCIe itself.  Node
 * blocks are fetched through the dependency-relaxed pipeline: the node fetched
 * at step i is chosen before the neighbour distances of up to `depth` earlier
 * steps are in (Section "Dependency Relaxed Strategy").  Every query runs on
 * one warp, which issues and waits for its own fetches only; no barrier spans
 * queries (Section "Resource-Efficient Query-Grained Concurrent I/O Stack").
 *
 * Conventions for every entry point:
 *  - The return value is an ann_status; nothing throws or aborts across the
 *    ABI.  On failure ann_last_error() gives a message (per host thread).
 *  - The caller owns every buffer it passes.  "host" means ordinary host
 *    memory (pinned or pageable); "device" means memory of the current CUDA
 *    device (e.g. a torch tensor's data_ptr()).
 *  - Distances are squared Euclidean (L2^2).  Ties are broken by lower id.
 *  - uint8 data is exact: distances are integers (< 2^24 for d <= 256), so
 *    results are bit-exact; float32 data uses FP32 arithmetic.
 */
#ifndef ANN_H_
#define ANN_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ANN_OK = 0,
  ANN_EINVAL = -1,   /* bad argument or malformed index data */
  ANN_ENOMEM = -2,   /* allocation failed */
  ANN_ECUDA = -3,    /* a CUDA runtime call failed */
  ANN_ETIMEOUT = -4, /* a bounded device-side wait ran out */
  ANN_EBUSY = -5,    /* the index is in use by another search */
  ANN_EIO = -6       /* file could not be read or written */
} ann_status;

typedef enum { ANN_U8 = 0, ANN_F32 = 1 } ann_dtype;

/* How navigation distances are computed (ann_graph_desc.nav). */
typedef enum {
  ANN_NAV_AUTO = 0, /* PQ codes if M > 0, otherwise the vectors themselves */
  ANN_NAV_BF16 = 1, /* BF16 copies of float32 vectors, FP32 accumulation */
  ANN_NAV_FP8 = 2   /* FP8-E4M3 copies of float32 vectors * nav_scale, FP32 accumulation */
} ann_nav;

/* Where the node blocks (full vector + adjacency) live. */
typedef enum {
  ANN_TIER_HOST_PINNED = 0, /* host pinned memory read by the GPU over PCIe (default) */
  ANN_TIER_HBM = 1          /* device memory */
} ann_tier;

typedef struct ann_index ann_index; /* opaque, owned by the library */

/*
 * Index description handed to ann_load_graph.  All pointers are host memory;
 * the library copies what it needs, so the caller may free them on return.
 *
 * Navigation mode:
 *  - M > 0: PQ navigation.  dtype must be ANN_U8, d % M == 0, (d/M) % 4 == 0,
 *    M % 16 == 0, M <= 64, and every codebook value an integer in [0, 255]
 *    (this makes the asymmetric distance an exact integer).  Node blocks go
 *    to `tier`; codes and codebook go to HBM.
 *  - M == 0: exact navigation; vectors and adjacency go to HBM (tier must be
 *    ANN_TIER_HBM).  dtype ANN_U8 or ANN_F32, d % 4 == 0.
 *  - Precision variants (dtype ANN_F32, tier ANN_TIER_HBM): navigation on
 *    compressed copies -- nav = ANN_NAV_BF16 or ANN_NAV_FP8 with M == 0, or
 *    float PQ with M > 0 (M % 16 == 0, M <= 64, d % M == 0, any float
 *    codebook) -- followed by an exact FP32 rerank of the top
 *    rerank_mult * k expanded candidates (at most 512, at most L).
 * Limits: 1 <= n < 2^31, 4 <= d <= 512, 1 <= R <= 128, 0 <= entry < n; every
 * adjacency id is -1 or in [0, n) and a row ends at its first -1.
 */
typedef struct {
  int64_t n;             /* number of base vectors */
  int32_t d;             /* dimension */
  int32_t dtype;         /* ann_dtype */
  int32_t R;             /* adjacency row length (maximum out-degree) */
  int32_t entry;         /* entry node of every search (the medoid) */
  const void* vectors;   /* n*d elements of dtype, row-major */
  const int32_t* adj;    /* n*R neighbour ids, -1 padded */
  int32_t M;             /* PQ subspaces; 0 = exact navigation */
  const float* codebook; /* M*256*(d/M): centroid c of subspace m at (m*256+c)*(d/M) */
  const uint8_t* codes;  /* n*M PQ codes */
  int32_t tier;          /* ann_tier of the node blocks */
  int32_t nav;           /* ann_nav (0 = ANN_NAV_AUTO) */
  float nav_scale;       /* ANN_NAV_FP8: values are encoded as x * nav_scale (> 0) */
  int32_t rerank_mult;   /* precision variants: rerank the top rerank_mult*k (0 means 4) */
  const int32_t* id_map; /* NULL, or n ids: the caller's id of each stored node.  Searches
                            report id_map[node] instead of the node's position (any int32
                            values; -1 still pads missing results).  Set by layouts that
                            store nodes in another order, e.g. ann_reorder_graph's. */
} ann_graph_desc;

/* Per-query outputs of a search (each pointer may be NULL).  Memory kind as
 * the ids/dists of the same call (host for ann_search, device for
 * ann_search_dev). */
typedef struct {
  int32_t* steps;   /* [nq] node blocks fetched and expanded (search steps) */
  int32_t* status;  /* [nq] ANN_OK, or ANN_ETIMEOUT (kernel-grained ablation only) */
  int64_t* t_begin; /* [nq] device global timer (ns) when the query started */
  int64_t* t_end;   /* [nq] device global timer (ns) when it finished */
} ann_trace;

/* Totals of one ann_search call, or of the ann_search_dev calls since the
 * previous ann_sync. */
typedef struct {
  int64_t queries;       /* queries searched */
  int64_t expansions;    /* node blocks fetched and expanded */
  int64_t bytes_per_expansion; /* bytes read from the node-block tier per expansion:
                                  the vector and the neighbour ids (PQ mode), or
                                  one adjacency row (exact navigation) */
  int32_t n_failed;      /* queries whose status is not ANN_OK */
  int32_t first_failed;  /* index of the first failed query, or -1 */
  float kernel_ms;       /* device time of the last search kernel (ann_search only) */
} ann_search_stats;

/* Message of the last failed call on this host thread ("" if none). */
const char* ann_last_error(void);

/* Library version string. */
const char* ann_version(void);

/*
 * Build an index from a description (see ann_graph_desc).  Validates every
 * field and adjacency id (ANN_EINVAL), allocates the node-block tier
 * (cudaHostAlloc, mapped) or HBM copies (ANN_ENOMEM / ANN_ECUDA on failure)
 * and uploads.  Node block layout: [vector: d*elt bytes][R int32 neighbour
 * ids, -1 padded][uint32 degree][zero pad to a multiple of 128 bytes].
 * A search step fetches only the vector and the ids (the first d*elt + 4R
 * bytes, rounded up to 16): the ids are -1 padded, so the degree is implied.
 * On success *out owns all of it until ann_free.  Uses the current device.
 */
int ann_load_graph(ann_index** out, const ann_graph_desc* desc);

/* Write / read an index as one file (header, vectors, adjacency, codebook,
 * codes, and the id map if the description has one).  ann_load_graph_file
 * returns ANN_EIO on unreadable or truncated files, then validates like
 * ann_load_graph, placing blocks in `tier`. */
int ann_save_graph_file(const char* path, const ann_graph_desc* desc);
int ann_load_graph_file(ann_index** out, const char* path, int32_t tier);

/* Release everything an index owns.  NULL is ignored. */
void ann_free(ann_index* index);

/* Bytes of one node block of this index, and the number of nodes. */
int64_t ann_index_block_bytes(const ann_index* index);
int64_t ann_index_size(const ann_index* index);

/*
 * Warps per query of later ann_search / ann_search_dev calls on this index:
 * 1 (default) or a warp group of 2 or 4 (PQ navigation on uint8 data only,
 * ANN_EINVAL otherwise).  The group shares one query's lookup table, list,
 * fetch ring and visited set; warp 0 runs the relaxed pipeline (selection,
 * fetches, waits) exactly as a single warp does, and for each expansion the
 * warps split the node's neighbours and the merge of the new candidates.
 * Results, step counts and the schedule do not depend on the setting, only
 * the time a step takes.  The serving loop, the kernel-grained ablation and
 * ann_search_dev_noalloc always use one warp per query.  ANN_EBUSY while a
 * search runs on the index.
 */
int ann_set_warps_per_query(ann_index* index, int32_t warps);

/*
 * Batched search, host buffers (the end-to-end call).
 *  queries: host, nq*d elements of the index's dtype.
 *  k: results per query, 1 <= k <= min(L, 256).   L: candidate list size, L <= 16384.
 *  depth: relaxed-pipeline depth 0..4 (fetches in flight beyond the one being
 *    expanded); 0 is synchronous best-first search.
 *  ids, dists: host, nq*k; the k expanded nodes with the smallest exact
 *    distance, ascending by (distance, id); padded with id -1 and +inf when
 *    fewer than k nodes were expanded.
 *  trace: host pointers, may be NULL.  stats: may be NULL.
 * Blocks until done.  One search at a time per index (ANN_EBUSY otherwise).
 * Each resident query keeps its visited set as one bit per node of the index
 * (n/8 bytes of device scratch per resident query), so it cannot overflow.
 */
int ann_search(ann_index* index, const void* queries, int64_t nq, int32_t k, int32_t L,
               int32_t depth, int32_t* ids, float* dists, const ann_trace* trace,
               ann_search_stats* stats);

/*
 * Same search with device buffers, enqueued on `stream` (a cudaStream_t, NULL
 * for the legacy default stream); returns once the kernels are launched.
 * Argument errors are reported at once; per-query failures are recorded on
 * the device and reported by ann_sync.  Calls on one index must not overlap
 * on the device (the index's scratch is shared).
 */
int ann_search_dev(ann_index* index, const void* queries, int64_t nq, int32_t k, int32_t L,
                   int32_t depth, int32_t* ids, float* dists, const ann_trace* trace,
                   void* stream);

/*
 * Kernel-grained I/O: the ablation of the paper's query-grained I/O stack
 * (Section "Resource-Efficient Query-Grained Concurrent I/O Stack", which
 * compares against CAM, where the kernel waits for every request of the
 * batch).  Same arguments, kernel and per-query results as ann_search_dev,
 * but launched cooperatively (every block resident) and with a grid-wide
 * barrier after each fetch wait: no query expands a node until the fetches
 * of every resident warp in that round have arrived.  The barrier's waits
 * are bounded; if one runs out, the queries still running report
 * ANN_ETIMEOUT, the queries not started yet are left unwritten, and the
 * next ann_sync returns ANN_ETIMEOUT; the index stays usable.  (Tests force
 * this path with the environment variable ANN_TEST_STALL_ROUNDS=1.)  For
 * measurement only -- query-grained I/O (ann_search_dev) is never slower.
 */
int ann_search_dev_kernel_grained(ann_index* index, const void* queries, int64_t nq, int32_t k,
                                  int32_t L, int32_t depth, int32_t* ids, float* dists,
                                  const ann_trace* trace, void* stream);

/*
 * CPU-agent I/O: the paper's I/O stack as it describes it (Section
 * "Resource-Efficient Query-Grained Concurrent I/O Stack": each warp writes
 * its block address into a request array in mapped pinned host memory, a CPU
 * agent serves the requests, and the warp checks a completion signal before
 * it uses the data), as an ablation against the warps reading node blocks
 * themselves (ann_search).  Same arguments and results as ann_search (host
 * buffers, k, L, depth; identical ids, distances and expansion counts), for a
 * PQ index with its node blocks in host pinned memory.
 *  agent_threads: host threads serving the requests (0..64); each owns a
 *    fixed share of the warps' request entries and copies a requested block
 *    into that entry's staging slot (mapped pinned memory), then writes the
 *    entry's completion word.  The warp then reads the block from the slot.
 *  wait_us: bound on one wait for a completion (1 .. 6e7); past it the query
 *    stops, the call returns ANN_ETIMEOUT, and the index stays usable.
 *  seconds (may be NULL): host wall time from the launch to the kernel's end.
 * Blocking; one warp per query whatever ann_set_warps_per_query set.
 */
int ann_search_cpu_agent(ann_index* index, const void* queries, int64_t nq, int32_t k, int32_t L,
                         int32_t depth, int32_t agent_threads, int64_t wait_us, int32_t* ids,
                         float* dists, ann_search_stats* stats, double* seconds);

/* Wait for `stream`, then report (and reset) the totals and failures of the
 * ann_search_dev calls since the previous ann_sync. */
int ann_sync(ann_index* index, void* stream, ann_search_stats* stats);

/*
 * ann_search_dev without any allocation at call time.  The paper has no
 * counterpart: this exists for callers that must not call cudaMalloc while
 * they search -- a serving thread with a latency budget (cudaMalloc may
 * synchronise the device), a process whose device memory is reserved up
 * front by its own pool, or code that must not grow its footprint after
 * start-up.  The search is the same kernel and gives the same results; its
 * scratch (visited bitsets, their clear logs, counters) lives in one 16 MiB
 * device array inside the library, which every GPU that loads the library
 * holds until the process exits.  The caller still passes queries and outputs
 * (device memory, as for ann_search_dev) and loads the index beforehand.
 *  - Limit: a call must fit the scratch of at least 32 warps.  A warp
 *    needs one bit per node of the index (rounded up to 128 bytes) and a
 *    32 KiB clear log, so indexes above 3,931,136 nodes are rejected with
 *    ANN_EINVAL.  At most 16 MiB / (per-warp scratch) warps run, fewer than
 *    ann_search_dev may use, so throughput is lower.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress with that device current).  With CUDA's lazy
 *    module loading (the default) that lookup is also what loads the
 *    library's device code on the device and places the 16 MiB array there,
 *    so the first call may allocate device memory: make it once per device
 *    at start-up, before any stream capture and before the phase that must
 *    not allocate (a call with nq = 0 does only this set-up).
 *  - The address is kept for the life of the process: do not use this entry
 *    point after cudaDeviceReset or after the device's primary context was
 *    destroyed and created again.
 *  - Every call shares the one array and zeroes what must start at zero, so
 *    calls that overlap on the GPU race: serialise them (one stream, or
 *    events).
 *  - Enqueued on `stream`; returns once launched.  Per-query failures are
 *    reported only through trace->status (device memory, may be NULL).
 */
int ann_search_dev_noalloc(ann_index* index, const void* queries, int64_t nq, int32_t k, int32_t L,
                           int32_t depth, int32_t* ids, float* dists, const ann_trace* trace,
                           void* stream);

/* ------------------------------------------------------------------------
 * Serving: a continuous-batching request loop over one index.
 *
 * The paper evaluates batched search; its I/O stack lets every query proceed
 * independently of the others (Section "Resource-Efficient Query-Grained
 * Concurrent I/O Stack": no synchronisation across queries).  This loop puts
 * that property to work for requests that arrive over time: each request is
 * a batch of queries with its own k and L; its queries become work items in
 * a ring of `slots` staging entries (mapped pinned host memory), admitted
 * while slots are free.  A persistent kernel keeps one query per resident
 * warp and a warp that finishes takes the next item of any request, so new
 * requests start as warps free up and overlap with running ones on the
 * device.  Results are written to host memory by the kernel.  A query's
 * results do not depend on what else is in flight.
 * ------------------------------------------------------------------------ */
typedef struct ann_server ann_server; /* opaque */

typedef struct {
  int32_t max_L;        /* largest L a request may use (sets the shared-memory layout), <= 16384 */
  int32_t max_k;        /* largest k, <= min(max_L, 256) */
  int32_t depth;        /* relaxed-pipeline depth 0..4 used for every query */
  int32_t slots;        /* staging ring size: queries queued or in flight at once */
  int32_t idle_exit_us; /* the kernel returns after this long without work (bounded polling);
                           it is relaunched when new work arrives */
} ann_serve_cfg;

typedef struct {
  int64_t queries;     /* queries of the request */
  int64_t expansions;  /* node blocks fetched for them */
  int32_t n_failed;    /* queries whose status is not ANN_OK */
  int64_t device_ns;   /* device time from the first query's start to the last one's end */
} ann_serve_result;

typedef struct {
  int64_t launches;       /* serving-kernel launches so far */
  int64_t published;      /* queries admitted so far */
  int64_t retired;        /* queries whose results were collected */
  int64_t resident_warps; /* queries the kernel works on at once */
  int32_t running;        /* 1 if the kernel is running now */
} ann_serve_counters;

/* Create a server (allocates the staging ring, scratch and a host launcher
 * thread; uses the current device).  The index must outlive the server. */
int ann_serve_create(ann_index* index, const ann_serve_cfg* cfg, ann_server** out);

/* Admit a request of nq queries (host memory, the index's dtype), 1 <= k <=
 * max_k, k <= L <= max_L.  Copies the queries; returns ANN_EBUSY if fewer
 * than nq staging slots are free (nothing is admitted then).  Thread-safe. */
int ann_serve_submit(ann_server* server, const void* queries, int64_t nq, int32_t k, int32_t L,
                     uint64_t* req_id);

/* Wait up to timeout_us (0: just check) for a request.  On completion copies
 * its nq*k ids and dists to host memory (same layout as ann_search), fills
 * `info` (may be NULL), frees its slots and forgets the request; returns
 * ANN_ETIMEOUT if it is not done yet (call again). */
int ann_serve_poll(ann_server* server, uint64_t req_id, int32_t* ids, float* dists,
                   int64_t timeout_us, ann_serve_result* info);

/* Wait up to timeout_us (0: just check) until at least one admitted request
 * is complete; writes up to `max` ids of complete, not yet collected requests
 * to req_ids and their number to *n_ready (0 on timeout).  Collect each with
 * ann_serve_poll (it returns at once). */
int ann_serve_poll_any(ann_server* server, uint64_t* req_ids, int32_t max, int64_t timeout_us,
                       int32_t* n_ready);

int ann_serve_stats(ann_server* server, ann_serve_counters* out);

/* Stop the kernel (after the queries in progress) and free everything. */
void ann_serve_destroy(ann_server* server);

/*
 * Train a product quantiser and encode the base (index-construction tooling;
 * runs on host threads).  The training sample is the first min(n, n_train)
 * rows.  Per subspace: k-means++ seeding (kpp_uniforms[m*256 + c] is the
 * uniform draw for centre c; NULL derives the draws from `seed`), then
 * `iters` Lloyd iterations (empty clusters take the point farthest from its
 * centroid).  For ANN_U8 the centroids are rounded half-to-even to integers.
 * codebook_out: host, M*256*(d/M) floats.  codes_out: host, n*M bytes.
 * nthreads <= 0 uses every hardware thread.
 */
int ann_build_pq(const void* base, int32_t dtype, int64_t n, int32_t d, int32_t M,
                 int64_t n_train, int32_t iters, const double* kpp_uniforms, uint64_t seed,
                 float* codebook_out, uint8_t* codes_out, int32_t nthreads);

/*
 * PQ encoding on the GPU (index-construction tooling): the code of every
 * vector and subspace is its nearest centroid, lowest index on ties -- the
 * same codes as ann_build_pq's encoder.  uint8 data with an integer
 * codebook in [0,255] (as ann_build_pq trains for uint8), (d/M) % 4 == 0.
 * base, codebook, codes_out: host buffers.  Uses the current device.
 */
int ann_pq_encode_gpu(const void* base, int32_t dtype, int64_t n, int32_t d, int32_t M,
                      const float* codebook, uint8_t* codes_out);

/*
 * Storage order of the node blocks (index-construction tooling; host
 * threads).  The paper places nodes on SSD pages; on this system the
 * storage tier is host memory that the GPU reads through an address
 * translation with a 64 KB granule, whose miss rate (about 65 million per
 * second) caps random 384-byte reads over tens of GB at half the PCIe link.
 * Storing nodes in breadth-first order from the entry node puts a node and
 * the neighbours it discovers in the same 64 KB pages, so successive
 * expansions of a query reuse translations.
 *
 * Computes the breadth-first order from `entry` over the rows of `adj`
 * (neighbours in row order, a row ending at its first -1; when the queue
 * runs dry, breadth-first again from the lowest id not yet placed) and
 * writes the index in that order: base_out row i = base row old_of_new[i],
 * codes_out likewise (codes may be NULL when M == 0), adj_out row i = the
 * row of old_of_new[i] with every id j replaced by its new position, and
 * *entry_out = the entry's new position (0).  Load the result with
 * id_map = old_of_new so that searches report the original ids.  All
 * buffers are host memory, the outputs disjoint from the inputs.
 * ANN_EINVAL on bad sizes or ids.
 */
int ann_reorder_graph(const void* base, int32_t dtype, int64_t n, int32_t d, int32_t R,
                      const int32_t* adj, int32_t entry, const uint8_t* codes, int32_t M,
                      void* base_out, int32_t* adj_out, uint8_t* codes_out,
                      int32_t* old_of_new, int32_t* entry_out);

/* Storage orders of ann_reorder_graph_ex. */
typedef enum {
  ANN_ORDER_BFS = 0,     /* breadth-first from the entry node (ann_reorder_graph) */
  ANN_ORDER_SPATIAL = 1  /* leaves of a 2-means bisection tree of the vectors, 128 nodes each */
} ann_order;

/*
 * ann_reorder_graph with a choice of order.  ANN_ORDER_SPATIAL splits the
 * vectors recursively in two by 2-means (two seed points from a hash of the
 * range, three rounds of Lloyd's step, the larger margins first, ties by id)
 * into parts whose sizes are multiples of 128, down to leaves of at most 128
 * nodes: 128 node blocks of 512 bytes fill one 64 KB translation granule, and
 * a query's successive expansions, which stay near the query in space, fall
 * into few of them.  Deterministic; *entry_out is wherever the entry lands.
 * Same outputs and errors as ann_reorder_graph otherwise.
 */
int ann_reorder_graph_ex(const void* base, int32_t dtype, int64_t n, int32_t d, int32_t R,
                         const int32_t* adj, int32_t entry, const uint8_t* codes, int32_t M,
                         int32_t order, void* base_out, int32_t* adj_out, uint8_t* codes_out,
                         int32_t* old_of_new, int32_t* entry_out);

/*
 * Build a Vamana graph (index-construction tooling; host threads).  Random
 * out-neighbours to start, then two passes (alpha 1, then `alpha`) of
 * GreedySearch(entry, x_p, L_build) + RobustPrune + back edges over a random
 * order of the nodes, in deterministic batches (the result does not depend
 * on the thread count).  alpha is compared with squared distances.
 * adj_out: host, n*R ids, -1 padded.  entry_out: the medoid used as entry.
 */
int ann_build_graph(const void* base, int32_t dtype, int64_t n, int32_t d, int32_t R,
                    float alpha, int32_t L_build, uint64_t seed, int32_t nthreads,
                    int32_t* adj_out, int32_t* entry_out);

/*
 * Computation / I/O balanced degree selector (Section "Sampling-Based Graph
 * Degree Selector": the workflow and its Eq. d = argmin_d |T_c(d) - T_f(d)|).
 * For each candidate degree a sample index of n_sample random uint8 vectors
 * with random links, random PQ codes (M subspaces) and an integer codebook is
 * built and a batch of nq random queries is searched at list size L (depth
 * 0), once with the node blocks in HBM and once in host pinned memory.
 * t_compute_us is the mean search time per step with the blocks in HBM (a
 * step is then its computation plus a short HBM fetch); t_fetch_us is the
 * extra time per step with the blocks in host memory.  *best_degree is the
 * degree with the smallest |t_compute - t_fetch|; at that degree the pipeline
 * depth 0..4 with the highest measured queries/s is *best_depth, and the
 * five measured rates go to depth_qps (may be NULL); at that degree and
 * depth the warps per query (1, 2 or 4, see ann_set_warps_per_query) with
 * the highest measured queries/s is *best_warps, the three rates in
 * warps_qps (may be NULL).  Uses the current device; takes seconds.
 */
typedef struct {
  int32_t n_sample;        /* sample size (the paper suggests ~100k) */
  int32_t d;               /* dimension of the workload (multiple of 16) */
  int32_t M;               /* PQ subspaces of the workload (multiple of 16) */
  const int32_t* degrees;  /* candidate degrees, each 1..128 */
  int32_t n_degrees;
  int32_t L;               /* list size used for the measurement */
  int32_t nq;              /* sample queries per measurement (>= 32) */
  uint64_t seed;
} ann_autotune_cfg;

typedef struct {
  int32_t degree;
  float t_compute_us;  /* per-step time, node blocks in HBM */
  float t_fetch_us;    /* extra per-step time, node blocks in host memory */
  float step_us_sync;  /* per-step time, node blocks in host memory, depth 0 */
  float qps_sync;      /* queries per second of that run */
} ann_autotune_point;

int ann_autotune_degree(const ann_autotune_cfg* cfg, ann_autotune_point* points,
                        int32_t* best_degree, int32_t* best_depth, float* depth_qps,
                        int32_t* best_warps, float* warps_qps);

/*
 * The same Vamana construction on the GPU (index-build tooling): the batch
 * searches run on the library's search kernel (exact navigation on the
 * vectors in HBM), and back edges are grouped by a device sort.
 * RobustPrune (Section "Background", Vamana) takes the distances between a
 * node's candidates from the tensor cores for uint8 rows with d <= 128
 * (BF16 MMAs with FP32 accumulation, exact for 8-bit integers), and from
 * one warp of CUDA cores per node otherwise; both make the same decisions.
 * The candidate pool of a node is the L_build expanded nodes nearest to it.
 * Deterministic.  Needs d % 16 == 0, 1 <= R <= 128, R <= L_build <= 256 - R.
 * Uses the current device; host buffers in and out, as ann_build_graph.
 */
int ann_build_graph_gpu(const void* base, int32_t dtype, int64_t n, int32_t d, int32_t R,
                        float alpha, int32_t L_build, uint64_t seed, int32_t* adj_out,
                        int32_t* entry_out);

/* Engines of ann_build_graph_gpu_ex (where RobustPrune's distances run). */
typedef enum {
  ANN_BUILD_AUTO = 0,         /* tensor cores where the data allow, else CUDA cores */
  ANN_BUILD_TENSOR_CORES = 1, /* uint8 data with d <= 128 only (ANN_EINVAL otherwise) */
  ANN_BUILD_CUDA_CORES = 2    /* one warp per node on the CUDA cores */
} ann_build_engine;

/* ann_build_graph_gpu with an engine choice; the graph does not depend on it. */
int ann_build_graph_gpu_ex(const void* base, int32_t dtype, int64_t n, int32_t d, int32_t R,
                           float alpha, int32_t L_build, uint64_t seed, int32_t engine,
                           int32_t* adj_out, int32_t* entry_out);

/*
 * Compressed navigation vectors (host-side encoders).  The precision
 * workload compares navigation on BF16 and FP8-E4M3 copies of float32
 * vectors with float32 navigation.
 *  ann_encode_bf16: the upper 16 bits of each float32, rounded to nearest,
 *    ties to even.
 *  ann_encode_fp8e4m3: x*scale in FP8-E4M3 (OCP 8-bit float, E4M3: bias 7,
 *    largest finite 448, no infinities, S.1111.111 = NaN), rounded to
 *    nearest, ties to even, finite values beyond 448 saturated to +-448.
 */
int ann_encode_bf16(const float* x, int64_t n, uint16_t* out);
int ann_encode_fp8e4m3(const float* x, int64_t n, float scale, uint8_t* out);

/*
 * Exact k nearest neighbours by brute force on the GPU (ground truth for
 * recall@k, Section "Evaluation Metrics").
 * base, queries: host; ids, dists: host, nq*k, ascending by (distance, id).
 * 1 <= k <= 128, n < 2^31.  ANN_U8 distances are exact integers; ANN_F32
 * uses FP32.  uint8 data with d <= 128 runs on the tensor cores: the dot
 * products of query and base tiles are BF16 x BF16 -> FP32 MMAs (tcgen05),
 * exact for 8-bit integers, with the top-k selected from the accumulator in
 * the same kernel; other data run on the CUDA cores.
 */
int ann_knn_exact(const void* base, int32_t dtype, int64_t n, int32_t d, const void* queries,
                  int64_t nq, int32_t k, int32_t* ids, float* dists);

/* Engines of ann_knn_exact_ex. */
typedef enum {
  ANN_KNN_AUTO = 0,         /* tensor cores where the data allow, else CUDA cores */
  ANN_KNN_TENSOR_CORES = 1, /* uint8 data with d <= 128 only (ANN_EINVAL otherwise) */
  ANN_KNN_CUDA_CORES = 2    /* the CUDA-core kernels (__dp4a for uint8, FP32 for float) */
} ann_knn_engine;

/* ann_knn_exact with an engine choice; *kernel_ms (may be NULL) receives
 * the device time of the search itself (after the upload, before the
 * download).  ANN_ETIMEOUT if a bounded wait of the tensor-core kernel ran
 * out (results are then not valid). */
int ann_knn_exact_ex(const void* base, int32_t dtype, int64_t n, int32_t d, const void* queries,
                     int64_t nq, int32_t k, int32_t engine, int32_t* ids, float* dists,
                     float* kernel_ms);

/*
 * Storage-tier read probe: `iters` passes in which every warp of a persistent
 * grid reads `block_bytes`-sized blocks at random block offsets of a
 * `bytes`-long region in `tier` (host pinned or HBM), the way the search
 * fetches node blocks.  Writes the achieved GB/s (10^9 bytes per second).
 */
int ann_probe_read_bandwidth(int64_t bytes, int32_t block_bytes, int32_t tier, int32_t iters,
                             double* gbps_out);

#ifdef __cplusplus
}
#endif

#endif /* ANN_H_ */
