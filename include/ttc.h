/*
 * ttc.h -- exact (d13, d12, d23)-temporal triangle counting on one GB300 GPU.
 *
 * Method: Pashanasangi & Seshadhri, "Faster and Generalized Temporal Triangle
 * Counting, via Degeneracy Ordering", KDD'21 (DOTTT).
 *
 * Input (Sec. 3): a directed temporal multigraph given as m edges
 * (src[i], dst[i], t[i]).  The edge index i breaks timestamp ties: edges are
 * totally ordered by the key (t, i).
 *
 * Output (Def. 1, Fig. 2): for a delta-triple (d13, d12, d23), the number of
 * edge triples e1 < e2 < e3 (key order) on the three vertex pairs of a static
 * triangle with t2 - t1 <= d12, t3 - t2 <= d23 and t3 - t1 <= d13, split by
 * triangle type: out[k-1] is the count of type T_k of Fig. 2 (k = 1..8).
 * Counts are exact unsigned 64-bit integers.
 *
 * Conventions shared by every entry point:
 *   - Inputs are owned by the caller and only read during the call.  Unless a
 *     flag says otherwise, pointers are host pointers; they are copied to the
 *     device before the call returns.  A load's edge arrays that are
 *     page-locked (cudaMallocHost, cudaHostAlloc or cudaHostRegister under
 *     the current device) are read by the load's first kernel directly, over
 *     the host link, which also writes the device copies.
 *   - Outputs are caller-allocated and written only when the call returns
 *     TTC_OK.
 *   - A ttc_graph owns all of its device memory until ttc_free().  It is
 *     immutable after loading; concurrent count calls on one graph are
 *     allowed.  All work runs on the graph's CUDA stream (one per graph).
 *   - On failure a call returns a negative ttc_status (or NULL), and
 *     ttc_last_error() gives a message for the calling thread.
 *   - Vertex ids must be < 2^31.  Timestamps must lie in [-2^62, 2^62] and
 *     every delta component in [0, 2^62].  m = 0 is valid and counts zero.
 *   - The load packs each edge's (t - min t), a tie-break rank and its
 *     direction into one 63-bit key.  The rank is the edge's input index
 *     when that fits, else its rank among the edges with the same timestamp.
 *     A graph whose span needs s bits and whose largest group of equal
 *     timestamps needs r bits is refused with TTC_ERR_RANGE when
 *     s + r + 1 > 63: a span of 2^62 or more always, a span of 2^61 or
 *     more when some timestamp repeats.
 *   - Self-loops (src == dst) can never lie on a triangle and are dropped
 *     (and counted in the statistics).
 */
#ifndef TTC_H
#define TTC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TTC_NUM_TYPES 8

typedef struct ttc_graph ttc_graph;
typedef struct ttc_server ttc_server;

/* One query: the three windows of Def. 1.  Any non-negative triple is legal;
 * the library normalises it (d12 <- min(d12, d13), d23 <- min(d23, d13),
 * d13 <- min(d13, d12 + d23)), which leaves every count unchanged. */
typedef struct {
    int64_t d13, d12, d23;
} ttc_delta;

typedef enum {
    TTC_OK = 0,
    TTC_PENDING = 1,          /* ttc_serve_poll: result not ready yet */
    TTC_ERR_INVALID = -1,     /* NULL pointer, bad flag or handle */
    TTC_ERR_RANGE = -2,       /* id, timestamp or delta outside the documented range */
    TTC_ERR_NOMEM = -3,       /* device or host allocation failed */
    TTC_ERR_CUDA = -4,        /* a CUDA call failed */
    TTC_ERR_TIMEOUT = -5,     /* a bounded wait gave up */
    TTC_ERR_OVERFLOW = -6,    /* a count does not fit in 64 bits */
    TTC_ERR_BUSY = -7,        /* server queue full */
    TTC_ERR_INTERNAL = -8,    /* an internal consistency check failed */
    TTC_ERR_NOT_FOUND = -9    /* unknown graph id or ticket */
} ttc_status;

/* ------------------------------------------------------------------ load */

/* Load flags. */
#define TTC_LOAD_DEVICE_INPUT 1u  /* src/dst/t are device pointers (same device) */
#define TTC_LOAD_PROFILE 2u       /* time the load's phases (ttc_profile_read after
                                     the load; profiling stays on for counts) */
#define TTC_LOAD_STREAM 4u        /* keep no list of light triangles: the handle keeps
                                     the oriented graph instead (about 28 B per vertex
                                     pair) and every count enumerates the triangles
                                     again, counting light ones as they are found
                                     (Alg. 1 with enumeration and counting fused);
                                     heavy triangles are still listed.  For graphs
                                     whose triangle list (16 B per triangle) does not
                                     fit.  ttc_count and ttc_count_batch only: the
                                     many-graph, sample and no-allocation entry points
                                     refuse such a handle with TTC_ERR_INVALID.  A count
                                     collects the light triangles chunk by chunk into a
                                     buffer of TTC_STREAM_CHUNK records (environment,
                                     read at load; default 2^24 = 256 MiB) */

#define TTC_LOAD_STRICT_TIME 8u   /* read Def. 1's t1 < t2 < t3 literally: a triple
                                     counts only if its three timestamps strictly
                                     increase.  Default: edges are ordered by the key
                                     (t, input index), so equal timestamps are ordered
                                     by input position (Sec. 3 assumes distinct
                                     timestamps; both readings agree on such inputs) */

/* Vertex orderings used to orient the static graph.  Any acyclic orientation
 * gives identical counts; the degeneracy ordering (Sec. 3, Matula-Beck) bounds
 * every out-degree by the degeneracy kappa (Theorem 1). */
#define TTC_ORIENT_DEGENERACY 0u  /* k-core peel order (default) */
#define TTC_ORIENT_ID 1u          /* by vertex id */
#define TTC_ORIENT_DEGREE 2u      /* by (degree, id) */
#define TTC_ORIENT_RANDOM 3u      /* by a seeded random permutation */

/* Which vertex of a static triangle plays u (the vertex whose two pairs are
 * enumerated).  The paper uses the first vertex in the ordering (Sec. 5,
 * "source vertex"); the default instead names u the vertex opposite the pair
 * with the most edges, so that the longest list is only ever searched.  Both
 * give identical counts. */
#define TTC_LABEL_HEAVIEST_VW 0u  /* default */
#define TTC_LABEL_SOURCE 1u       /* the paper's labelling */

/* How the one-CTA class of the prefix-sum path finds the window ends of
 * Algs. 2-4 (this library's choice; both give identical counts). */
#define TTC_HEAVY_BINARY 1u  /* a binary search per bound and enumerated edge (default) */
#define TTC_HEAVY_MERGE 2u   /* the two-pointer form: along a key-sorted list every
                                bound only grows, so a thread takes a run of
                                consecutive edges, binary-searches the first and
                                steps forward from there for the rest; used for the
                                triangles whose C list is staged in shared memory and
                                holds at most sigma_A + sigma_B edges, binary
                                searches elsewhere (and in the many-graph launch) */

typedef struct {
    uint32_t flags;            /* TTC_LOAD_* */
    uint32_t orientation;      /* TTC_ORIENT_* */
    uint32_t labeling;         /* TTC_LABEL_* */
    uint32_t light_max_pairs;  /* triangles with sigma_A * sigma_B below this use the
                                  one-thread-per-triangle path, the others the
                                  prefix-sum path (1 = all prefix-sum); 0 = the
                                  tuned value for graphs of this shape
                                  (ttc_tune_light), else the default; values
                                  above 2^20 count as 2^20 */
    uint32_t heavy_warp_cap;   /* prefix-sum-path triangles whose two enumerated
                                  lists hold at most this many edges together are
                                  counted by one warp each; 0 = tuned
                                  (ttc_tune_heavy), else the kernel's capacity
                                  (128 edges, 64 when a pair holds 2^16 edges or
                                  more); larger values count as the capacity */
    uint32_t heavy_cta_cap;    /* the others up to this many edges by one CTA
                                  each, the rest by the flat path; 0 = tuned,
                                  else the capacity (2048, 1024 when a pair holds
                                  2^16 edges or more); clamped to
                                  [heavy_warp_cap, capacity] */
    uint32_t heavy_merge;      /* TTC_HEAVY_BINARY or TTC_HEAVY_MERGE; 0 = tuned
                                  (ttc_tune_heavy), else TTC_HEAVY_BINARY */
    uint64_t seed;             /* TTC_ORIENT_RANDOM permutation seed */
    void *stream;              /* cudaStream_t to adopt; NULL = create one */
} ttc_load_opts;

typedef struct {
    uint64_t n;              /* max vertex id + 1 */
    uint64_t m;              /* temporal edges kept (self-loops dropped) */
    uint64_t m_self_loops;   /* self-loops dropped */
    uint64_t m_s;            /* static edges (vertex pairs with >= 1 edge) */
    uint64_t tau;            /* static triangles */
    uint64_t kappa;          /* max out-degree of the orientation (= degeneracy for
                                TTC_ORIENT_DEGENERACY) */
    uint64_t sigma_max;      /* largest number of edges on one pair */
    uint64_t peel_rounds;    /* rounds of the k-core peel */
    uint64_t work_bytes;     /* sum over static triangles of 8 (s_uv + s_uw + s_vw) + 12 */
    uint64_t enum_elems;     /* sum over static triangles of the enumerated list lengths */
    uint64_t tau_light;      /* triangles on the one-thread-per-triangle path */
    uint64_t tau_heavy;      /* triangles on the prefix-sum (CEC) path */
    uint64_t device_bytes;   /* device memory held by the graph */
    uint64_t work_bytes_heavy; /* the part of work_bytes from prefix-sum-path triangles */
    uint64_t tau_huge;       /* prefix-sum-path triangles too large for one CTA (flat path) */
    uint64_t tau_hwarp;      /* prefix-sum-path triangles counted by one warp each */
    uint64_t tau_hcta;       /* prefix-sum-path triangles counted by one CTA each */
    uint64_t light_pairs;    /* sum over one-thread-per-triangle-path triangles of
                                sigma_A * sigma_B (the (a, b) pairs that path visits) */
    uint32_t key_bits;       /* bits of the packed per-edge key */
    uint32_t light_max_pairs; /* the light threshold the load used (given, tuned or default) */
    uint32_t heavy_warp_cap;  /* the one-warp class's cap the load used (edges of A plus B) */
    uint32_t heavy_cta_cap;   /* the one-CTA class's cap the load used */
    uint32_t heavy_merge;     /* the one-CTA class's search form (TTC_HEAVY_*) */
} ttc_graph_stats;

/* Build the device-resident graph (Alg. 1 steps up to the triangle list:
 * static graph, degeneracy ordering, orientation, per-pair key-sorted edge
 * lists, static triangles).  Uses default options.  Returns NULL on error. */
ttc_graph *ttc_load(const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m);

/* As ttc_load with options (opts may be NULL).  *out receives the handle. */
ttc_status ttc_load_ex(const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m,
                       const ttc_load_opts *opts, ttc_graph **out);

/* Tuning of the light threshold (this library's split of the static
 * triangles between the direct Lemma 1 sum over A x B and the prefix-sum
 * form of Algs. 2-4; the paper has no such split).  Loads the graph once per
 * candidate threshold (ttc_tune_candidates), times load plus one
 * ttc_count_batch of the k probe queries (host arrays) with CUDA events on
 * opts->stream (the faster of two timed runs after an untimed one), and
 * keeps the fastest: *chosen receives it, ms (may be NULL)
 * the time of each candidate.  The choice is cached for graphs of the same
 * shape (bit lengths of m, m_s, largest multiplicity and kappa) on a GPU
 * with the same number of SMs, in the JSON file $TTC_TUNE_CACHE (default
 * ~/.cache/ttc/tune.json); ttc_load_ex with light_max_pairs = 0 then uses
 * it.  opts->light_max_pairs must be 0.  Processes that must bin a graph
 * identically (ttc_count_shard) should pass one explicit threshold. */
#define TTC_TUNE_CANDIDATES 6
static const uint32_t ttc_tune_candidates[TTC_TUNE_CANDIDATES] = {17, 65, 257, 1025, 4097, 16385};
ttc_status ttc_tune_light(const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m,
                          const ttc_load_opts *opts, const ttc_delta *probe, uint32_t k, uint32_t *chosen,
                          float *ms);

/* Tuning of the prefix-sum path's split into its three classes (one warp,
 * one CTA, flat; this library's, not the paper's) and of the one-CTA class's
 * search form, at the light threshold opts->light_max_pairs (0: tuned or
 * default).  Loads the graph once per (warp cap, CTA cap, search form) of
 * ttc_tune_heavy_candidates (caps capped as in ttc_load_opts), times load
 * plus one ttc_count_batch of the k probe queries (the fastest of three
 * timed runs after an untimed one), and keeps the fastest, the first
 * candidate (the kernels' capacities, binary searches) unless another is
 * more than 1% faster: *warp_cap, *cta_cap and *merge receive what the loads
 * used, ms (may be NULL) the time of each candidate.  With no
 * prefix-sum-path triangle it stops after the first.  The choice is cached
 * like the light threshold's (per shape, SM count and light threshold);
 * ttc_load_ex with both caps 0 then uses the caps, with heavy_merge 0 the
 * search form.  opts->heavy_warp_cap, opts->heavy_cta_cap and
 * opts->heavy_merge must be 0. */
#define TTC_TUNE_HEAVY_CANDIDATES 8
static const uint32_t ttc_tune_heavy_candidates[TTC_TUNE_HEAVY_CANDIDATES][3] = {
    {128, 2048, TTC_HEAVY_BINARY}, {64, 2048, TTC_HEAVY_BINARY},  {32, 2048, TTC_HEAVY_BINARY},
    {128, 1024, TTC_HEAVY_BINARY}, {64, 1024, TTC_HEAVY_BINARY},  {128, 512, TTC_HEAVY_BINARY},
    {128, 2048, TTC_HEAVY_MERGE},  {64, 2048, TTC_HEAVY_MERGE}};
ttc_status ttc_tune_heavy(const uint32_t *src, const uint32_t *dst, const int64_t *t, uint64_t m,
                          const ttc_load_opts *opts, const ttc_delta *probe, uint32_t k, uint32_t *warp_cap,
                          uint32_t *cta_cap, uint32_t *merge, float *ms);

/* Release a graph and all of its device memory.  NULL is a no-op. */
void ttc_free(ttc_graph *g);

/* Statistics of a loaded graph (the static quantities of Sec. 3 and Table 2:
 * n, m, m_s, static triangles tau, degeneracy kappa, largest multiplicity;
 * and this library's work figures: the work bytes of the count, W = sum over
 * static triangles of 8 (s_uv + s_uw + s_vw) + 12, the enumerated list
 * lengths of Sec. 5, the bin sizes and device memory).  *s is a
 * caller-owned host struct, written on TTC_OK; TTC_ERR_INVALID for NULL. */
ttc_status ttc_graph_info(const ttc_graph *g, ttc_graph_stats *s);

/* ----------------------------------------------------------------- count */

/* One query (Alg. 1, counting step; Lemma 1 and Algs. 2-4 per static
 * triangle; Table 1 maps each (ordering, orientation) to a type).
 * out[8] is a host array. */
ttc_status ttc_count(ttc_graph *g, const ttc_delta *d, uint64_t out[TTC_NUM_TYPES]);

/* k queries in one pass over the triangles.  d[k] host array; out is a host
 * array of k * 8 counts, row q for d[q].  The flat heavy path takes the
 * queries in passes whose prefix scratch stays within 64 MB
 * ($TTC_HUGE_PASS_BYTES, environment, replaces that cap). */
ttc_status ttc_count_batch(ttc_graph *g, const ttc_delta *d, uint32_t k, uint64_t *out);

/* One shard of ttc_count_batch, for counting one graph on several GPUs (or
 * processes): every static triangle is counted on its own (Alg. 1 counts
 * each triangle of the oriented graph independently; Sec. 5, proof of
 * Theorem 1), so the triangle list can be divided.  Each of the handle's bins
 * (light, warp, CTA and flat records) is cut into nshards consecutive slices
 * of near-equal length, and this call counts slice `shard` of every bin.  The
 * shards partition the triangles: summing out over shard = 0 .. nshards - 1
 * gives ttc_count_batch's counts (the caller sums; TTC_ERR_OVERFLOW covers
 * this shard's counts only).  Every process loads the same edges, and the
 * load is deterministic, so all hold the same bins.  d[k], out[k * 8] host
 * arrays as in ttc_count_batch.  TTC_ERR_INVALID for shard >= nshards,
 * nshards = 0, or a TTC_LOAD_STREAM handle. */
ttc_status ttc_count_shard(ttc_graph *g, const ttc_delta *d, uint32_t k, uint32_t shard, uint32_t nshards,
                           uint64_t *out);

/* δ-grid analytics: the counts at every (δ1,2, δ2,3) of the grid
 * d12[0..n12) x d23[0..n23) for one δ1,3, in one batched pass (the
 * dependence of the type mix on the windows, Sec. 6 and Figs. 1 and 5).
 * out: n12 * n23 * TTC_NUM_TYPES uint64, row-major [i12][i23][type].
 * cyclic (may be NULL): n12 * n23 doubles, the share of the two cyclic types
 * (T4 + T8) in the total of that grid point (0 when the total is 0).
 * Each δ as in ttc_count; TTC_ERR_RANGE if n12 * n23 exceeds 2^20. */
ttc_status ttc_count_grid(ttc_graph *g, int64_t d13, const int64_t *d12, uint32_t n12, const int64_t *d23,
                          uint32_t n23, uint64_t *out, double *cyclic);

/* As ttc_count_batch, but asynchronous: d_dev (k deltas, each component in
 * [0, 2^62]; normalised on the device) and out_dev (k * 8 uint64) are device
 * pointers, and the work is queued on `stream` (cudaStream_t; NULL = the
 * graph's stream).  The caller synchronises.  Overflow is not detected and
 * out-of-range deltas are not reported on this path. */
ttc_status ttc_count_batch_async(ttc_graph *g, const ttc_delta *d_dev, uint32_t k,
                                 uint64_t *out_dev, void *stream);

/* Many graphs in one launch: graph q is counted under d[q]; out is a host
 * array of G * 8 counts.  All graphs must live on the current device.  The
 * launch is captured into a CUDA graph on first use for a given set of
 * handles and replayed afterwards.  Graphs loaded with TTC_LOAD_STREAM keep
 * no triangle list to share: they are counted one by one (as ttc_count)
 * after the shared launch of the others. */
ttc_status ttc_count_multi(ttc_graph *const *g, const ttc_delta *d, uint32_t G, uint64_t *out);

/* Streaming many-graph count, for collections of graphs that need not fit
 * in device memory together (the paper has no counterpart).  Graph i is the
 * host arrays (src[i], dst[i], t[i]) of m[i] edges, counted under d[i].  The
 * graphs are loaded in order (ttc_load_ex with opts, which may be NULL;
 * TTC_LOAD_DEVICE_INPUT and TTC_LOAD_STREAM are refused) and gathered into
 * batches: a graph joins the current batch while the batch's device
 * footprint (ttc_graph_stats.device_bytes) stays within budget_bytes
 * (0: half of the device memory free at the call), else the batch is counted
 * by one ttc_count_multi launch and freed first.  So device memory holds at
 * most one batch plus the graph being loaded; a graph larger than the budget
 * forms a batch of its own.  A load that fails with TTC_ERR_NOMEM while a
 * batch is resident is tried once more after that batch is counted and
 * freed.  out: G * 8 counts (host); *batches (may be NULL) receives the
 * number of batches.  On an error the graphs loaded so far are freed. */
ttc_status ttc_count_stream(const uint32_t *const *src, const uint32_t *const *dst, const int64_t *const *t,
                            const uint64_t *m, const ttc_delta *d, uint32_t G, const ttc_load_opts *opts,
                            uint64_t budget_bytes, uint64_t *out, uint32_t *batches);

/* Sampled per-triangle counts, for checking against a slow reference at full
 * size: every `stride`-th static triangle of the graph's own list, starting
 * at `first`, is counted under d by the same kernels as ttc_count.  Writes up
 * to `cap` triangles as vertex triples tri[3 * i] (host) and their counts
 * out[8 * i] (host); *written receives the number written. */
ttc_status ttc_count_sample(ttc_graph *g, const ttc_delta *d, uint64_t first, uint64_t stride,
                            uint64_t cap, uint32_t *tri, uint64_t *out, uint64_t *written);

/* Participation counts (analytics on Def. 1's counts; the paper has no
 * counterpart).  vertex[v], v < n: the number of delta-temporal triangles
 * (all eight types) that have v as a vertex.  pair[p], p < m_s: the number
 * that use an edge of static pair p, pairs numbered as ttc_graph_pairs
 * lists them.  Either output (host) may be NULL.  Each static triangle's
 * count comes from the same kernels as ttc_count_sample and is added to its
 * three vertices and its three pairs, so sum(vertex) = sum(pair) = 3 times
 * ttc_count's total.  TTC_ERR_OVERFLOW if a sum passes 2^64; refused
 * (TTC_ERR_INVALID) for a TTC_LOAD_STREAM handle. */
ttc_status ttc_count_participation(ttc_graph *g, const ttc_delta *d, uint64_t *vertex, uint64_t *pair);

/* The static pairs (vertex pairs with at least one edge) in the library's
 * pair order: lohi[2 p], lohi[2 p + 1] = the lower and the higher vertex id
 * of pair p, for p < m_s (host). */
ttc_status ttc_graph_pairs(ttc_graph *g, uint32_t *lohi);

/* No-allocation variant of ttc_count (the paper has no counterpart; this is
 * an interface convenience).  For callers that cannot allocate device memory
 * when they count: beside a framework allocator that owns the device's
 * memory, or in latency-critical loops where an allocation may stall.  It
 * runs the same kernels as ttc_count, but its device scratch (the counts, the
 * delta and the prefix-sum arrays of the heavy bin) is one static __device__
 * array of TTC_NOALLOC_SCRATCH_BYTES that every device holds from library
 * load to process exit; it calls no cudaMalloc, cudaFree or other allocator.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current.
 *   - A graph whose heavy-bin prefix arrays need more than the array holds
 *     (TTC_NOALLOC_SCRATCH_BYTES - 512 bytes) is rejected with TTC_ERR_RANGE;
 *     use ttc_count for it.
 *   - Every call shares the one array and keeps the previous call's contents;
 *     each call zeroes the counts it needs.  Calls are serialised by a lock;
 *     other work that overlapped a call on the GPU while using the same
 *     array would race.
 *   - The call is synchronous: it waits on `stream` for its kernels and
 *     copies the counts to out before it returns.  The caller's current
 *     device is current again on return.
 * d and out are host pointers; stream is a cudaStream_t (NULL = the graph's
 * stream). */
#define TTC_NOALLOC_SCRATCH_BYTES (64u << 20)
ttc_status ttc_count_noalloc(ttc_graph *g, const ttc_delta *d, uint64_t out[TTC_NUM_TYPES], void *stream);

/* ----------------------------------------------------------------- serve */

typedef struct {
    uint64_t hbm_reserve_bytes;  /* device memory kept free when admitting graphs */
    uint32_t max_batch;          /* most queries per graph per launch (0 = 256) */
    uint32_t max_queue;          /* most pending queries (0 = 65536) */
    uint32_t streams;            /* concurrent launch streams (0 = 4) */
    uint32_t wait_limit_us;      /* longest the worker sleeps between checks for finished
                                    launches and new queries, in microseconds (0 = 200):
                                    every wait of the server is bounded */
} ttc_server_opts;

/* A server keeps graphs resident and runs queries as they arrive: pending
 * queries on one graph are packed into one batched launch, launches on
 * different graphs overlap on separate streams, and new graphs are admitted
 * while free device memory (minus the reserve) allows, evicting the
 * least-recently-used idle graph otherwise. */
ttc_server *ttc_server_create(const ttc_server_opts *o);
void ttc_server_destroy(ttc_server *s);

/* Load a graph into the server (host arrays, as ttc_load).  *graph_id
 * receives its id. */
ttc_status ttc_serve_load(ttc_server *s, const uint32_t *src, const uint32_t *dst, const int64_t *t,
                          uint64_t m, uint64_t *graph_id);

/* Queue one query; *ticket identifies it.  TTC_ERR_BUSY if the queue is
 * full, TTC_ERR_NOT_FOUND for an unknown or evicted graph. */
ttc_status ttc_serve_submit(ttc_server *s, uint64_t graph_id, const ttc_delta *d, uint64_t *ticket);

/* TTC_PENDING until the query is done; then TTC_OK with out[8] and the
 * submit-to-completion latency in seconds (latency_s may be NULL).  A ticket
 * can be collected once. */
ttc_status ttc_serve_poll(ttc_server *s, uint64_t ticket, uint64_t out[TTC_NUM_TYPES], double *latency_s);

/* Hold (paused = 1) or resume (0) the launching of new batches; queries
 * submitted meanwhile wait in the queue.  Batches already on the device run
 * to completion. */
ttc_status ttc_serve_pause(ttc_server *s, int paused);

/* Change the device memory that admission keeps free (the server option
 * hbm_reserve_bytes) for later ttc_serve_load calls.  Resident graphs stay;
 * the next load evicts idle ones if it no longer fits. */
ttc_status ttc_serve_set_reserve(ttc_server *s, uint64_t hbm_reserve_bytes);

/* Block until every submitted query has completed, or timeout_s passes
 * (TTC_ERR_TIMEOUT). */
ttc_status ttc_serve_drain(ttc_server *s, double timeout_s);

typedef struct {
    uint64_t submitted, completed, launches, graphs_resident, admissions, evictions;
    uint64_t queue_depth_max;
} ttc_server_stats;

ttc_status ttc_server_info(ttc_server *s, ttc_server_stats *st);

/* ----------------------------------------------------------------- misc */

/* Message for the calling thread's last failure ("" if none). */
const char *ttc_last_error(void);

/* Library version string. */
const char *ttc_version(void);

/* Device memory.  Every device allocation of the library comes from one
 * stream-ordered pool per device that keeps freed blocks (of ttc_free and of
 * a load's temporaries) mapped for reuse, so repeated loads do not map and
 * unmap memory.  ttc_release_cached synchronises the calling thread's device
 * and returns those cached blocks to it; *released (may be NULL) receives
 * the bytes released.  Server admission counts cached bytes as free. */
ttc_status ttc_release_cached(uint64_t *released);

/* Device memory as admission sees it, for the calling thread's device:
 * *device_free = free device memory (cudaMemGetInfo), *pool_reserved and
 * *pool_used = bytes the library's pool has mapped and has handed out.
 * Admission counts device_free + (pool_reserved - pool_used) as free.  Any
 * pointer may be NULL. */
ttc_status ttc_memory_info(uint64_t *device_free, uint64_t *pool_reserved, uint64_t *pool_used);

/* Testing hook: make the n-th device allocation from now fail with
 * TTC_ERR_NOMEM (n = 0 disables).  Process-wide. */
void ttc_debug_fail_alloc_after(uint64_t n);

/* Number of kernels this library has launched in the process so far. */
uint64_t ttc_debug_launch_count(void);

/* Per-kernel timing of count calls.  While profiling is on for a graph, each
 * count call records a CUDA event pair around every kernel it launches (on
 * the graph's stream); ttc_profile_read returns the kernels of the most
 * recent count call: name and duration in milliseconds.  Returns the number
 * of kernels written (at most cap). */
typedef struct {
    char name[32];
    float ms;
} ttc_kernel_time;

ttc_status ttc_set_profiling(ttc_graph *g, int on);
uint32_t ttc_profile_read(ttc_graph *g, ttc_kernel_time *out, uint32_t cap);

#ifdef __cplusplus
}
#endif

#endif /* TTC_H */
