/*
 * jag.h -- C ABI of the GB300 filtered nearest-neighbour search library.
 *
 * The library implements the query path of JAG (Joint Attribute Graphs,
 * arXiv 2602.10258): a greedy beam search over a proximity graph in which
 * candidates are ranked lexicographically by the filter distance dist_F and
 * then by the squared L2 distance (Sec. 3.2, "Unified comparison rule";
 * Algorithm 1 "GreedySearch" called with comparator D_F by Algorithm 2
 * "Query"), for label, range, subset and boolean filters (Sec. 2 "Filter
 * Constraints", Sec. 3.1 "Examples"); an exact pre-filter scan for the most
 * selective queries (the Pre-Filtering baseline of the experiments); and the
 * index build of Algorithms 3 ("Insert") and 4 ("JointRobustPrune") run on
 * the GPU.
 *
 * Conventions shared by every entry point:
 *   - Plain pointers and sizes only.  "device" pointers are CUDA device
 *     memory of the index's device; "host" pointers are CPU memory.
 *   - The caller owns every buffer it passes.  The index owns its own copies
 *     of vectors, attributes and graph until jag_free().
 *   - Every call returns a jag_status; JAG_OK is 0.  On failure a message
 *     for the calling thread is available from jag_last_error().  No call
 *     aborts, exits or throws across the ABI.
 *   - Device work is stream-ordered on the stream the caller passes
 *     (cudaStream_t given as void*, NULL = the legacy default stream).
 *     Outputs are valid once that stream has reached the call.
 *   - An index is read-only after jag_build(): concurrent searches on
 *     different streams are safe.
 */
#ifndef JAG_H
#define JAG_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define JAG_API __attribute__((visibility("default")))
#else
#define JAG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  JAG_OK = 0,
  JAG_EINVAL = 1,       /* bad argument (NULL pointer, size out of range, ...) */
  JAG_ENOMEM = 2,       /* device memory or scratch budget exhausted           */
  JAG_ECUDA = 3,        /* a CUDA runtime call failed                           */
  JAG_ETIMEOUT = 4,     /* a bounded device-side wait gave up                   */
  JAG_EUNSUPPORTED = 5  /* valid request this build does not handle            */
} jag_status;

/* Filter kinds (Sec. 2, "Filter Constraints"). */
typedef enum {
  JAG_F_NONE = 0,       /* no filter: dist_F = 0 for every point               */
  JAG_F_LABEL = 1,      /* equality on the int32 attribute                     */
  JAG_F_RANGE_I32 = 2,  /* lo <= a <= hi on the int32 attribute (inclusive)    */
  JAG_F_RANGE_F32 = 3,  /* lo <= a <= hi on the float32 attribute (inclusive)  */
  JAG_F_SUBSET = 4,     /* (f & a) == f on the 64-bit mask attribute           */
  JAG_F_BOOL = 5        /* f(a) == 1, f a predicate over <= 16 mask bits       */
} jag_filter_kind;

/* One query filter, 16 bytes.  payload by kind:
 *   LABEL      low 32 bits: the label (int32)
 *   RANGE_I32  low 32 bits: lo, high 32 bits: hi (int32, inclusive)
 *   RANGE_F32  low 32 bits: lo, high 32 bits: hi (float32 bit patterns)
 *   SUBSET     the required bits
 *   BOOL       the mask of the involved attribute bits (at most 16 set);
 *              aux_off is the byte offset in filter_aux of the truth table:
 *              bit s (little-endian within bytes) is f for the assignment
 *              whose bit j is the value of the j-th lowest involved bit.
 * dist_F (Sec. 3.1): label 1[a != f]; range f_min - a below, a - f_max above,
 * 0 inside; subset popcount(f & ~a); boolean the least number of bit flips
 * of a that satisfies f (computed exactly from the truth table).  An
 * unsatisfiable boolean filter matches nothing. */
typedef struct jag_filter {
  int32_t kind;
  int32_t aux_off;
  uint64_t payload;
} jag_filter;

/* Element format of the stored base vectors. */
typedef enum { JAG_VEC_F32 = 0, JAG_VEC_BF16 = 1, JAG_VEC_FP8 = 2 } jag_vec_format;

typedef struct jag_build_params {
  int64_t n;                    /* number of points, >= 1                      */
  int64_t d;                    /* dimension, 1..1024                          */
  const float *x;               /* host [n][d] fp32 base vectors               */
  const int32_t *attr_i32;      /* host [n] label / integer attribute, or NULL */
  const float *attr_f32;        /* host [n] float attribute (finite), or NULL  */
  const uint64_t *attr_mask;    /* host [n] bit-set attribute, or NULL         */
  int32_t dist_a;               /* attribute the build's dist_A compares:
                                   JAG_F_LABEL (1[a1 != a2]), JAG_F_RANGE_I32 or
                                   JAG_F_RANGE_F32 (|a1 - a2|), JAG_F_SUBSET
                                   (popcount(a1 ^ a2)); Sec. 3.1            */
  int32_t R;                    /* out-degree bound, 1..64                     */
  int32_t l_b;                  /* build beam (Algorithm 3), 1..256            */
  float alpha;                  /* pruning parameter (Algorithm 4), >= 1       */
  int32_t n_thresholds;         /* |T|, 1..4                                   */
  int32_t threshold_pct[4];     /* per-point quantiles of dist_A, in percent   */
  int32_t sample_size;          /* points sampled per threshold estimate (500) */
  uint64_t seed;                /* seed of the threshold sampling              */
  int32_t storage;              /* jag_vec_format of the searched vectors      */
  int32_t device;               /* CUDA device ordinal                         */
  const int32_t *graph;         /* optional host [n][R] out-lists (-1 padded):
                                   when given, the build is skipped            */
  int64_t entry;                /* entry vertex when graph is given            */
  int32_t n_weights;            /* Weight-JAG (the weighted variant of Sec. 3):
                                   0 = Threshold-JAG; 1..8 = build with the
                                   comparators D_A^w = w dist_A + dist, one per
                                   weight w = weight_mult[i] * h_p, with
                                   h_p = sigma / sigma_A of point p over the
                                   threshold sample (implementation-details
                                   appendix); the thresholds are then unused  */
  int32_t reserved;             /* 0                                           */
  double weight_mult[8];        /* multipliers c_i >= 0 of h (e.g. 0, 1, 10)   */
} jag_build_params;

typedef struct jag_index jag_index;   /* opaque */

/* Flags of jag_search_args.flags. */
#define JAG_SEARCH_SCAN_ALL 0x1  /* answer every query by the exact scan      */

/* Learned beam width and stop hop (an extension; the paper's search uses
 * one fixed beam l_s).  A graph-routed query runs h0 hops of Algorithm 1 at
 * the call's beam; then 12 features of its state go through a small network
 * (12 -> 64 ReLU -> 64 ReLU -> n_ladder + 1): the largest of the first
 * n_ladder outputs picks a beam from the ladder, the last output times
 * stop_scale (rounded to an integer, at least h0) is a hop count after which
 * the search stops.  If the two largest beam outputs differ by less than tau
 * the call's beam is kept and there is no stop hop.  The new beam is at most
 * the call's beam (a larger choice is taken as the call's beam) and L is cut
 * to it: the search only ever shrinks L, so a point it has set aside can
 * never qualify again and the visited set may still forget.  Features (exact integer / fp32 arithmetic): bucket
 * 0.05 * bit-length(est + 1) of the estimated passing count; filter kind one
 * hot (label, int range, float range, subset, boolean); passing fraction of
 * L; 0.125 * lg(d) of the best, k-th passing (or last) and last distances,
 * lg(x) = (bits(x) >> 16) / 128 - 127; answers found / k; expanded prefix
 * of L / |L|.  Inference: BF16 weights, fp32 fma accumulation over the
 * inputs in order from the bias. */
#define JAG_POLICY_PLAIN 0
#define JAG_POLICY_LEARNED 1
#define JAG_POLICY_FORCED 2      /* beam / stop per query from `forced`        */
#define JAG_MLP_FEATURES 12
#define JAG_MLP_HIDDEN 64

typedef struct jag_policy {
  int32_t mode;                /* JAG_POLICY_*                                  */
  int32_t h0;                  /* hops before the decision, >= 1                */
  const uint16_t *w_bf16;      /* device: W1 [64][12], W2 [64][64],
                                  W3 [n_ladder+1][64], BF16 codes, row-major    */
  const float *b_f32;          /* device: b1 [64], b2 [64], b3 [n_ladder+1]     */
  float tau;                   /* least margin of the winning beam output       */
  float stop_scale;            /* stop hop = rint(output * stop_scale); <= 0:
                                  no stop hop                                   */
  int32_t n_ladder;            /* beam classes, 1..16                           */
  int32_t ladder[16];          /* beam of each class, each in [k, 256]; a beam
                                  above the call's beam acts as the call's beam */
  const int32_t *forced;       /* device [nq][2] (beam, stop; <= 0: none), FORCED;
                                  a beam is taken into [k, call's beam]         */
  float *features;             /* device [nq][12] out, or NULL                  */
  int32_t *decisions;          /* device [nq][4] out, or NULL: final beam, stop
                                  hop (0 none), last hop that changed the first
                                  k entries of L, 1 if the network decided     */
} jag_policy;

typedef struct jag_search_args {
  const float *queries;        /* [nq][d] fp32, row-major, unpadded            */
  const jag_filter *filters;   /* [nq]                                         */
  const uint8_t *filter_aux;   /* truth tables of boolean filters, or NULL     */
  int64_t aux_bytes;           /* bytes in filter_aux                          */
  int64_t nq;                  /* number of queries, >= 0                      */
  int32_t k;                   /* answers per query, 1..min(beam, 256)         */
  int32_t beam;                /* l_s of Algorithm 1, k..512 (at most 256 with
                                  a policy, and 512 only for rows of at most
                                  512 bytes in their stored format)            */
  int32_t *out_ids;            /* [nq][k] point ids, -1 padded                 */
  float *out_dist;             /* [nq][k] squared L2 distances, +inf padded    */
  void *stream;                /* cudaStream_t, NULL = legacy default stream   */
  int64_t s0;                  /* route to the exact scan when the estimated
                                  number of passing points is below s0;
                                  0 = never, < 0 = default (2048)              */
  int64_t scan_cap;            /* largest passing set a routed query may have
                                  (larger ones go back to the graph); <= 0 =
                                  default (8192)                               */
  int32_t *counters;           /* optional [nq][4] int32: hops, first-seen
                                  neighbours, distance computations, routed    */
  int32_t flags;               /* JAG_SEARCH_* bits                            */
  int32_t hash_bits;           /* log2 slots of the visited set, in [5, 16];
                                  0 = default: 10, or 9 where that lets the
                                  graph kernel reach its blocks per SM.  The
                                  set only saves recomputed distances: answers
                                  do not depend on its size                    */
  void *ev_graph_begin;        /* optional cudaEvent_t recorded just before
                                  the graph-search kernel                      */
  void *ev_graph_end;          /* ... and just after it                        */
  const jag_policy *policy;    /* host struct, or NULL for the plain search    */
} jag_search_args;

/* Build an index on a device (Algorithms 3-4 run on the GPU; Sec. 3.3 and the
 * implementation-details appendix), or upload a given graph.  Host inputs
 * are copied; the call returns when the index is ready.  Errors: JAG_EINVAL
 * for bad sizes, NULL vectors, a missing attribute column for dist_a,
 * non-finite vectors or float attributes; JAG_ENOMEM; JAG_ECUDA. */
JAG_API jag_status jag_build(const jag_build_params *params, jag_index **out);

/* Query (Algorithm 2) for nq queries: device pointers, asynchronous on
 * args->stream.  Queries whose estimated passing count is below s0 are
 * answered by the exact scan, the others by GreedySearch with D_F.  Each
 * answer list holds the best k points with dist_F = 0 among the final
 * candidate list, sorted by (distance, id), padded with -1 / +inf.  Uses a
 * library-owned scratch buffer per stream (allocated on first use).
 * Errors: JAG_EINVAL (NULL pointers, k/beam out of range, d mismatch),
 * JAG_ENOMEM, JAG_ECUDA. */
JAG_API jag_status jag_search(jag_index *idx, const jag_search_args *args);

/* Query(G, q, l_s, k) of Algorithm 2 as one flat call: the same search as
 * jag_search with its defaults (s0 = 2048, scan_cap = 8192, default visited
 * set, no counters, no policy), device pointers queries [nq][d] fp32,
 * filters [nq], filter_aux (aux_bytes bytes of boolean truth tables, or
 * NULL), outputs out_ids / out_dist [nq][k]; asynchronous on stream
 * (cudaStream_t, NULL = legacy default stream).  Errors as jag_search. */
JAG_API jag_status jag_query(jag_index *idx, const float *queries, const jag_filter *filters,
                             const uint8_t *filter_aux, int64_t aux_bytes, int64_t nq, int32_t k, int32_t beam,
                             int32_t *out_ids, float *out_dist, void *stream);

/* Same as jag_search with HOST buffers for queries, filters, aux and
 * outputs: copies them to and from the device inside the call and returns
 * when the answers are in host memory.  args->stream may be NULL. */
JAG_API jag_status jag_search_host(jag_index *idx, const jag_search_args *args);

/* Search that allocates no device memory.  It does the same work, with the
 * same arguments and answers, as jag_search, but keeps its scratch in a
 * fixed 16 MiB area that the library reserves on each device where it builds
 * an index (held until the process exits), so it never calls cudaMalloc or
 * any other allocating routine.  It serves callers that cannot allocate while
 * they search: a latency-bound serving thread must not wait for the device
 * to drain, as cudaMalloc may; a process may have handed all device memory
 * to its own allocator up front; some deployments forbid allocation after
 * start-up.  The paper has no counterpart; it is a deployment option of this
 * library.
 *   - Set-up: jag_build puts the area in place on the index's device and
 *     looks up its device address; if that failed there, the first call on
 *     the device does it (then make that first call before any stream
 *     capture).  With CUDA's lazy module loading the first launch of each of
 *     the library's kernels in the process loads its code, which the CUDA
 *     runtime itself may place in device memory: a caller that must not see
 *     any allocation makes one warm-up call of each kind it will use first.
 *   - Every call, on any stream, uses the same area, which keeps the
 *     previous call's contents; calls whose device work overlaps race, so
 *     issue them on one stream or wait for one before starting the next.
 *   - Scratch a call needs (each region rounded up to 256 bytes): 32 bytes
 *     per query (plans) + 4 per query (counts) + 8 per filter_aux byte
 *     (boolean tables) + 512; when s0 > 0: nq * T * (12 * k + 8) bytes
 *     (partial lists and scan work items, T = ceil(max(s0, scan_cap) / 1024))
 *     and, on an index with a mask column, nq * scan_cap * 4 (gathered passing
 *     sets) + 12 * H + 8 * nq (grouping of identical filters, H the least
 *     power of two >= max(64, 2 nq)); with JAG_SEARCH_SCAN_ALL: nq * ceil(n / 65536) * 12 * k; on a
 *     BF16 / FP8 index: nq * min(4k, beam) * 4 (re-ranked ids).  A call that
 *     would need more than 16 MiB returns JAG_EINVAL with the size it needed
 *     in jag_last_error(); split the batch, lower scan_cap, or set s0 = 0.
 * Other errors as jag_search. */
JAG_API jag_status jag_search_noalloc(jag_index *idx, const jag_search_args *args);

/* Training of the policy network on the GPU (an extension, like the policy
 * itself).  params: device fp32 [P] with P = 64*12 + 64 + 64*64 + 64 +
 * (nl+1)*64 + (nl+1), laid out W1 [64][12], b1, W2 [64][64], b2,
 * W3 [nl+1][64], b3 (row-major, output by input).  X: device [m][12]
 * features, y: device [m] beam classes in [0, nl), t: device [m] stop
 * targets (hop / stop_scale).  Loss of a batch: mean cross-entropy of the
 * first nl outputs against y plus lam * mean squared error of the last
 * output against t.  Every sum is taken in a fixed order, so results repeat
 * bit for bit.  A y outside [0, nl) makes the loss NaN.  Both calls allocate
 * temporary device memory (stream-ordered) and return JAG_EINVAL for bad
 * sizes or NULL pointers, JAG_ENOMEM, JAG_ECUDA. */

/* Loss and gradient d loss / d params of one batch of all m rows (device
 * outputs grad [P] and loss [1]); asynchronous on stream. */
JAG_API jag_status jag_mlp_loss_grad(int32_t n_ladder, const float *params, const float *X, const int32_t *y,
                                     const float *t, int64_t m, float lam, float *grad, float *loss, void *stream);

/* Adam (beta 0.9 / 0.999, eps 1e-8, learning rate lr) over `epochs` passes
 * of the rows in order, in mini-batches of `batch` rows (the last one may be
 * shorter).  adam_m / adam_v: device [P] moments, zero before the first
 * step; adam_step: host in/out count of steps taken (bias correction).
 * loss_trace: host [epochs] mean batch loss of each pass, or NULL.
 * Synchronous: returns when params are updated. */
JAG_API jag_status jag_mlp_train(int32_t n_ladder, float *params, float *adam_m, float *adam_v, int64_t *adam_step,
                                 const float *X, const int32_t *y, const float *t, int64_t m, int32_t epochs,
                                 int32_t batch, float lr, float lam, float *loss_trace, void *stream);

/* Inference blobs of the policy from params: BF16 weights (round to nearest
 * even) and fp32 biases, device outputs. */
JAG_API jag_status jag_mlp_export(int32_t n_ladder, const float *params, uint16_t *w_bf16, float *b_f32,
                                  void *stream);

/* ------------------------------------------------------------------------
 * Serving: a device-resident request loop with continuous batching (an
 * extension of this library; the paper evaluates batches of queries only).
 *
 * A persistent kernel keeps one warp per query in flight, like jag_search,
 * but takes its queries from a ring of requests in mapped host memory as
 * they arrive: a warp that finishes a query claims the next published one,
 * whatever request it belongs to, so requests that arrive while others are
 * running are admitted as soon as warps free up and their work overlaps on
 * the device.  Each query is answered exactly as jag_search answers it with
 * the same k, beam, s0, scan_cap, hash_bits and policy (the same routing,
 * scan and graph search), so a result does not depend on what else is in
 * flight.  Inputs and outputs stay in pinned host memory that the kernel
 * reads and writes directly; there is no copy call per request.
 *
 * Admission: a request is admitted when a ring slot, room for its inputs and
 * outputs in the host arena, and room for its boolean filter tables in the
 * device scratch budget (lut_bytes) are all free; space is returned when its
 * results are collected by jag_serve_wait.  Every wait of the device loop is
 * bounded: it exits after idle_exit_s without work (the library starts it
 * again when work arrives) and on jag_serve_stop.
 *
 * One thread may submit while another waits; calls on one server are
 * serialised internally.
 * ------------------------------------------------------------------------ */
typedef struct jag_server jag_server;   /* opaque */

typedef struct jag_serve_params {
  int32_t k;                   /* answers per query, 1..beam                   */
  int32_t beam;                /* l_s, k..256                                  */
  int64_t s0;                  /* as jag_search_args.s0                        */
  int64_t scan_cap;            /* as jag_search_args.scan_cap                  */
  int32_t hash_bits;           /* as jag_search_args.hash_bits                 */
  int32_t max_requests;        /* ring slots (admitted, not yet collected);
                                  0 = 1024, at most 65536                      */
  int64_t max_queries;         /* queries admitted at once, counted from the
                                  first query of the oldest uncollected
                                  request to the last published; 0 = 65536   */
  int64_t arena_bytes;         /* host arena for inputs / outputs; 0 = enough
                                  for max_queries queries with 64 bytes of
                                  truth tables each                            */
  int64_t lut_bytes;           /* device budget for boolean filter tables
                                  (8 bytes per truth-table byte); 0 = 16 MiB   */
  int32_t ctas;                /* persistent CTAs; 0 = as many as are resident */
  int32_t reserved;            /* 0                                            */
  double idle_exit_s;          /* device loop exits after this long with no
                                  work; 0 = 1.0                                */
  const jag_policy *policy;    /* LEARNED or PLAIN policy, or NULL; its
                                  forced / features / decisions must be NULL;
                                  copied at start                              */
} jag_serve_params;

typedef struct jag_serve_timing {
  double submit_s;             /* host steady clock at submission (seconds)    */
  double done_s;               /* host steady clock when completion was seen   */
  double device_s;             /* device time from the claim of the request's
                                  first query to the end of its last one       */
  uint32_t status;             /* bit 2: a query had an invalid filter (its
                                  answers are padded)                          */
  uint32_t reserved;
} jag_serve_timing;

/* Start a server on idx (which must outlive it).  Allocates the ring, the
 * arena (pinned, mapped) and the device scratch, and launches the loop.
 * Errors: JAG_EINVAL (bad parameters), JAG_ENOMEM, JAG_ECUDA. */
JAG_API jag_status jag_serve_start(jag_index *idx, const jag_serve_params *params, jag_server **out);

/* Submit one request of nq >= 1 queries from HOST buffers: queries [nq][d]
 * fp32, filters [nq], aux: the truth tables the boolean filters point into
 * (aux_bytes bytes; may be NULL if no filter is boolean).  The inputs are
 * copied (boolean tables are repacked; aux_off is rewritten in the copy), so
 * the caller may reuse its buffers on return.  Waits up to timeout_s for
 * admission: JAG_ETIMEOUT if there was no room in time (nothing is
 * submitted), JAG_EINVAL if the request could never fit.  *ticket
 * identifies the request. */
JAG_API jag_status jag_serve_submit(jag_server *srv, const float *queries, const jag_filter *filters,
                                    const uint8_t *aux, int64_t aux_bytes, int32_t nq, double timeout_s,
                                    uint64_t *ticket);

/* Wait up to timeout_s (0: just test) for a request, then copy its answers
 * to HOST buffers ids [nq][k], dist [nq][k] (either may be NULL) and its
 * timing to *timing (may be NULL), and release its space.  JAG_ETIMEOUT if
 * it is not complete in time (the ticket stays valid); JAG_EINVAL for an
 * unknown ticket. */
JAG_API jag_status jag_serve_wait(jag_server *srv, uint64_t ticket, int32_t *ids, float *dist,
                                  jag_serve_timing *timing, double timeout_s);

/* Open-loop driver for measurements: request r, of sizes[r] queries taken
 * from rows first[r].. of the HOST pools (queries [*][d], filters [*], aux),
 * is submitted arrival_s[r] seconds after the call starts (arrival_s
 * non-decreasing), or later when there is no room; completions are
 * collected as they happen.  Outputs (HOST, each may be NULL): ids / dist
 * [*][k] at the requests' rows; latency_s[r] = completion seen - scheduled
 * arrival; device_s[r] as in jag_serve_timing.  Returns when every request
 * is complete, or JAG_ETIMEOUT after timeout_s in total. */
JAG_API jag_status jag_serve_replay(jag_server *srv, int64_t n_req, const double *arrival_s, const int32_t *sizes,
                                    const int64_t *first, const float *queries, const jag_filter *filters,
                                    const uint8_t *aux, int64_t aux_bytes, int32_t *ids, float *dist,
                                    double *latency_s, double *device_s, double timeout_s);

/* Counters of a server: launches of the device loop so far, and queries
 * completed. */
JAG_API jag_status jag_serve_info(const jag_server *srv, int64_t *launches, int64_t *queries_done);

/* Drain: wait for every admitted request to finish on the device (the loop
 * then exits), release everything (uncollected results are dropped).  NULL
 * is allowed.  JAG_ETIMEOUT if the device did not finish within 60 s (the
 * server is then leaked rather than freed under running work). */
JAG_API jag_status jag_serve_stop(jag_server *srv);

/* Index facts. */
typedef struct jag_info {
  int64_t n, d;
  int32_t R, storage;
  int64_t entry;
  int64_t device_bytes;         /* bytes the index holds on the device         */
  double build_seconds;         /* wall time of the GPU build, 0 if uploaded   */
  int32_t n_thresholds, dist_a;  /* n_thresholds: |T|, or |W| of a Weight-JAG build */
  int32_t weighted, reserved;      /* 1 for a Weight-JAG build                   */
} jag_info;
JAG_API jag_status jag_get_info(const jag_index *idx, jag_info *out);

/* Copy the out-lists [n][R] (-1 padded) to host memory. */
JAG_API jag_status jag_get_graph(const jag_index *idx, int32_t *host_out);

/* Copy the per-point thresholds [n][n_thresholds] (dist_A in the ordered
 * 32-bit form: integer value, or float bit pattern) to host memory -- for a
 * Weight-JAG build, the per-point weights [n][n_weights] as fp32 bit
 * patterns; JAG_EINVAL if the graph was uploaded rather than built. */
JAG_API jag_status jag_get_thresholds(const jag_index *idx, uint32_t *host_out);

/* Copy the stored BF16 / FP8 rows [n][row_bytes] (row_bytes = d * element
 * bytes rounded up to 16; zero padded) and the per-row scales [n] to host
 * memory (the paper stores fp32 vectors; this is the low-precision storage option).
 * row_bytes_out receives row_bytes.  JAG_EINVAL for an fp32 index. */
JAG_API jag_status jag_get_stored_rows(const jag_index *idx, uint8_t *rows_out, float *scales_out,
                                       int32_t *row_bytes_out);

/* Release the index and its device memory.  NULL is allowed. */
JAG_API void jag_free(jag_index *idx);

/* Message of the calling thread's last failed call ("" if none). */
JAG_API const char *jag_last_error(void);

/* Library version string. */
JAG_API const char *jag_version(void);

#ifdef __cplusplus
}
#endif

#endif /* JAG_H */
