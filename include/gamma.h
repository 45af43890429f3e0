/*
 * gamma.h -- C-ABI of libgamma: batch-dynamic subgraph matching (BDSM) on one
 * GB300 GPU.
 *
 * Problem (Sec. II-A, Def. 1, Def. 2 and the Problem Statement): a labelled
 * undirected data graph G receives a batch of edge insertions and deletions
 * and becomes G'.  For every registered labelled, connected query graph Q the
 * library enumerates the incremental matches: embeddings of Q (injective,
 * label-preserving, every query edge mapped onto a data edge; non-induced)
 * that are in G' but not in G (positive) or in G but not in G' (negative).
 * Every such match uses at least one update edge of its own sign and is
 * charged to exactly one update, the lowest-indexed one among those edges
 * (Sec. IV-C: a total order over updates so that no match is found twice).
 *
 * State machine: create -> [reserve_vertices] -> load_graph -> register_query* ->
 *   (apply_batch -> [fetch_matches | update_counts]* -> commit | add_vertices)*
 *   -> destroy.
 * A second apply_batch before commit returns GAMMA_ESTATE.
 *
 * Pointers: every input array may be host memory (pageable or pinned) or
 * device memory of the context's device; the library tells them apart with
 * cudaPointerGetAttributes and copies host arrays on the context's stream.
 * Inputs stay owned by the caller and are not retained after a call returns.
 * Output buffers are owned by the caller.  All calls are synchronous with
 * respect to the host (they return after their device work has finished).
 *
 * Errors: every int-returning call returns GAMMA_OK (0) or a negative code;
 * gamma_last_error gives a message.  Nothing aborts the process and no call
 * leaves the graph half-updated: an invalid batch is rejected before the
 * graph changes.  One context is used by one host thread at a time.
 */
#ifndef GAMMA_H
#define GAMMA_H

#include <stdint.h>

#if defined(__GNUC__)
#define GAMMA_API __attribute__((visibility("default")))
#else
#define GAMMA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define GAMMA_OK 0
#define GAMMA_EINVAL (-1)    /* bad argument, graph, query or batch */
#define GAMMA_ENOMEM (-2)    /* device or host allocation failed */
#define GAMMA_ESTATE (-3)    /* call not allowed in the current state */
#define GAMMA_EOVERFLOW (-4) /* match buffer too small; counts still exact */
#define GAMMA_ETIMEOUT (-5)  /* work budget exceeded; counts incomplete */
#define GAMMA_ECUDA (-6)     /* CUDA runtime error */

/* option flags */
#define GAMMA_F_PER_UPDATE 0x1u  /* keep per-update charged counts (gamma_update_counts) */
#define GAMMA_F_NO_FILTER 0x2u   /* disable the neighbour-label-count candidate filter */
#define GAMMA_F_PER_QUERY 0x4u   /* plain form: one seed+DFS launch sequence per query */
#define GAMMA_F_GRAPH 0x8u       /* replay the match phase as a captured CUDA graph */
#define GAMMA_F_COUNT_BYTES 0x10u /* count the DFS kernel's algorithmic bytes (gamma_stats.alg_bytes) */
#define GAMMA_F_NO_LEAF 0x20u   /* always enumerate a last query vertex that has one earlier neighbour
                                   (default: count it in closed form when no rows are requested) */
#define GAMMA_F_NO_SHARE 0x40u  /* expand every partial match at the last query vertex (default: when that
                                   vertex is not adjacent to the one before it and no rows are requested,
                                   the children of one partial match share their candidates) */
#define GAMMA_F_SEED_IN_ORDER 0x80u /* create DFS work in update order (default with one staged request:
                                   grouped by each update's higher-degree endpoint, so that warps running
                                   together search around the same vertex); results are the same */
#define GAMMA_F_SEED_BY_QUERY 0x100u /* batched form: create the DFS work query by query (still one DFS launch),
                                   so that warps running together search for the same query */

typedef struct gamma_ctx gamma_ctx;

typedef struct {
  int device;            /* CUDA device ordinal */
  void *cuda_stream;     /* cudaStream_t to run on; NULL = a stream owned by the context */
  uint32_t flags;        /* GAMMA_F_* */
  uint64_t work_budget;  /* max 32-candidate expansion steps per apply; 0 = unlimited */
  int warps_per_block;   /* DFS kernel warps per block (1..16); 0 = 8 */
  int frontier_tile;     /* partial matches buffered per DFS level per warp (32..4096); 0 = 64 */
  int steal_grain;       /* level-2 candidates per work item; 0 = 64 */
  /* Bounded waits of the DFS kernel's work donation (an expired wait ends the
   * apply with GAMMA_ETIMEOUT, counts incomplete, the context still usable): */
  uint32_t idle_limit_us;    /* longest an idle warp waits for donated work while
                                others still hold some; 0 = 60 s */
  uint32_t handoff_limit_us; /* longest a donor waits for a free task slot, or a
                                receiver for its reserved task; 0 = 1 s */
  int32_t hub_min_degree;    /* lists with at least this many entries at load get a
                                hash index for membership tests (memory: about 12
                                bytes per entry of such lists); 0 = 128; takes
                                effect at the next gamma_load_graph */
} gamma_options;

/* Match rows: row r is rows[r*stride .. r*stride+stride): query id, update
 * index, sign (+1/-1), then phi(u_0) .. phi(u_{q-1}) in query-vertex order,
 * then -1 padding.  stride >= 3 + the largest q of the requested queries. */
typedef struct {
  int32_t *rows;      /* caller buffer, host or device */
  int64_t capacity;   /* rows that fit */
  int32_t stride;     /* int32 per row */
  int64_t written;    /* out: rows written (<= capacity) */
  int64_t required;   /* out: rows that exist (written < required => GAMMA_EOVERFLOW) */
} gamma_matches;

typedef struct {
  double ms_stage;     /* batch validation + staging into the dynamic CSR */
  double ms_seed;      /* seeding */
  double ms_match;     /* DFS extension */
  double ms_finalize;  /* count reduction and row compaction */
  double ms_commit;    /* last commit */
  int64_t seeds;       /* seeds that passed the label and filter tests */
  int64_t work_items;  /* DFS work items (seeds split by steal_grain) */
  int64_t touched;     /* vertices whose adjacency the last batch touched */
  int64_t pool_used;   /* adjacency slots allocated (entries) */
  int64_t pool_cap;    /* adjacency slots available */
  int64_t live_edges;  /* directed adjacency entries of the current graph */
  uint64_t expansions; /* 32-candidate expansion steps of the last apply */
  uint64_t alg_bytes;  /* DFS algorithmic bytes of the last apply (GAMMA_F_COUNT_BYTES) */
  uint64_t kernel_launches; /* kernels the library has launched in this process so far */
  int64_t graph_captures;   /* CUDA graphs captured by this context (GAMMA_F_GRAPH) */
  int64_t donated_tasks;    /* work pieces idle warps received from busy ones in the last DFS launch */
} gamma_stats;

/* Create a context on options->device (options may be NULL: defaults).
 * *out receives the context; GAMMA_ECUDA if the device cannot be used. */
GAMMA_API int gamma_create(const gamma_options *options, gamma_ctx **out);

/* Free all device and host state of ctx (NULL is ignored). */
GAMMA_API void gamma_destroy(gamma_ctx *ctx);

/* Load the data graph G (Sec. II-A): n vertices with labels[n] (>= 0), m
 * undirected edges (src[e], dst[e]).  Repeated edges, in either direction,
 * are merged; a self-loop, an id outside [0, n) or a negative label gives
 * GAMMA_EINVAL.  Limit: 1 + ceil(log2 n) + ceil(log2(max label + 1)) <= 32
 * (vertex id and label are packed into one 32-bit adjacency key); labels < 256.
 * Replaces any previously loaded graph and forgets registered queries. */
GAMMA_API int gamma_load_graph(gamma_ctx *ctx, int32_t n, const int32_t *labels,
                     int64_t m, const int32_t *src, const int32_t *dst);

/* Edge-labelled graph (Sec. II-A: the label function covers edges too; the
 * paper's NF and LS datasets, Table II, have edge labels): as
 * gamma_load_graph, with elabels[m] the label of edge e in [0, 255] (host or
 * device).  A repeated edge must repeat its label (else GAMMA_EINVAL).  An
 * embedding must then map every query edge onto a data edge of the query
 * edge's label.  With elabels NULL this is gamma_load_graph (every edge label
 * 0).  Limits: gamma_apply_batches (several requests) and gamma_checkpoint
 * refuse an edge-labelled graph (GAMMA_EINVAL). */
GAMMA_API int gamma_load_graph_el(gamma_ctx *ctx, int32_t n, const int32_t *labels, int64_t m, const int32_t *src,
                                  const int32_t *dst, const int32_t *elabels);

/* Register a query graph Q (Sec. II-A): 2 <= q <= 16 vertices with
 * qlabels[q], eq undirected edges (qsrc[e], qdst[e]) in [0, q).  Q must be
 * connected and simple.  The host builds one matching order per query edge
 * and orientation (Alg. 1 input pi; Sec. IV-C).  *out_qid receives the id. */
GAMMA_API int gamma_register_query(gamma_ctx *ctx, int32_t q, const int32_t *qlabels,
                         int32_t eq, const int32_t *qsrc, const int32_t *qdst,
                         int32_t *out_qid);

/* As gamma_register_query, with qelabels[eq] the label in [0, 255] of each
 * query edge (host array; NULL: all 0).  On a graph without edge labels a
 * query edge labelled other than 0 has no image, so the query never matches. */
GAMMA_API int gamma_register_query_el(gamma_ctx *ctx, int32_t q, const int32_t *qlabels, int32_t eq,
                                      const int32_t *qsrc, const int32_t *qdst, const int32_t *qelabels,
                                      int32_t *out_qid);

/* Apply one update batch Delta-B (Def. 1) of b updates: op[k] = +1 inserts
 * edge (src[k], dst[k]), -1 deletes it; the position k is the update's index
 * in the total order used for charging.  The batch is rejected with
 * GAMMA_EINVAL, leaving G unchanged, if an update has an id out of range, a
 * self-loop, an op other than +1/-1, repeats an edge of an earlier update,
 * inserts an existing edge or deletes a missing one (the message names the
 * smallest offending index).  Otherwise G' is staged and, for each of the nq
 * queries qids[j], out_pos[j] / out_neg[j] (host arrays) receive the number
 * of positive / negative incremental matches.  With opt_out non-NULL the
 * match rows are written too (GAMMA_EOVERFLOW when they do not fit; the
 * counts are exact regardless).  GAMMA_ETIMEOUT: work budget exceeded. */
GAMMA_API int gamma_apply_batch(gamma_ctx *ctx, int64_t b, const int8_t *op,
                      const int32_t *src, const int32_t *dst,
                      int32_t nq, const int32_t *qids,
                      uint64_t *out_pos, uint64_t *out_neg,
                      gamma_matches *opt_out);

/* As gamma_apply_batch on an edge-labelled graph (gamma_load_graph_el):
 * elab[k] in [0, 255] is the label of the edge update k inserts (ignored for
 * a deletion, which removes the edge whatever its label; a label outside the
 * range makes update k invalid).  elab NULL: every insertion gets label 0.
 * GAMMA_EINVAL with elab on a graph loaded without edge labels. */
GAMMA_API int gamma_apply_batch_el(gamma_ctx *ctx, int64_t b, const int8_t *op, const int32_t *src,
                                   const int32_t *dst, const int32_t *elab, int32_t nq, const int32_t *qids,
                                   uint64_t *out_pos, uint64_t *out_neg, gamma_matches *opt_out);

/* Several update requests staged as one batch (continuous batching): request
 * r is updates [req_off[r], req_off[r+1]) of the arrays (req_off[0] = 0,
 * host array of nreq + 1 offsets).  The result is the same as applying the
 * requests one after another (apply + commit each): request r sees the graph
 * after requests 0..r-1, and its counts, out_pos[r*nq + j] / out_neg[r*nq + j]
 * for query qids[j], are its own incremental matches.  Requests may touch the
 * same edges (a later request may delete an edge an earlier one inserted, or
 * insert one it deleted); each request must be valid on the graph the earlier
 * ones leave and touch an edge at most once, else GAMMA_EINVAL with the
 * smallest offending update index and the graph unchanged.  Afterwards the
 * batch is staged as with gamma_apply_batch; gamma_commit applies all of it.
 * No match rows. */
GAMMA_API int gamma_apply_batches(gamma_ctx *ctx, int32_t nreq, const int64_t *req_off, const int8_t *op,
                                  const int32_t *src, const int32_t *dst, int32_t nq, const int32_t *qids,
                                  uint64_t *out_pos, uint64_t *out_neg);

/* Re-run the matching of the staged batch and write its match rows into out
 * (after GAMMA_EOVERFLOW, with a larger buffer).  GAMMA_ESTATE if no batch is
 * staged. */
GAMMA_API int gamma_fetch_matches(gamma_ctx *ctx, gamma_matches *out);

/* Per-update charged counts of the staged batch for the j-th requested query
 * (0 <= j < nq of the last apply_batch): out[k] (host, b entries) = number of
 * incremental matches charged to update k.  Needs GAMMA_F_PER_UPDATE. */
GAMMA_API int gamma_update_counts(gamma_ctx *ctx, int32_t j, uint64_t *out);

/* Make G' the current graph: drop deleted edges, clear batch tags.
 * GAMMA_ESTATE if no batch is staged. */
GAMMA_API int gamma_commit(gamma_ctx *ctx);

/* Copy the current adjacency to host arrays, for checking the dynamic CSR
 * (staging and commit) against a host model.  While a batch is staged this is the union
 * graph G u G'.  off[n+1] (int64) delimits each vertex's list; for entry i,
 * nbr[i] is the neighbour id and tag[i] is -1 for an edge the staged batch
 * does not touch, else 2 * (update index) + (1 for a deletion).  Lists are in
 * the library's order (neighbour label, then id).  cap = room in nbr/tag;
 * returns GAMMA_EOVERFLOW when the entries do not fit (off is still filled). */
GAMMA_API int gamma_export_adjacency(gamma_ctx *ctx, int64_t *off, int32_t *nbr, int32_t *tag, int64_t cap);

/* Vertex updates (Sec. II-A treats a vertex insertion or deletion as edge
 * updates; this build follows that reduction).  The vertex id and the label
 * share one 32-bit adjacency key, so room for vertices added later must be
 * reserved before gamma_load_graph: n_max is the largest vertex count the
 * context will hold (0 = just the loaded n).  Affects the next load only;
 * GAMMA_EINVAL for a negative n_max.  A graph loaded with a larger reserve
 * must still satisfy 1 + ceil(log2 n_max) + label bits <= 32. */
GAMMA_API int gamma_reserve_vertices(gamma_ctx *ctx, int32_t n_max);

/* Append k isolated vertices with labels[k] (host or device; each in the
 * loaded graph's label range [0, max label]).  They get ids n .. n+k-1
 * (*out_first = n, may be NULL) and join G with no edges; edges to them are
 * then inserted by ordinary batches.  GAMMA_ESTATE without a graph or with a
 * staged batch; GAMMA_EINVAL for a bad label or when n + k exceeds the
 * reserved id space (nothing changes then).  Registered queries stay. */
GAMMA_API int gamma_add_vertices(gamma_ctx *ctx, int32_t k, const int32_t *labels, int32_t *out_first);

/* The current neighbours of vertex v (host array out[cap], in the library's
 * order: neighbour label, then id); *count = the degree.  Deleting a vertex
 * is the batch that deletes these edges (the vertex stays, isolated).
 * GAMMA_ESTATE with a staged batch; GAMMA_EOVERFLOW when cap < degree (the
 * first cap ids are written). */
GAMMA_API int gamma_vertex_neighbors(gamma_ctx *ctx, int32_t v, int32_t *out, int64_t cap, int64_t *count);

/* Checkpoint and restore (no counterpart in the paper; commit is the
 * consistency point).  gamma_checkpoint writes the committed graph (labels,
 * edges, reserved vertex count) and the registered queries into the host
 * buffer buf[cap] and sets *size to the bytes needed; GAMMA_EOVERFLOW when
 * cap is too small (nothing partial is usable then; call again with *size),
 * GAMMA_ESTATE without a graph or with a staged batch.  gamma_restore
 * replaces the context's graph and queries with a checkpoint through the
 * ordinary load and register calls (same validation), so the queries keep
 * their ids; GAMMA_EINVAL for a damaged checkpoint.  The format is a plain
 * byte layout of int32 words (see the library source); it is not meant to
 * move between machines of different endianness. */
GAMMA_API int gamma_checkpoint(gamma_ctx *ctx, void *buf, int64_t cap, int64_t *size);
GAMMA_API int gamma_restore(gamma_ctx *ctx, const void *buf, int64_t size);

/* The matching order the library uses when an update is mapped onto query
 * edge (a, b) (Alg. 1 input pi; Sec. IV-C): pi[0] = a, pi[1] = b, then
 * repeatedly the unplaced query vertex with the most placed neighbours, then
 * the higher query degree, then the rarer label in G (label_freq[nlab], the
 * number of data vertices per label; NULL with nlab = 0 treats all labels
 * alike), then the smaller id.  out_order[q] receives pi, out_bwd[q] (may be
 * NULL) the placed-neighbour bit mask of each position.  Host only: needs no
 * context and no GPU.  GAMMA_EINVAL for a query gamma_register_query would
 * refuse, or when (a, b) is not one of its edges. */
GAMMA_API int gamma_plan_order(int32_t q, const int32_t *qlabels, int32_t eq, const int32_t *qsrc,
                               const int32_t *qdst, int32_t a, int32_t b, int32_t nlab,
                               const int64_t *label_freq, int32_t *out_order, uint16_t *out_bwd);

/* Timings and sizes of the last apply/commit. */
GAMMA_API int gamma_get_stats(gamma_ctx *ctx, gamma_stats *out);

/* Change flags / tuning knobs between batches (fields as in gamma_options;
 * 0 keeps the current value for the three tuning fields and the two wait
 * limits; device and cuda_stream are ignored). */
GAMMA_API int gamma_set_options(gamma_ctx *ctx, const gamma_options *options);

/* Autotuner for the batched form: one point of the search grid. */
typedef struct {
  int32_t warps_per_block;  /* 1..16 */
  int32_t frontier_tile;    /* 32..4096 */
  int32_t steal_grain;      /* >= 1 */
  float ms;                 /* out: median seed + DFS time of the point (-1: not runnable) */
} gamma_tune_point;

/* Time the matching of the staged batch (seed + DFS, repeated `repeats` times)
 * at every point of points[0..npoints) and keep the fastest point as the
 * context's configuration (*best receives it, with its time).  The counts do
 * not depend on the point.  GAMMA_ESTATE if no batch is staged. */
GAMMA_API int gamma_autotune(gamma_ctx *ctx, int32_t npoints, gamma_tune_point *points, int32_t repeats,
                             gamma_tune_point *best);

/* Recount the staged batch without allocating anything.  No counterpart in
 * the paper: an operational addition for callers that cannot allocate device
 * memory at the moment they need the counts -- an application whose device
 * memory is entirely reserved by another allocator (a framework's caching
 * allocator or a preallocated arena, where cudaMalloc would fail), or a
 * latency-critical loop that may not pay for cudaMalloc / cudaFree, which can
 * synchronize the whole device.  It re-runs the DFS kernel over the work
 * items the last gamma_apply_batch or gamma_apply_batches kept and writes
 * the counts to the host arrays out_pos / out_neg, laid out as for
 * gamma_apply_batches: entry r * nq + j for request r and query j; nreq = 1
 * after gamma_apply_batch.  cap = entries in each of out_pos / out_neg;
 * GAMMA_EINVAL when cap < nreq * max(nq, 1), nothing written.  The DFS
 * scratch (donated-task ring, scheduling counters, count accumulators)
 * lives in a static device array of about 1.2 MB that every GPU loading the
 * library holds until the process exits; its limits: nreq * nq <= 256 count
 * slots (GAMMA_EINVAL beyond) and 16,384 donated-task slots (a donation that
 * would not fit is not made; the warp keeps the work).  The batched form
 * only (GAMMA_ESTATE with GAMMA_F_PER_QUERY).  The first call on a device
 * looks up the array's device address, with that device current, and keeps
 * it.  All calls share the array, which keeps the last call's contents: each
 * call clears what must start at zero.  Calls whose GPU work overlaps (from
 * several threads or contexts at once) race on the array; do not issue
 * them. */
GAMMA_API int gamma_recount_noalloc(gamma_ctx *ctx, int32_t cap, uint64_t *out_pos, uint64_t *out_neg);

/* ------------------------------------------------------------------------
 * Served form: a worker thread applies a stream of update requests to the
 * device-resident graph, in arrival order.  Requests that arrive while the
 * GPU is busy wait; when it is free the worker stages every waiting request
 * it can admit together (gamma_apply_batches: continuous batching, each
 * request still gets exactly its own result) and commits them.  A group
 * stops at max_requests / max_updates, or when its estimated device memory
 * (staging buffers, work items and adjacency growth per update) would exceed
 * hbm_fraction of the free HBM (admission).  A group that contains an
 * invalid request is served again one request at a time, so only the invalid
 * request fails (GAMMA_EINVAL) and the others get their one-at-a-time
 * results.  A group is one apply, so the context's work_budget bounds the
 * whole group: give it the budget of every request a group may hold, or 0,
 * else a group can end with GAMMA_ETIMEOUT (for all its requests) although
 * each request alone stays within the budget.  While a server runs, its
 * context belongs to the worker thread: call nothing else on it.
 * ------------------------------------------------------------------------ */
typedef struct gamma_server gamma_server;

typedef struct {
  int64_t max_updates;   /* updates staged together at most (0 = 2^21) */
  int32_t max_requests;  /* requests staged together at most (0 = 256) */
  double hbm_fraction;   /* admit while the estimate <= this share of free HBM (0 = 0.5) */
} gamma_server_options;

typedef struct {
  double arrival_ms;   /* submit time (ms since the server started) */
  double start_ms;     /* its group was handed to the GPU */
  double done_ms;      /* its group was committed and counts were on the host */
  int32_t group_size;  /* requests staged together with it (itself included) */
  int32_t status;      /* GAMMA_* of its group */
} gamma_request_info;

typedef struct {
  int64_t groups, requests, updates, max_group;
  double busy_ms;      /* worker time spent in apply + commit */
} gamma_server_stats;

/* Start serving ctx for the nq queries qids (counts are per query). */
GAMMA_API int gamma_server_start(gamma_ctx *ctx, int32_t nq, const int32_t *qids,
                                 const gamma_server_options *options, gamma_server **out);
/* Queue one request of b updates (host arrays, copied before returning; same
 * rules as gamma_apply_batch).  *ticket identifies it.  Thread-safe. */
GAMMA_API int gamma_server_submit(gamma_server *s, int64_t b, const int8_t *op, const int32_t *src,
                                  const int32_t *dst, int64_t *ticket);
/* Block until the request is done; out_pos/out_neg (host, nq each) receive its
 * counts, info its times.  Returns its status; each ticket is waited once. */
GAMMA_API int gamma_server_wait(gamma_server *s, int64_t ticket, uint64_t *out_pos, uint64_t *out_neg,
                                gamma_request_info *info);
GAMMA_API int gamma_server_stats_get(gamma_server *s, gamma_server_stats *out);
/* Finish the queued requests, stop the worker and free the server. */
GAMMA_API int gamma_server_stop(gamma_server *s);

/* Read bandwidth of device `device` for a working set of `bytes` bytes (at
 * least 1 MiB): a streaming kernel reads the buffer `reps` times with loads
 * that bypass L1, best of `trials` timed launches after one warm-up, so a
 * buffer smaller than L2 measures L2 and a larger one DRAM.  *out_gbs gets
 * GB/s (1e9 bytes/s).  No counterpart in the paper: it is the denominator of
 * the roofline of kernels whose working set stays in L2.  Allocates and
 * frees its buffer; GAMMA_ENOMEM if it cannot. */
GAMMA_API int gamma_probe_bandwidth(int device, int64_t bytes, int32_t reps, int32_t trials, double *out_gbs);

/* Message for the last error on ctx (never NULL; "" when none). */
GAMMA_API const char *gamma_last_error(gamma_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* GAMMA_H */
