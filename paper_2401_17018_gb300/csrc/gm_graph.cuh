// gm_graph.cuh -- host entry points of the dynamic-CSR kernels (gm_graph.cu)
// and the match kernels (gm_match.cu).
#pragma once
#include "gm_common.cuh"

// per-batch device buffers (sized for 2b directed entries)
struct StageBufs {
  uint32_t *cu = nullptr, *cv = nullptr;  // canonical endpoints (min, max) per update
  int8_t *cop = nullptr;                  // op per update
  uint64_t *keys = nullptr, *tk = nullptr;
  uint32_t *vals = nullptr, *tv = nullptr;
  uint32_t *head = nullptr, *gid = nullptr;
  uint32_t *gv = nullptr, *gstart = nullptr, *gins = nullptr, *greloc = nullptr;
  uint32_t *bkeys = nullptr;
  // several requests staged together: the updates of one edge form a chain
  // in index order; only its first update (the head) enters the adjacency
  uint32_t *cnext = nullptr;  // [b] next update of the same edge, or ~0
  uint8_t *cinfo = nullptr;   // [b] GM_CHAIN_* bits
  // edge-labelled graphs: the label of each update's edge (an insertion's
  // given label; a deletion's label in G, read while staging)
  uint8_t *ulab = nullptr;    // [b]
  int64_t cap = 0;  // updates
};
#define GM_CHAIN_HEAD 1u      // the update is the first of its edge's chain
#define GM_CHAIN_LONG 2u      // (head) later updates of the same edge follow
#define GM_CHAIN_PRESENT 4u   // (head) the edge exists once the whole chain is applied

// elabels: [m] edge labels in [0, 255] (null: an unlabelled graph)
int gm_load_validate(const int32_t *labels, int32_t n, const int32_t *src, const int32_t *dst,
                     const int32_t *elabels, int64_t m, GmStatus *st, cudaStream_t s);
int gm_load_build(GraphDev g, const int32_t *src, const int32_t *dst, const int32_t *elabels, int64_t m,
                  uint32_t **col_out, uint32_t **etag_out, uint8_t **elab_out, uint32_t *pool_cap_out,
                  double pool_factor, uint64_t pool_reserve, GmStatus *st, GmStatus *h_st, cudaStream_t s);
int gm_nlf(GraphDev g, const uint32_t *verts, const uint32_t *nverts_dev, uint32_t nverts_max, cudaStream_t s);
int gm_hub(GraphDev g, const uint32_t *verts, const uint32_t *nverts_dev, uint32_t nverts_max, GmStatus *st,
           cudaStream_t s);
// req: [b] request of each update when several requests are staged together
// (null: one request); then updates of different requests may touch the same
// edge, each request valid on the graph the earlier ones leave
// elab_in: [b] insertion labels (edge-labelled graphs; null: all 0)
int gm_stage(GraphDev g, const int8_t *op, const int32_t *src, const int32_t *dst, const int32_t *elab_in, int64_t b,
             const uint32_t *req, StageBufs &sb, GmStatus *st, cudaStream_t s);
int gm_commit(GraphDev g, const StageBufs &sb, int64_t b, bool chains, GmStatus *st, cudaStream_t s);
// per-query form: the next DFS launch starts at the items the next seed launch appends
int gm_begin_group(GmStatus *st, cudaStream_t s);

// ---------------------------------------------------------------- matching
struct MatchArgs {
  GraphDev g;
  const uint32_t *cu, *cv;     // canonical endpoints per update
  const int8_t *op;
  const uint8_t *ulab;         // [b] label of each update's edge (edge-labelled graphs), else null
  int64_t b;
  const Plan *plans;
  int nplans;
  const uint32_t *pair_off;    // [nlab*nlab + 1] plans per (L(min), L(max)) label pair
  const uint16_t *pair_plans;
  int grain;                   // level-2 candidates per work item
  WorkItem *items;
  uint64_t item_cap;
  uint64_t *cnt;               // [nreq * nq * 2] positive / negative counts
  const uint32_t *req;         // [b] request of each update (null: one request)
  const uint32_t *cnext;       // [b] next update of the same edge (with req), else null
  int nq;                      // query slots per request
  uint64_t *per_upd;           // [nq * b] or null
  int use_filter;
  int32_t *rows;               // match rows or null
  uint64_t row_cap;
  int row_stride;
  uint64_t budget;
  int tile;                    // DFS frontier tile
  int nlev;                    // stored DFS levels (max q - 3, >= 1)
  int warps_per_block;
  int count_bytes;             // accumulate algorithmic bytes into st->alg_bytes
  int leaf;                    // count a last position with one backward neighbour in closed form
  int share;                   // siblings share last-position candidates (counts only)
  int seed_sorted;             // seed in the order of the sorted batch, each update at its
                               // higher-degree endpoint (needs both entries of every update)
  int qfilter;                 // seed only the plans of this query slot (-1: all)
  const uint64_t *bkeys;       // the staged batch, sorted: (vertex << 33 | deletion << 32 | key)
  const uint32_t *bvals;       // its tags
  const uint32_t *gstart;      // [groups] first sorted entry of each touched vertex
  const uint32_t *gins;        // [groups] insertions of each touched vertex (they come first)
  uint32_t n2;                 // sorted entries (2 per update)
  Task *tasks;                 // donated work (null: no donation)
  uint32_t *sched;             // [GM_SCHED_WORDS] scheduling counters
  uint32_t *task_seq;          // [task_cap] 1 once the task in the slot is written
  uint32_t task_cap;
  uint64_t idle_limit_ns;      // longest an idle warp waits for work before flagging an error
  uint64_t handoff_limit_ns;   // longest a donor waits for a free ring slot, or a receiver for its task
  GmStatus *st;
};

int gm_seed(const MatchArgs &a, cudaStream_t s);
int gm_dfs(const MatchArgs &a, int num_sms, cudaStream_t s);
size_t gm_dfs_smem_per_warp(int tile, int nlev);
