// gm_api.cu -- the C-ABI of libgamma (include/gamma.h): context and state
// machine, host planner (matching orders, Alg. 1 input pi), buffer management
// and the launch sequence of one batch: stage -> seed -> DFS with row
// compaction -> counts to the host; commit separately.  Also here: several
// requests staged together (gamma_apply_batches), the apply recorded once as
// a CUDA graph and replayed (GAMMA_F_GRAPH), the autotuner, vertex additions,
// and checkpoint / restore through the ordinary load and register calls.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "gm_graph.cuh"

static thread_local char g_cuda_msg[512];
unsigned long long gm_launch_count = 0;

int gm_cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
  snprintf(g_cuda_msg, sizeof(g_cuda_msg), "CUDA error %s (%s) in %s at %s:%d", cudaGetErrorName(e),
           cudaGetErrorString(e), what, file, line);
  return (e == cudaErrorMemoryAllocation) ? GAMMA_ENOMEM : GAMMA_ECUDA;
}

namespace {

struct HostQuery {
  int q = 0;
  std::vector<int32_t> lab;
  std::vector<std::pair<int, int>> edges;
  std::vector<int32_t> elab;  // label of each edge (0 without edge labels)
  std::vector<Plan> plans;
  bool never = false;  // a label absent from G: no embedding can exist
};

template <class T>
int ensure(T *&p, int64_t &cap, int64_t need) {
  if (need <= cap && p) return GAMMA_OK;
  if (p) cudaFree(p);
  p = nullptr;
  int64_t c = std::max<int64_t>(need, 1);
  cudaError_t e = cudaMalloc((void **)&p, sizeof(T) * (size_t)c);
  if (e != cudaSuccess) { cap = 0; p = nullptr; return gm_cuda_fail(e, "cudaMalloc", __FILE__, __LINE__); }
  cap = c;
  return GAMMA_OK;
}

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

struct gamma_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  uint32_t flags = 0;
  uint64_t budget = 0;
  int wpb = 8, tile = 64, grain = 64;
  uint64_t idle_ns = 60ull * 1000000000ull;  // bounded waits of the DFS kernel's work donation
  uint64_t handoff_ns = 1000000000ull;
  int hub_min = GM_HUB_MIN;  // list length that gets a hash index at load
  int num_sms = 0;
  std::string err;

  // graph
  bool loaded = false;
  int32_t n = 0;
  int32_t n_reserve = 0;  // vertex count to make room for at the next load
  int32_t n_cap = 0;      // vertices the loaded graph may grow to
  int idb = 1, nlab = 1, nlfw = 4;
  int32_t *d_label = nullptr;
  uint2 *d_adj = nullptr;
  uint32_t *d_cap = nullptr, *d_col = nullptr, *d_etag = nullptr;
  uint8_t *d_elab = nullptr;  // edge label per adjacency entry (edge-labelled graphs only)
  uint8_t *d_nlf = nullptr;
  int32_t *d_vgroup = nullptr;
  int32_t *d_hub_id = nullptr;
  uint32_t *d_hub_lofs = nullptr;
  uint2 *d_hub_tab = nullptr;
  uint32_t *d_hub_keys = nullptr;
  uint32_t hub_keys_cap = 0;
  uint64_t hub_top = 0;
  int32_t nhub = 0;
  uint32_t pool_cap = 0;
  uint64_t pool_top = 0;
  int64_t live = 0;
  std::vector<int64_t> label_freq;

  // queries
  std::vector<HostQuery> queries;

  // batch
  StageBufs sb;
  int64_t in_cap = 0;
  int8_t *d_in_op = nullptr;
  int32_t *d_in_src = nullptr, *d_in_dst = nullptr, *d_in_elab = nullptr;
  bool staged = false;
  int64_t b = 0;
  std::vector<int32_t> qids;

  // match
  Plan *d_plans = nullptr;
  int64_t plans_cap = 0;
  uint32_t *d_pair_off = nullptr;
  int64_t pair_off_cap = 0;
  uint16_t *d_pair_plans = nullptr;
  int64_t pair_plans_cap = 0;
  std::vector<int32_t> plan_key;  // qids + form the device tables were built for
  std::vector<int> group_nplans;
  int nplans = 0, maxq = 2;
  WorkItem *d_items = nullptr;
  int64_t items_cap = 0;
  uint64_t *d_cnt = nullptr;
  int64_t cnt_cap = 0;
  uint64_t *d_per_upd = nullptr;
  int64_t per_upd_cap = 0;
  int32_t *d_rows = nullptr;
  int64_t rows_cap = 0;
  uint32_t *d_sched = nullptr;
  int64_t sched_cap = 0;
  Task *d_tasks = nullptr;
  int64_t tasks_cap = 0;
  uint32_t *d_task_seq = nullptr;
  int64_t task_seq_cap = 0;

  uint32_t *d_req = nullptr;      // request of each update (several requests staged together)
  int64_t req_cap = 0;
  int nreq = 1;
  cudaGraphExec_t gexec = nullptr;  // last captured apply (GAMMA_F_GRAPH)
  std::vector<int64_t> gkey;
  int64_t graph_captures = 0;

  GmStatus *d_st = nullptr;
  GmStatus *h_st_init = nullptr;  // pinned: status at the start of an apply
  GmStatus *h_st = nullptr;       // pinned
  uint64_t *h_cnt = nullptr;      // pinned
  int64_t h_cnt_cap = 0;
  cudaEvent_t ev[8] = {};
  gamma_stats stats = {};

  GraphDev gd() const {
    GraphDev g;
    g.label = d_label; g.adj = d_adj; g.cap = d_cap; g.col = d_col; g.etag = d_etag; g.nlf = d_nlf;
    g.elab = d_elab;
    g.vgroup = d_vgroup;
    g.hub_id = d_hub_id; g.hub_lofs = d_hub_lofs; g.hub_tab = d_hub_tab; g.hub_keys = d_hub_keys;
    g.hub_keys_cap = hub_keys_cap; g.nhub = nhub;
    g.n = n; g.idb = idb; g.nlab = nlab; g.nlfw = nlfw;
    g.idmask = (idb >= 32) ? 0xffffffffu : ((1u << idb) - 1u);
    g.pool_cap = pool_cap;
    return g;
  }

  int fail(int code, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    err = buf;
    return code;
  }
  int cuda_fail(int code) {
    err = g_cuda_msg;
    return code;
  }
};

#define CK(call)                                        \
  do {                                                  \
    int rc__ = (call);                                  \
    if (rc__ != GAMMA_OK) return ctx->cuda_fail(rc__);  \
  } while (0)
#define CKC(call) CK(((call) == cudaSuccess) ? GAMMA_OK : gm_cuda_fail(cudaGetLastError(), #call, __FILE__, __LINE__))

namespace {

// a captured apply bakes the graph's device pointers into its kernels: forget
// it whenever those arrays are freed or moved
void drop_graph_exec(gamma_ctx *ctx) {
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  ctx->gexec = nullptr;
  ctx->gkey.clear();
}

// grow a per-vertex device array from n to n2 elements: old contents kept,
// the new tail set to the byte `fill`
template <typename T>
int grow_vertex_array(gamma_ctx *ctx, T **arr, size_t per, int32_t n, int32_t n2, int fill) {
  T *fresh = nullptr;
  CKC(cudaMalloc((void **)&fresh, per * (size_t)n2));
  CKC(cudaMemcpyAsync(fresh, *arr, per * (size_t)n, cudaMemcpyDeviceToDevice, ctx->stream));
  CKC(cudaMemsetAsync(reinterpret_cast<char *>(fresh) + per * (size_t)n, fill, per * (size_t)(n2 - n), ctx->stream));
  CKC(cudaStreamSynchronize(ctx->stream));
  cudaFree(*arr);
  *arr = fresh;
  return GAMMA_OK;
}

void free_graph(gamma_ctx *ctx) {
  drop_graph_exec(ctx);
  cudaFree(ctx->d_label); cudaFree(ctx->d_adj); cudaFree(ctx->d_cap);
  cudaFree(ctx->d_col); cudaFree(ctx->d_etag); cudaFree(ctx->d_nlf); cudaFree(ctx->d_elab);
  ctx->d_elab = nullptr;
  cudaFree(ctx->d_hub_id); cudaFree(ctx->d_hub_lofs); cudaFree(ctx->d_hub_tab); cudaFree(ctx->d_hub_keys);
  cudaFree(ctx->d_vgroup);
  ctx->d_vgroup = nullptr;
  ctx->d_label = nullptr; ctx->d_adj = nullptr; ctx->d_cap = nullptr;
  ctx->d_col = nullptr; ctx->d_etag = nullptr; ctx->d_nlf = nullptr;
  ctx->d_hub_id = nullptr; ctx->d_hub_lofs = nullptr; ctx->d_hub_tab = nullptr; ctx->d_hub_keys = nullptr;
  ctx->nhub = 0; ctx->hub_keys_cap = 0; ctx->hub_top = 0;
  ctx->loaded = false;
  ctx->staged = false;
}

int bits_for(int64_t x) {  // bits to represent values 0..x-1 (>= 1)
  int b = 1;
  while (b < 63 && ((int64_t)1 << b) < x) b++;
  return b;
}

// matching order for one seeded query edge (Alg. 1 input pi; Sec. IV-C: more
// selective vertices first): every next vertex has an already placed query
// neighbour; prefer more placed neighbours, then higher degree, then a rarer
// label in G, then the smaller id.
void make_plan(const HostQuery &Q, int qid, int a, int b, const std::vector<int64_t> &freq, Plan &P) {
  const int q = Q.q;
  std::vector<std::vector<char>> adjq(q, std::vector<char>(q, 0));
  std::vector<std::vector<int>> elq(q, std::vector<int>(q, 0));  // query edge labels
  std::vector<int> deg(q, 0);
  for (size_t i = 0; i < Q.edges.size(); i++) {
    const auto &e = Q.edges[i];
    adjq[e.first][e.second] = adjq[e.second][e.first] = 1;
    deg[e.first]++; deg[e.second]++;
    elq[e.first][e.second] = elq[e.second][e.first] = i < Q.elab.size() ? Q.elab[i] : 0;
  }
  std::vector<int> order = {a, b};
  std::vector<char> placed(q, 0);
  placed[a] = placed[b] = 1;
  while ((int)order.size() < q) {
    int best = -1;
    long long bk[4] = {0, 0, 0, 0};
    for (int u = 0; u < q; u++) {
      if (placed[u]) continue;
      int nb = 0;
      for (int w : order) nb += adjq[u][w];
      if (!nb) continue;
      long long f = (Q.lab[u] < (int)freq.size()) ? freq[Q.lab[u]] : 0;
      long long key[4] = {nb, deg[u], -f, -u};
      if (best < 0 || std::lexicographical_compare(bk, bk + 4, key, key + 4)) {
        best = u;
        memcpy(bk, key, sizeof(bk));
      }
    }
    order.push_back(best);
    placed[best] = 1;
  }
  memset(&P, 0, sizeof(P));
  P.q = q;
  P.qid = qid;
  for (int l = 0; l < q; l++) {
    int u = order[l];
    P.qv[l] = (int8_t)u;
    P.lab[l] = Q.lab[u];
    uint16_t bw = 0, sl = 0;
    for (int k = 0; k < l; k++) {
      if (adjq[u][order[k]]) bw |= (uint16_t)(1u << k);
      P.el[l][k] = (uint8_t)elq[u][order[k]];
      if (Q.lab[order[k]] == Q.lab[u]) sl |= (uint16_t)(1u << k);
    }
    P.bwd[l] = bw;
    P.samelab[l] = sl;
    // neighbour-label counts of u in Q (Sec. IV-B: |N^l(v)| >= |N^l(u)|)
    std::vector<std::pair<int, int>> req;
    for (int w = 0; w < q; w++) {
      if (!adjq[u][w]) continue;
      bool found = false;
      for (auto &r : req) if (r.first == Q.lab[w]) { r.second++; found = true; }
      if (!found) req.push_back({Q.lab[w], 1});
    }
    P.nreq[l] = (uint8_t)req.size();
    for (size_t r = 0; r < req.size(); r++) {
      P.req_lab[l][r] = (uint8_t)req[r].first;
      P.req_cnt[l][r] = (uint8_t)req[r].second;
    }
  }
}

// Plan table for one call: all plans of the requested queries (qslot = the
// query's position in the call), plus one (L(pi[0]), L(pi[1])) -> plans index
// per launch group (one group in the batched form, one per query in the
// per-query form).  Uploaded once; reused while the request is unchanged.
int build_tables(gamma_ctx *ctx, const std::vector<int32_t> &qids, bool per_query) {
  std::vector<int32_t> key(qids);
  key.push_back(per_query ? -2 : -1);
  key.push_back((int32_t)ctx->nlab);
  if (key == ctx->plan_key && ctx->d_plans) return GAMMA_OK;
  const int nq = (int)qids.size();
  std::vector<Plan> table;
  std::vector<int> qstart(nq + 1, 0);
  int maxq = 2;
  for (int j = 0; j < nq; j++) {
    qstart[j] = (int)table.size();
    const HostQuery &Q = ctx->queries[qids[j]];
    if (!Q.never) {
      for (const Plan &p0 : Q.plans) {
        Plan p = p0;
        p.qslot = j;
        table.push_back(p);
        maxq = std::max(maxq, p.q);
      }
    }
  }
  qstart[nq] = (int)table.size();
  if (table.size() > 65535) return ctx->fail(GAMMA_EINVAL, "too many matching plans in one call (%zu > 65535)", table.size());
  const int np = ctx->nlab * ctx->nlab;
  const int ngroups = per_query ? nq : 1;
  std::vector<uint32_t> off((size_t)ngroups * (np + 1), 0);
  std::vector<uint16_t> pp;
  ctx->group_nplans.assign(ngroups, 0);
  for (int gi = 0; gi < ngroups; gi++) {
    int p0 = per_query ? qstart[gi] : 0, p1 = per_query ? qstart[gi + 1] : (int)table.size();
    uint32_t *o = off.data() + (size_t)gi * (np + 1);
    for (int i = p0; i < p1; i++) o[table[i].lab[0] * ctx->nlab + table[i].lab[1] + 1]++;
    for (int i = 0; i < np; i++) o[i + 1] += o[i];
    size_t base = pp.size();
    pp.resize(base + (p1 - p0));
    std::vector<uint32_t> fill(o, o + np);
    for (int i = p0; i < p1; i++) pp[base + fill[table[i].lab[0] * ctx->nlab + table[i].lab[1]]++] = (uint16_t)i;
    for (int i = 0; i <= np; i++) o[i] += (uint32_t)base;
    ctx->group_nplans[gi] = p1 - p0;
  }
  if (pp.empty()) pp.push_back(0);
  CK(ensure(ctx->d_plans, ctx->plans_cap, (int64_t)std::max<size_t>(table.size(), 1)));
  CK(ensure(ctx->d_pair_off, ctx->pair_off_cap, (int64_t)off.size()));
  CK(ensure(ctx->d_pair_plans, ctx->pair_plans_cap, (int64_t)pp.size()));
  if (!table.empty())
    CKC(cudaMemcpyAsync(ctx->d_plans, table.data(), sizeof(Plan) * table.size(), cudaMemcpyHostToDevice, ctx->stream));
  CKC(cudaMemcpyAsync(ctx->d_pair_off, off.data(), sizeof(uint32_t) * off.size(), cudaMemcpyHostToDevice, ctx->stream));
  CKC(cudaMemcpyAsync(ctx->d_pair_plans, pp.data(), sizeof(uint16_t) * pp.size(), cudaMemcpyHostToDevice, ctx->stream));
  CKC(cudaStreamSynchronize(ctx->stream));  // host vectors go out of scope
  ctx->nplans = (int)table.size();
  ctx->maxq = maxq;
  ctx->plan_key = key;
  return GAMMA_OK;
}

int grow_pool(gamma_ctx *ctx, uint64_t need) {
  uint64_t cap = std::max<uint64_t>((uint64_t)(ctx->pool_cap * 1.5), need + (need >> 2) + 1024);
  if (cap >= (1ull << 32) - 64) cap = (1ull << 32) - 64;
  if (cap <= ctx->pool_cap) return ctx->fail(GAMMA_ENOMEM, "adjacency pool cannot grow past 2^32 slots");
  uint32_t *col = nullptr, *etag = nullptr;
  uint8_t *elab = nullptr;
  CKC(cudaMalloc((void **)&col, sizeof(uint32_t) * (cap + GM_COL_PAD)));  // padded: short lists are read in 16-byte words
  CKC(cudaMalloc((void **)&etag, sizeof(uint32_t) * cap));
  if (ctx->d_elab) CKC(cudaMalloc((void **)&elab, cap + GM_COL_PAD));
  CKC(cudaMemcpyAsync(col, ctx->d_col, sizeof(uint32_t) * ctx->pool_top, cudaMemcpyDeviceToDevice, ctx->stream));
  CKC(cudaMemcpyAsync(etag, ctx->d_etag, sizeof(uint32_t) * ctx->pool_top, cudaMemcpyDeviceToDevice, ctx->stream));
  if (elab) CKC(cudaMemcpyAsync(elab, ctx->d_elab, ctx->pool_top, cudaMemcpyDeviceToDevice, ctx->stream));
  CKC(cudaStreamSynchronize(ctx->stream));
  cudaFree(ctx->d_col);
  cudaFree(ctx->d_etag);
  cudaFree(ctx->d_elab);
  ctx->d_col = col;
  ctx->d_etag = etag;
  ctx->d_elab = elab;
  ctx->pool_cap = (uint32_t)cap;
  return GAMMA_OK;
}

void reset_status_host(gamma_ctx *ctx) {
  GmStatus *t = ctx->h_st_init;
  memset(t, 0, sizeof(GmStatus));
  t->bad_index = INT64_MAX;
  t->pool_top = (uint32_t)ctx->pool_top;
  t->hub_top = (uint32_t)ctx->hub_top;
}

float ev_ms(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) { cudaGetLastError(); return 0.f; }
  return ms;
}

// device buffers for a batch of b updates, nreq requests and the requested queries
int prepare_buffers(gamma_ctx *ctx, int64_t b) {
  StageBufs &sb = ctx->sb;
  if (b > sb.cap) {
    int64_t c = std::max<int64_t>(b, 1024);
    void *ps[] = {sb.cu, sb.cv, sb.cop, sb.keys, sb.tk, sb.vals, sb.tv, sb.head, sb.gid, sb.gv, sb.gstart,
                  sb.gins, sb.greloc, sb.bkeys, sb.cnext, sb.cinfo, sb.ulab};
    for (void *p : ps) if (p) cudaFree(p);
    sb = StageBufs();
    CKC(cudaMalloc((void **)&sb.cu, 4 * c)); CKC(cudaMalloc((void **)&sb.cv, 4 * c));
    CKC(cudaMalloc((void **)&sb.cop, c));
    CKC(cudaMalloc((void **)&sb.keys, 16 * c)); CKC(cudaMalloc((void **)&sb.tk, 16 * c));
    CKC(cudaMalloc((void **)&sb.vals, 8 * c)); CKC(cudaMalloc((void **)&sb.tv, 8 * c));
    CKC(cudaMalloc((void **)&sb.head, 8 * c)); CKC(cudaMalloc((void **)&sb.gid, 8 * c));
    CKC(cudaMalloc((void **)&sb.gv, 8 * c)); CKC(cudaMalloc((void **)&sb.gstart, 8 * c));
    CKC(cudaMalloc((void **)&sb.gins, 8 * c)); CKC(cudaMalloc((void **)&sb.greloc, 8 * c));
    CKC(cudaMalloc((void **)&sb.bkeys, 8 * c));
    CKC(cudaMalloc((void **)&sb.cnext, 4 * c));
    CKC(cudaMalloc((void **)&sb.cinfo, c));
    CKC(cudaMalloc((void **)&sb.ulab, c));
    sb.cap = c;
  }
  if (b > ctx->in_cap) {
    cudaFree(ctx->d_in_op); cudaFree(ctx->d_in_src); cudaFree(ctx->d_in_dst); cudaFree(ctx->d_in_elab);
    ctx->d_in_op = nullptr; ctx->d_in_src = nullptr; ctx->d_in_dst = nullptr; ctx->d_in_elab = nullptr;
    int64_t c = std::max<int64_t>(b, 1024);
    CKC(cudaMalloc((void **)&ctx->d_in_op, c));
    CKC(cudaMalloc((void **)&ctx->d_in_src, 4 * c));
    CKC(cudaMalloc((void **)&ctx->d_in_dst, 4 * c));
    CKC(cudaMalloc((void **)&ctx->d_in_elab, 4 * c));
    ctx->in_cap = c;
  }
  const int nq = (int)ctx->qids.size();
  const int64_t ncnt = (int64_t)2 * std::max(nq, 1) * ctx->nreq;
  CK(ensure(ctx->d_cnt, ctx->cnt_cap, ncnt));
  if (ctx->flags & GAMMA_F_PER_UPDATE) CK(ensure(ctx->d_per_upd, ctx->per_upd_cap, std::max<int64_t>((int64_t)nq * b, 1)));
  if (ctx->h_cnt_cap < ncnt) {
    if (ctx->h_cnt) cudaFreeHost(ctx->h_cnt);
    CKC(cudaMallocHost((void **)&ctx->h_cnt, sizeof(uint64_t) * ncnt));
    ctx->h_cnt_cap = ncnt;
  }
  if (ctx->items_cap == 0) CK(ensure(ctx->d_items, ctx->items_cap, std::max<int64_t>(1 << 20, 8 * b)));
  if (ctx->tasks_cap == 0) {
    CK(ensure(ctx->d_tasks, ctx->tasks_cap, (int64_t)1 << 20));
    CK(ensure(ctx->d_task_seq, ctx->task_seq_cap, ctx->tasks_cap));
    CK(ensure(ctx->d_sched, ctx->sched_cap, GM_SCHED_WORDS));
  }
  if (ctx->nreq > 1) CK(ensure(ctx->d_req, ctx->req_cap, std::max<int64_t>(b, 1)));
  return build_tables(ctx, ctx->qids, (ctx->flags & GAMMA_F_PER_QUERY) != 0);
}

// status reset + stage; no host sync
int enqueue_stage(gamma_ctx *ctx, const int8_t *dop, const int32_t *dsrc, const int32_t *ddst, const int32_t *delab) {
  cudaStream_t s = ctx->stream;
  CKC(cudaMemcpyAsync(ctx->d_st, ctx->h_st_init, sizeof(GmStatus), cudaMemcpyHostToDevice, s));
  CKC(cudaEventRecord(ctx->ev[0], s));
  if (ctx->b > 0)
    CK(gm_stage(ctx->gd(), dop, dsrc, ddst, delab, ctx->b, ctx->nreq > 1 ? ctx->d_req : nullptr, ctx->sb, ctx->d_st,
                s));
  CKC(cudaEventRecord(ctx->ev[1], s));
  return GAMMA_OK;
}

// seed + DFS (with counting and rows) for the staged batch, then counts and status to
// the host; no host sync.  The kernels do nothing once an error is flagged.
int enqueue_match(gamma_ctx *ctx, int32_t *rows_dev, uint64_t row_cap, int row_stride, bool clear_err) {
  const int nq = (int)ctx->qids.size();
  const int64_t b = ctx->b;
  const bool per_query = (ctx->flags & GAMMA_F_PER_QUERY) != 0;
  const int64_t ncnt = (int64_t)2 * std::max(nq, 1) * ctx->nreq;
  cudaStream_t s = ctx->stream;
  CKC(cudaMemsetAsync(ctx->d_cnt, 0, sizeof(uint64_t) * ncnt, s));
  if (ctx->flags & GAMMA_F_PER_UPDATE)
    CKC(cudaMemsetAsync(ctx->d_per_upd, 0, sizeof(uint64_t) * std::max<int64_t>((int64_t)nq * b, 1), s));
  // clear the match part of the status (abort and nseeds..rows); errors of the stage stay
  if (clear_err) CKC(cudaMemsetAsync(&ctx->d_st->err, 0, sizeof(int32_t), s));
  CKC(cudaMemsetAsync(&ctx->d_st->abort, 0, sizeof(int32_t), s));
  CKC(cudaMemsetAsync(&ctx->d_st->nseeds, 0, 5 * sizeof(uint64_t), s));
  CKC(cudaMemsetAsync(&ctx->d_st->alg_bytes, 0, sizeof(uint64_t), s));
  CKC(cudaEventRecord(ctx->ev[2], s));
  MatchArgs a;
  a.g = ctx->gd();
  a.cu = ctx->sb.cu; a.cv = ctx->sb.cv; a.op = ctx->sb.cop; a.b = b;
  a.ulab = ctx->d_elab ? ctx->sb.ulab : nullptr;
  a.grain = ctx->grain;
  a.items = ctx->d_items; a.item_cap = (uint64_t)ctx->items_cap;
  a.cnt = ctx->d_cnt;
  a.req = (ctx->nreq > 1) ? ctx->d_req : nullptr;
  a.cnext = (ctx->nreq > 1) ? ctx->sb.cnext : nullptr;
  a.nq = std::max(nq, 1);
  a.per_upd = (ctx->flags & GAMMA_F_PER_UPDATE) ? ctx->d_per_upd : nullptr;
  a.use_filter = (ctx->flags & GAMMA_F_NO_FILTER) ? 0 : 1;
  a.rows = rows_dev; a.row_cap = row_cap; a.row_stride = row_stride;
  a.budget = ctx->budget;
  a.tile = ctx->tile;
  a.warps_per_block = ctx->wpb;
  a.count_bytes = (ctx->flags & GAMMA_F_COUNT_BYTES) ? 1 : 0;
  // the closed-form count of a last vertex assumes every slot of its driver
  // slice is an edge it may use; edge labels break that, so it is off then
  a.leaf = ((ctx->flags & GAMMA_F_NO_LEAF) || ctx->d_elab) ? 0 : 1;
  a.share = (rows_dev == nullptr && !(ctx->flags & GAMMA_F_NO_SHARE)) ? 1 : 0;
  a.bkeys = ctx->sb.keys;
  a.bvals = ctx->sb.vals;
  a.gstart = ctx->sb.gstart;
  a.gins = ctx->sb.gins;
  a.n2 = (uint32_t)(2 * b);
  // the sorted batch holds both entries of every update only when one request is staged
  // (a later update of an edge shared by several requests has none)
  a.seed_sorted = (ctx->nreq <= 1 && !(ctx->flags & GAMMA_F_SEED_IN_ORDER)) ? 1 : 0;
  a.qfilter = -1;
  a.tasks = ctx->d_tasks;
  a.sched = ctx->d_sched;
  a.task_seq = ctx->d_task_seq;
  a.task_cap = (uint32_t)ctx->tasks_cap;
  a.idle_limit_ns = ctx->idle_ns;
  a.handoff_limit_ns = ctx->handoff_ns;
  a.st = ctx->d_st;
  a.plans = ctx->d_plans; a.nplans = ctx->nplans;
  a.pair_plans = ctx->d_pair_plans;
  a.nlev = std::max(1, ctx->maxq - 3);
  const int np = ctx->nlab * ctx->nlab;
  const int ngroups = per_query ? nq : 1;
  bool seeded = false;
  for (int gi = 0; gi < ngroups; gi++) {
    if (ctx->group_nplans[gi] == 0) continue;
    a.pair_off = ctx->d_pair_off + (size_t)gi * (np + 1);
    if (per_query) CK(gm_begin_group(ctx->d_st, s));
    if (!per_query && (ctx->flags & GAMMA_F_SEED_BY_QUERY) && nq > 1) {
      // one seeding pass per query into the same work list, one DFS launch
      for (int j = 0; j < nq; j++) {
        a.qfilter = j;
        CK(gm_seed(a, s));
      }
      a.qfilter = -1;
    } else {
      CK(gm_seed(a, s));
    }
    CKC(cudaMemsetAsync(ctx->d_task_seq, 0, sizeof(uint32_t) * ctx->tasks_cap, s));
    if (!per_query) { CKC(cudaEventRecord(ctx->ev[3], s)); seeded = true; }
    CK(gm_dfs(a, ctx->num_sms, s));
  }
  if (!seeded) CKC(cudaEventRecord(ctx->ev[3], s));
  CKC(cudaEventRecord(ctx->ev[4], s));
  CKC(cudaMemcpyAsync(ctx->h_cnt, ctx->d_cnt, sizeof(uint64_t) * ncnt, cudaMemcpyDeviceToHost, s));
  CKC(cudaMemcpyAsync(ctx->h_st, ctx->d_st, sizeof(GmStatus), cudaMemcpyDeviceToHost, s));
  CKC(cudaEventRecord(ctx->ev[5], s));
  return GAMMA_OK;
}

void match_stats(gamma_ctx *ctx) {
  const GmStatus &st = *ctx->h_st;
  ctx->stats.ms_seed = ev_ms(ctx->ev[2], ctx->ev[3]);
  ctx->stats.ms_match = ev_ms(ctx->ev[3], ctx->ev[4]);
  ctx->stats.ms_finalize = ev_ms(ctx->ev[4], ctx->ev[5]);
  ctx->stats.seeds = (int64_t)st.nseeds;
  ctx->stats.work_items = (int64_t)st.nitems;
  ctx->stats.expansions = st.expansions;
  ctx->stats.alg_bytes = st.alg_bytes;
  ctx->stats.donated_tasks = st.tasks_donated;
}

// the match phase alone, with retries when the work item buffer was too small
int run_match(gamma_ctx *ctx, int32_t *rows_dev, uint64_t row_cap, int row_stride) {
  for (int attempt = 0; attempt < 4; attempt++) {
    CK(prepare_buffers(ctx, ctx->b));
    CK(enqueue_match(ctx, rows_dev, row_cap, row_stride, true));
    CKC(cudaStreamSynchronize(ctx->stream));
    GmStatus &st = *ctx->h_st;
    if (st.err == 0 && st.nitems > (uint64_t)ctx->items_cap) {
      int64_t need = (int64_t)(st.nitems + (st.nitems >> 2) + 1024);
      ctx->items_cap = 0;
      CK(ensure(ctx->d_items, ctx->items_cap, need));
      continue;
    }
    match_stats(ctx);
    return GAMMA_OK;
  }
  return ctx->fail(GAMMA_ENOMEM, "work item buffer kept overflowing");
}

// rows destination for a gamma_matches request (device pointer to write)
int rows_target(gamma_ctx *ctx, gamma_matches *out, int32_t **rows, bool *dev) {
  *rows = nullptr;
  *dev = false;
  if (!out) return GAMMA_OK;
  if (out->capacity < 0 || (out->capacity > 0 && !out->rows)) return ctx->fail(GAMMA_EINVAL, "bad gamma_matches buffer");
  int need_stride = 3 + 2;
  for (int32_t id : ctx->qids) need_stride = std::max(need_stride, 3 + ctx->queries[id].q);
  if (out->stride < need_stride) return ctx->fail(GAMMA_EINVAL, "gamma_matches.stride %d < %d", out->stride, need_stride);
  *dev = is_device_ptr(out->rows);
  *rows = out->rows;
  if (!*dev) {
    CK(ensure(ctx->d_rows, ctx->rows_cap, std::max<int64_t>(out->capacity * out->stride, 1)));
    *rows = ctx->d_rows;
  }
  return GAMMA_OK;
}

int copy_rows_out(gamma_ctx *ctx, gamma_matches *out, bool dev_rows) {
  uint64_t produced = ctx->h_st->rows;
  int64_t written = (int64_t)std::min<uint64_t>(produced, (uint64_t)out->capacity);
  if (!dev_rows && written > 0)
    CKC(cudaMemcpy(out->rows, ctx->d_rows, sizeof(int32_t) * (size_t)written * out->stride, cudaMemcpyDeviceToHost));
  out->written = written;
  out->required = (int64_t)produced;
  return (int64_t)produced > out->capacity ? GAMMA_EOVERFLOW : GAMMA_OK;
}

int match_with_rows(gamma_ctx *ctx, gamma_matches *out) {
  int32_t *rows;
  bool dev;
  CK(rows_target(ctx, out, &rows, &dev));
  int rc = run_match(ctx, rows, out ? (uint64_t)out->capacity : 0, out ? out->stride : 0);
  if (rc) return rc;
  if (!out || ctx->h_st->err) return GAMMA_OK;  // errors are reported by the caller
  return copy_rows_out(ctx, out, dev);
}

// stage + match in one stream sequence (optionally replayed as a CUDA graph),
// one host sync; retried after growing the adjacency pool or the item buffer
int run_apply(gamma_ctx *ctx, const int8_t *dop, const int32_t *dsrc, const int32_t *ddst, const int32_t *delab,
              int32_t *rows, uint64_t row_cap, int row_stride) {
  cudaStream_t s = ctx->stream;
  for (int attempt = 0; attempt < 4; attempt++) {
    CK(prepare_buffers(ctx, ctx->b));
    reset_status_host(ctx);
    if (ctx->flags & GAMMA_F_GRAPH) {
      std::vector<int64_t> key = {ctx->b, ctx->nreq, (int64_t)ctx->flags, ctx->tile, ctx->wpb, ctx->grain,
                                  (int64_t)ctx->budget, (int64_t)(intptr_t)rows, (int64_t)row_cap, row_stride,
                                  (int64_t)(intptr_t)dop, (int64_t)(intptr_t)dsrc, (int64_t)(intptr_t)ddst,
                                  (int64_t)(intptr_t)ctx->d_col, (int64_t)(intptr_t)ctx->d_etag, ctx->pool_cap,
                                  (int64_t)(intptr_t)ctx->d_items, ctx->items_cap, (int64_t)(intptr_t)ctx->d_plans,
                                  (int64_t)(intptr_t)ctx->d_pair_off, (int64_t)(intptr_t)ctx->d_pair_plans,
                                  (int64_t)(intptr_t)ctx->sb.cu, (int64_t)(intptr_t)ctx->d_cnt,
                                  (int64_t)(intptr_t)ctx->d_per_upd, (int64_t)(intptr_t)ctx->d_req,
                                  (int64_t)(intptr_t)ctx->h_cnt, ctx->nplans, ctx->maxq, (int64_t)(intptr_t)delab,
                                  (int64_t)(intptr_t)ctx->d_elab, (int64_t)(intptr_t)ctx->sb.ulab};
      key.insert(key.end(), ctx->plan_key.begin(), ctx->plan_key.end());
      if (key != ctx->gkey || !ctx->gexec) {
        cudaGraph_t graph = nullptr;
        CKC(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
        int rc1 = enqueue_stage(ctx, dop, dsrc, ddst, delab);
        int rc2 = rc1 ? rc1 : enqueue_match(ctx, rows, row_cap, row_stride, false);
        cudaError_t ce = cudaStreamEndCapture(s, &graph);
        if (rc2) { if (graph) cudaGraphDestroy(graph); return ctx->cuda_fail(rc2); }
        CKC(ce);
        if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; }
        cudaError_t ie = cudaGraphInstantiate(&ctx->gexec, graph, 0);
        cudaGraphDestroy(graph);
        CKC(ie);
        ctx->gkey = key;
        ctx->graph_captures++;
      }
      CKC(cudaGraphLaunch(ctx->gexec, s));
    } else {
      CK(enqueue_stage(ctx, dop, dsrc, ddst, delab));
      CK(enqueue_match(ctx, rows, row_cap, row_stride, false));
    }
    CKC(cudaStreamSynchronize(s));
    GmStatus &st = *ctx->h_st;
    if (st.err == GAMMA_ENOMEM) {  // the stage changed nothing; grow the pool and redo
      CK(grow_pool(ctx, ctx->pool_top + st.reloc_total));
      continue;
    }
    // a stage error (invalid batch) leaves the graph unchanged; a timeout is
    // raised by the match phase, after the batch was staged
    if (st.err && st.err != GAMMA_ETIMEOUT) return GAMMA_OK;  // reported by the caller
    ctx->pool_top = st.pool_top;
    ctx->hub_top = st.hub_top;
    ctx->stats.ms_stage = ev_ms(ctx->ev[0], ctx->ev[1]);
    ctx->stats.touched = st.ntouched;
    ctx->staged = true;
    if (!st.err && st.nitems > (uint64_t)ctx->items_cap) {  // staged; redo the match phase with more room
      int64_t need = (int64_t)(st.nitems + (st.nitems >> 2) + 1024);
      ctx->items_cap = 0;
      CK(ensure(ctx->d_items, ctx->items_cap, need));
      return run_match(ctx, rows, row_cap, row_stride);
    }
    match_stats(ctx);
    return GAMMA_OK;
  }
  return ctx->fail(GAMMA_ENOMEM, "apply kept running out of device memory");
}

int apply_impl(gamma_ctx *ctx, const char *fn, int32_t nreq, const int64_t *req_off, int64_t b, const int8_t *op,
               const int32_t *src, const int32_t *dst, const int32_t *elab, int32_t nq, const int32_t *qids,
               uint64_t *out_pos, uint64_t *out_neg, gamma_matches *opt_out) {
  if (!ctx) return GAMMA_EINVAL;
  ctx->err.clear();
  if (!ctx->loaded) return ctx->fail(GAMMA_ESTATE, "%s: no graph loaded", fn);
  if (ctx->staged) return ctx->fail(GAMMA_ESTATE, "%s: previous batch not committed", fn);
  if (b < 0 || b >= ((int64_t)1 << 31) || nq < 0 || nreq < 1 || (b > 0 && (!op || !src || !dst)) ||
      (nq > 0 && (!qids || !out_pos || !out_neg)))
    return ctx->fail(GAMMA_EINVAL, "%s: bad sizes or null arrays", fn);
  for (int j = 0; j < nq; j++)
    if (qids[j] < 0 || qids[j] >= (int)ctx->queries.size())
      return ctx->fail(GAMMA_EINVAL, "%s: unknown query id %d", fn, qids[j]);
  if (elab && !ctx->d_elab)
    return ctx->fail(GAMMA_EINVAL, "%s: edge labels need a graph loaded with gamma_load_graph_el", fn);
  if (nreq > 1 && ctx->d_elab)
    return ctx->fail(GAMMA_EINVAL, "%s: requests staged together need a graph without edge labels", fn);
  cudaSetDevice(ctx->device);
  cudaStream_t s = ctx->stream;
  ctx->b = b;
  ctx->nreq = nreq;
  ctx->qids.assign(qids, qids + nq);
  int rc = prepare_buffers(ctx, b);
  if (rc) return ctx->err.empty() ? ctx->cuda_fail(rc) : rc;
  if (nreq > 1) {
    std::vector<uint32_t> req(b);
    for (int r = 0; r < nreq; r++) {
      if (req_off[r] > req_off[r + 1] || req_off[r] < 0 || req_off[r + 1] > b)
        return ctx->fail(GAMMA_EINVAL, "%s: bad request offsets", fn);
      for (int64_t k = req_off[r]; k < req_off[r + 1]; k++) req[k] = (uint32_t)r;
    }
    if (req_off[0] != 0 || req_off[nreq] != b) return ctx->fail(GAMMA_EINVAL, "%s: request offsets must cover the batch", fn);
    CKC(cudaMemcpyAsync(ctx->d_req, req.data(), sizeof(uint32_t) * b, cudaMemcpyHostToDevice, s));
    CKC(cudaStreamSynchronize(s));
  }
  const int8_t *dop = op;
  const int32_t *dsrc = src, *ddst = dst, *delab = nullptr;
  if (b > 0) {
    bool dev = is_device_ptr(op) && is_device_ptr(src) && is_device_ptr(dst);
    if (!dev || (ctx->flags & GAMMA_F_GRAPH)) {  // the graph reads fixed staging buffers
      CKC(cudaMemcpyAsync(ctx->d_in_op, op, b, cudaMemcpyDefault, s));
      CKC(cudaMemcpyAsync(ctx->d_in_src, src, 4 * b, cudaMemcpyDefault, s));
      CKC(cudaMemcpyAsync(ctx->d_in_dst, dst, 4 * b, cudaMemcpyDefault, s));
      dop = ctx->d_in_op; dsrc = ctx->d_in_src; ddst = ctx->d_in_dst;
    }
    if (elab) {  // insertion labels, always through the context's buffer
      CKC(cudaMemcpyAsync(ctx->d_in_elab, elab, 4 * b, cudaMemcpyDefault, s));
      delab = ctx->d_in_elab;
    }
  }
  int32_t *rows;
  bool devrows;
  rc = rows_target(ctx, opt_out, &rows, &devrows);
  if (rc) return rc;
  rc = run_apply(ctx, dop, dsrc, ddst, delab, rows, opt_out ? (uint64_t)opt_out->capacity : 0,
                 opt_out ? opt_out->stride : 0);
  if (rc) return ctx->err.empty() ? ctx->fail(rc, "%s failed", fn) : rc;
  GmStatus st = *ctx->h_st;
  if (!ctx->staged) {
    if (st.err == GAMMA_EINVAL) {
      if (st.bad_index != INT64_MAX)
        return ctx->fail(GAMMA_EINVAL,
                         "%s: update %lld is invalid (bad op or id, self-loop, repeated edge, "
                         "insertion of an existing edge or deletion of a missing one); graph unchanged",
                         fn, (long long)st.bad_index);
      return ctx->fail(GAMMA_EINVAL, "%s: invalid batch; graph unchanged", fn);
    }
    return ctx->fail(st.err ? st.err : GAMMA_ECUDA, "%s: staging failed (code %d)", fn, st.err);
  }
  for (int r = 0; r < nreq; r++)
    for (int j = 0; j < nq; j++) {
      out_pos[(int64_t)r * nq + j] = ctx->h_cnt[((int64_t)r * nq + j) * 2];
      out_neg[(int64_t)r * nq + j] = ctx->h_cnt[((int64_t)r * nq + j) * 2 + 1];
    }
  ctx->stats.pool_used = (int64_t)ctx->pool_top;
  ctx->stats.pool_cap = ctx->pool_cap;
  if (st.err == GAMMA_ETIMEOUT)
    return ctx->fail(GAMMA_ETIMEOUT, "%s: work budget exceeded or a wait timed out; counts are incomplete", fn);
  if (st.err) return ctx->fail(st.err, "%s: matching failed (code %d)", fn, st.err);
  if (opt_out) {
    rc = copy_rows_out(ctx, opt_out, devrows);
    if (rc == GAMMA_EOVERFLOW)
      return ctx->fail(GAMMA_EOVERFLOW, "%s: %lld match rows do not fit in %lld", fn, (long long)opt_out->required,
                       (long long)opt_out->capacity);
    if (rc) return rc;
  }
  return GAMMA_OK;
}

}  // namespace

// ==========================================================================
// C-ABI
// ==========================================================================
extern "C" {

int gamma_create(const gamma_options *options, gamma_ctx **out) {
  if (!out) return GAMMA_EINVAL;
  *out = nullptr;
  gamma_options o;
  memset(&o, 0, sizeof(o));
  if (options) o = *options;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || o.device < 0 || o.device >= ndev) {
    cudaGetLastError();
    return GAMMA_ECUDA;
  }
  if (cudaSetDevice(o.device) != cudaSuccess) return GAMMA_ECUDA;
  gamma_ctx *ctx = new gamma_ctx();
  ctx->device = o.device;
  ctx->flags = o.flags;
  ctx->budget = o.work_budget;
  if (o.warps_per_block > 0) ctx->wpb = o.warps_per_block;
  if (o.frontier_tile > 0) ctx->tile = o.frontier_tile;
  if (o.steal_grain > 0) ctx->grain = o.steal_grain;
  if (o.idle_limit_us) ctx->idle_ns = 1000ull * o.idle_limit_us;
  if (o.handoff_limit_us) ctx->handoff_ns = 1000ull * o.handoff_limit_us;
  if (o.hub_min_degree > 0) ctx->hub_min = o.hub_min_degree;
  if (ctx->tile < 32 || ctx->tile > 4096 || ctx->wpb > 16) { delete ctx; return GAMMA_EINVAL; }
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, o.device);
  if (o.cuda_stream) {
    ctx->stream = (cudaStream_t)o.cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) { delete ctx; return GAMMA_ECUDA; }
    ctx->own_stream = true;
  }
  if (cudaMalloc((void **)&ctx->d_st, sizeof(GmStatus)) != cudaSuccess ||
      cudaMallocHost((void **)&ctx->h_st, sizeof(GmStatus)) != cudaSuccess ||
      cudaMallocHost((void **)&ctx->h_st_init, sizeof(GmStatus)) != cudaSuccess) {
    gamma_destroy(ctx);
    return GAMMA_ENOMEM;
  }
  for (auto &e : ctx->ev) cudaEventCreate(&e);
  *out = ctx;
  return GAMMA_OK;
}

void gamma_destroy(gamma_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  free_graph(ctx);
  StageBufs &sb = ctx->sb;
  void *ps[] = {sb.cu, sb.cv, sb.cop, sb.keys, sb.tk, sb.vals, sb.tv, sb.head, sb.gid, sb.gv, sb.gstart,
                sb.gins, sb.greloc, sb.bkeys, sb.cnext, sb.cinfo, sb.ulab, ctx->d_in_elab, ctx->d_in_op, ctx->d_in_src, ctx->d_in_dst, ctx->d_plans,
                ctx->d_pair_off, ctx->d_pair_plans, ctx->d_items, ctx->d_cnt, ctx->d_per_upd, ctx->d_rows,
                ctx->d_tasks, ctx->d_task_seq, ctx->d_sched, ctx->d_req, ctx->d_st};
  for (void *p : ps) if (p) cudaFree(p);
  if (ctx->h_st) cudaFreeHost(ctx->h_st);
  if (ctx->h_st_init) cudaFreeHost(ctx->h_st_init);
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  if (ctx->h_cnt) cudaFreeHost(ctx->h_cnt);
  for (auto &e : ctx->ev) if (e) cudaEventDestroy(e);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char *gamma_last_error(gamma_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

}  // extern "C"

int gm_ctx_device(gamma_ctx *ctx) { return ctx->device; }

// Arguments for re-running the DFS over the work items of the staged batch,
// from buffers the context already holds (nothing is allocated here).  The
// caller supplies the counts, task queue and scheduling scratch.
int gm_recount_prepare(gamma_ctx *ctx, MatchArgs *a, int *nslots, int *num_sms, cudaStream_t *stream) {
  if (!ctx) return GAMMA_EINVAL;
  ctx->err.clear();
  if (!ctx->staged) return ctx->fail(GAMMA_ESTATE, "no staged batch to recount");
  if (ctx->flags & GAMMA_F_PER_QUERY)
    return ctx->fail(GAMMA_ESTATE, "the recount needs the batched form (GAMMA_F_PER_QUERY keeps one query's items)");
  if (ctx->h_st->err) return ctx->fail(GAMMA_ESTATE, "the staged batch's matching failed (code %d)", ctx->h_st->err);
  if (ctx->h_st->nitems > (uint64_t)ctx->items_cap) return ctx->fail(GAMMA_ESTATE, "work items of the batch were not kept");
  const int nq = (int)ctx->qids.size();
  *nslots = std::max(nq, 1) * ctx->nreq;
  *num_sms = ctx->num_sms;
  *stream = ctx->stream;
  MatchArgs &m = *a;
  m.g = ctx->gd();
  m.cu = ctx->sb.cu; m.cv = ctx->sb.cv; m.op = ctx->sb.cop; m.b = ctx->b;
  m.ulab = ctx->d_elab ? ctx->sb.ulab : nullptr;
  m.seed_sorted = 0;  // the recount reuses the staged batch's work items; it seeds nothing
  m.qfilter = -1;
  m.plans = ctx->d_plans; m.nplans = ctx->nplans;
  m.pair_off = ctx->d_pair_off; m.pair_plans = ctx->d_pair_plans;
  m.grain = ctx->grain;
  m.items = ctx->d_items; m.item_cap = (uint64_t)ctx->items_cap;
  m.cnt = nullptr;
  m.req = (ctx->nreq > 1) ? ctx->d_req : nullptr;
  m.cnext = (ctx->nreq > 1) ? ctx->sb.cnext : nullptr;
  m.nq = std::max(nq, 1);
  m.per_upd = nullptr;
  m.use_filter = (ctx->flags & GAMMA_F_NO_FILTER) ? 0 : 1;
  m.rows = nullptr; m.row_cap = 0; m.row_stride = 0;
  m.budget = ctx->budget;
  m.tile = ctx->tile;
  m.nlev = std::max(1, ctx->maxq - 3);
  m.warps_per_block = ctx->wpb;
  m.count_bytes = 0;
  m.leaf = ((ctx->flags & GAMMA_F_NO_LEAF) || ctx->d_elab) ? 0 : 1;
  m.share = (ctx->flags & GAMMA_F_NO_SHARE) ? 0 : 1;
  m.bkeys = ctx->sb.keys; m.bvals = ctx->sb.vals; m.gstart = ctx->sb.gstart; m.gins = ctx->sb.gins;
  m.n2 = (uint32_t)(2 * ctx->b);
  m.tasks = nullptr; m.sched = nullptr; m.task_seq = nullptr; m.task_cap = 0;
  m.idle_limit_ns = ctx->idle_ns;
  m.handoff_limit_ns = ctx->handoff_ns;
  m.st = ctx->d_st;
  return GAMMA_OK;
}

int gm_ctx_fail(gamma_ctx *ctx, int code, const char *msg) { return ctx->fail(code, "%s", msg); }

// what a recount learned about its DFS launch, for gamma_get_stats
void gm_recount_done(gamma_ctx *ctx, uint64_t expansions, uint32_t donated) {
  ctx->stats.expansions = expansions;
  ctx->stats.donated_tasks = donated;
}

extern "C" {

int gamma_set_options(gamma_ctx *ctx, const gamma_options *o) {
  if (!ctx || !o) return GAMMA_EINVAL;
  if (o->frontier_tile && (o->frontier_tile < 32 || o->frontier_tile > 4096))
    return ctx->fail(GAMMA_EINVAL, "frontier_tile must be in [32, 4096]");
  if (o->warps_per_block < 0 || o->warps_per_block > 16) return ctx->fail(GAMMA_EINVAL, "warps_per_block must be in [1, 16]");
  ctx->flags = o->flags;
  ctx->budget = o->work_budget;
  if (o->warps_per_block) ctx->wpb = o->warps_per_block;
  if (o->frontier_tile) ctx->tile = o->frontier_tile;
  if (o->steal_grain) ctx->grain = o->steal_grain;
  if (o->idle_limit_us) ctx->idle_ns = 1000ull * o->idle_limit_us;
  if (o->handoff_limit_us) ctx->handoff_ns = 1000ull * o->handoff_limit_us;
  if (o->hub_min_degree < 0) return ctx->fail(GAMMA_EINVAL, "hub_min_degree must be >= 0");
  if (o->hub_min_degree > 0) ctx->hub_min = o->hub_min_degree;
  ctx->plan_key.clear();
  return GAMMA_OK;
}

int gamma_load_graph(gamma_ctx *ctx, int32_t n, const int32_t *labels, int64_t m, const int32_t *src,
                     const int32_t *dst) {
  return gamma_load_graph_el(ctx, n, labels, m, src, dst, nullptr);
}

int gamma_load_graph_el(gamma_ctx *ctx, int32_t n, const int32_t *labels, int64_t m, const int32_t *src,
                        const int32_t *dst, const int32_t *elabels) {
  if (!ctx) return GAMMA_EINVAL;
  ctx->err.clear();
  if (n <= 0 || m < 0 || !labels || (m > 0 && (!src || !dst)))
    return ctx->fail(GAMMA_EINVAL, "gamma_load_graph: bad sizes or null arrays");
  if (m > ((int64_t)1 << 31) - 1) return ctx->fail(GAMMA_EINVAL, "gamma_load_graph: too many edges");
  cudaSetDevice(ctx->device);
  free_graph(ctx);
  ctx->queries.clear();
  ctx->plan_key.clear();
  cudaStream_t s = ctx->stream;
  // device copies of the inputs
  const int32_t *dl = labels, *ds = src, *dd = dst, *de = elabels;
  int32_t *ts = nullptr, *td = nullptr, *te = nullptr;
  CKC(cudaMalloc((void **)&ctx->d_label, sizeof(int32_t) * n));
  CKC(cudaMemcpyAsync(ctx->d_label, labels, sizeof(int32_t) * n, cudaMemcpyDefault, s));
  dl = ctx->d_label;
  if (m > 0 && !is_device_ptr(src)) {
    CKC(cudaMalloc((void **)&ts, sizeof(int32_t) * m));
    CKC(cudaMemcpyAsync(ts, src, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
    ds = ts;
  }
  if (m > 0 && !is_device_ptr(dst)) {
    CKC(cudaMalloc((void **)&td, sizeof(int32_t) * m));
    CKC(cudaMemcpyAsync(td, dst, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
    dd = td;
  }
  if (elabels && !is_device_ptr(elabels)) {
    CKC(cudaMalloc((void **)&te, sizeof(int32_t) * std::max<int64_t>(m, 1)));
    if (m > 0) CKC(cudaMemcpyAsync(te, elabels, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
    de = te;
  }
  reset_status_host(ctx);
  CKC(cudaMemcpyAsync(ctx->d_st, ctx->h_st_init, sizeof(GmStatus), cudaMemcpyHostToDevice, s));
  CK(gm_load_validate(dl, n, ds, dd, de, m, ctx->d_st, s));
  CKC(cudaMemcpyAsync(ctx->h_st, ctx->d_st, sizeof(GmStatus), cudaMemcpyDeviceToHost, s));
  CKC(cudaStreamSynchronize(s));
  if (ctx->h_st->err) {
    cudaFree(ts); cudaFree(td); cudaFree(te);
    free_graph(ctx);
    if (ctx->h_st->bad_index != INT64_MAX)
      return ctx->fail(GAMMA_EINVAL, "gamma_load_graph: edge %lld has an id out of range, is a self-loop or has a "
                       "label outside [0, 255]", (long long)ctx->h_st->bad_index);
    return ctx->fail(GAMMA_EINVAL, "gamma_load_graph: negative vertex label");
  }
  if (ctx->h_st->max_label > 255) {
    cudaFree(ts); cudaFree(td); cudaFree(te);
    free_graph(ctx);
    return ctx->fail(GAMMA_EINVAL, "gamma_load_graph: vertex labels must be < 256");
  }
  ctx->n = n;
  ctx->nlab = (int)ctx->h_st->max_label + 1;
  ctx->n_cap = std::max(n, ctx->n_reserve);
  ctx->idb = bits_for(ctx->n_cap);
  int lb = bits_for(ctx->nlab);
  if (1 + ctx->idb + lb > 32) {
    cudaFree(ts); cudaFree(td); cudaFree(te);
    free_graph(ctx);
    return ctx->fail(GAMMA_EINVAL, "gamma_load_graph: %d vertex-id bits + %d label bits + 1 exceed 32", ctx->idb, lb);
  }
  ctx->nlfw = (ctx->nlab + 3) & ~3;
  CKC(cudaMalloc((void **)&ctx->d_adj, sizeof(uint2) * n));
  CKC(cudaMalloc((void **)&ctx->d_cap, sizeof(uint32_t) * n));
  CKC(cudaMalloc((void **)&ctx->d_nlf, (size_t)n * ctx->nlfw));
  CKC(cudaMalloc((void **)&ctx->d_vgroup, sizeof(int32_t) * n));
  CKC(cudaMemsetAsync(ctx->d_vgroup, 0xff, sizeof(int32_t) * n, s));
  CKC(cudaMemsetAsync(ctx->d_nlf, 0, (size_t)n * ctx->nlfw, s));
  uint32_t pool_cap = 0;
  GraphDev g = ctx->gd();
  CK(gm_load_build(g, ds, dd, de, m, &ctx->d_col, &ctx->d_etag, &ctx->d_elab, &pool_cap, 1.25, (uint64_t)1 << 20,
                   ctx->d_st, ctx->h_st, s));
  if (ctx->h_st->err) {  // a repeated edge whose copies carry different labels
    CKC(cudaStreamSynchronize(s));
    cudaFree(ts); cudaFree(td); cudaFree(te);
    free_graph(ctx);
    return ctx->fail(GAMMA_EINVAL, "gamma_load_graph: an edge is listed twice with different labels");
  }
  ctx->pool_cap = pool_cap;
  ctx->pool_top = ctx->h_st->pool_top;
  g = ctx->gd();
  CK(gm_nlf(g, nullptr, nullptr, (uint32_t)n, s));
  // live entries and label histogram
  std::vector<int32_t> hl(n);
  CKC(cudaMemcpyAsync(hl.data(), ctx->d_label, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
  std::vector<uint2> hadj;
  CKC(cudaStreamSynchronize(s));
  cudaFree(ts);
  cudaFree(td);
  cudaFree(te);
  ctx->label_freq.assign(ctx->nlab, 0);
  for (int32_t v = 0; v < n; v++) ctx->label_freq[hl[v]]++;
  // live directed entries = sum of list lengths
  {
    hadj.resize(n);
    CKC(cudaMemcpy(hadj.data(), ctx->d_adj, sizeof(uint2) * n, cudaMemcpyDeviceToHost));
    int64_t live = 0;
    for (auto &a : hadj) live += a.y;
    ctx->live = live;
  }
  // hub index for long lists (label-segment starts + hash sets of the keys)
  {
    std::vector<int32_t> hid(n, -1);
    uint64_t slots = 0;
    int32_t nh = 0;
    for (int32_t v = 0; v < n; v++) {
      if (hadj[v].y >= (uint32_t)ctx->hub_min) {
        hid[v] = nh++;
        uint64_t c = 8;
        while (c < 3ull * hadj[v].y + 8) c <<= 1;
        slots += c;
      }
    }
    ctx->nhub = nh;
    CKC(cudaMalloc((void **)&ctx->d_hub_id, sizeof(int32_t) * n));
    CKC(cudaMemcpy(ctx->d_hub_id, hid.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
    // hash-table descriptor per vertex (zero: none), so a membership test
    // reads it with one load instead of going through the hub number
    CKC(cudaMalloc((void **)&ctx->d_hub_tab, sizeof(uint2) * (size_t)n));
    CKC(cudaMemset(ctx->d_hub_tab, 0, sizeof(uint2) * (size_t)n));
    if (nh > 0) {
      CKC(cudaMalloc((void **)&ctx->d_hub_lofs, sizeof(uint32_t) * (size_t)nh * (ctx->nlab + 1)));
      // keys need their top bit free for the empty marker
      if (1 + ctx->idb + lb < 32) {
        uint64_t cap = 2 * slots + (1u << 20);
        if (cap > 0xF0000000ull) cap = 0xF0000000ull;
        CKC(cudaMalloc((void **)&ctx->d_hub_keys, sizeof(uint32_t) * cap));
        ctx->hub_keys_cap = (uint32_t)cap;
      }
      ctx->hub_top = 0;
      reset_status_host(ctx);
      CKC(cudaMemcpyAsync(ctx->d_st, ctx->h_st_init, sizeof(GmStatus), cudaMemcpyHostToDevice, s));
      CK(gm_hub(ctx->gd(), nullptr, nullptr, (uint32_t)n, ctx->d_st, s));
      CKC(cudaMemcpyAsync(ctx->h_st, ctx->d_st, sizeof(GmStatus), cudaMemcpyDeviceToHost, s));
      CKC(cudaStreamSynchronize(s));
      ctx->hub_top = ctx->h_st->hub_top;
    }
  }
  ctx->loaded = true;
  ctx->staged = false;
  return GAMMA_OK;
}

int gamma_register_query(gamma_ctx *ctx, int32_t q, const int32_t *qlabels, int32_t eq, const int32_t *qsrc,
                         const int32_t *qdst, int32_t *out_qid) {
  return gamma_register_query_el(ctx, q, qlabels, eq, qsrc, qdst, nullptr, out_qid);
}

int gamma_register_query_el(gamma_ctx *ctx, int32_t q, const int32_t *qlabels, int32_t eq, const int32_t *qsrc,
                            const int32_t *qdst, const int32_t *qelabels, int32_t *out_qid) {
  if (!ctx) return GAMMA_EINVAL;
  ctx->err.clear();
  if (!ctx->loaded) return ctx->fail(GAMMA_ESTATE, "gamma_register_query: no graph loaded");
  if (q < 2 || q > GM_MAXQ || eq < q - 1 || eq > q * (q - 1) / 2 || !qlabels || !qsrc || !qdst || !out_qid)
    return ctx->fail(GAMMA_EINVAL, "gamma_register_query: need 2 <= q <= %d and a connected simple edge list", GM_MAXQ);
  HostQuery Q;
  Q.q = q;
  Q.lab.assign(qlabels, qlabels + q);
  std::vector<std::vector<char>> adjq(q, std::vector<char>(q, 0));
  for (int e = 0; e < eq; e++) {
    int a = qsrc[e], b = qdst[e];
    if (a < 0 || a >= q || b < 0 || b >= q || a == b || adjq[a][b])
      return ctx->fail(GAMMA_EINVAL, "gamma_register_query: edge %d is out of range, a self-loop or repeated", e);
    adjq[a][b] = adjq[b][a] = 1;
    Q.edges.push_back({a, b});
    const int32_t el = qelabels ? qelabels[e] : 0;
    if (el < 0 || el > 255) return ctx->fail(GAMMA_EINVAL, "gamma_register_query: edge label outside [0, 255]");
    Q.elab.push_back(el);
    if (el != 0 && !ctx->d_elab) Q.never = true;  // every edge of an unlabelled graph has label 0
  }
  for (int u = 0; u < q; u++) {
    if (Q.lab[u] < 0) return ctx->fail(GAMMA_EINVAL, "gamma_register_query: negative label");
    if (Q.lab[u] >= ctx->nlab) Q.never = true;
  }
  // connectivity
  std::vector<int> stack = {0};
  std::vector<char> seen(q, 0);
  seen[0] = 1;
  while (!stack.empty()) {
    int u = stack.back();
    stack.pop_back();
    for (int w = 0; w < q; w++) if (adjq[u][w] && !seen[w]) { seen[w] = 1; stack.push_back(w); }
  }
  for (int u = 0; u < q; u++) if (!seen[u]) return ctx->fail(GAMMA_EINVAL, "gamma_register_query: query is not connected");
  int qid = (int)ctx->queries.size();
  if (!Q.never) {
    for (auto &e : Q.edges) {
      for (int o = 0; o < 2; o++) {
        Plan P;
        make_plan(Q, qid, o ? e.second : e.first, o ? e.first : e.second, ctx->label_freq, P);
        Q.plans.push_back(P);
      }
    }
  }
  ctx->queries.push_back(Q);
  *out_qid = qid;
  return GAMMA_OK;
}

int gamma_apply_batch(gamma_ctx *ctx, int64_t b, const int8_t *op, const int32_t *src, const int32_t *dst,
                      int32_t nq, const int32_t *qids, uint64_t *out_pos, uint64_t *out_neg,
                      gamma_matches *opt_out) {
  const int64_t off[2] = {0, b};
  return apply_impl(ctx, "gamma_apply_batch", 1, off, b, op, src, dst, nullptr, nq, qids, out_pos, out_neg, opt_out);
}

int gamma_apply_batch_el(gamma_ctx *ctx, int64_t b, const int8_t *op, const int32_t *src, const int32_t *dst,
                         const int32_t *elab, int32_t nq, const int32_t *qids, uint64_t *out_pos, uint64_t *out_neg,
                         gamma_matches *opt_out) {
  const int64_t off[2] = {0, b};
  return apply_impl(ctx, "gamma_apply_batch_el", 1, off, b, op, src, dst, elab, nq, qids, out_pos, out_neg, opt_out);
}

int gamma_apply_batches(gamma_ctx *ctx, int32_t nreq, const int64_t *req_off, const int8_t *op,
                        const int32_t *src, const int32_t *dst, int32_t nq, const int32_t *qids,
                        uint64_t *out_pos, uint64_t *out_neg) {
  if (!ctx) return GAMMA_EINVAL;
  if (nreq < 1 || !req_off) return ctx->fail(GAMMA_EINVAL, "gamma_apply_batches: need nreq >= 1 and offsets");
  return apply_impl(ctx, "gamma_apply_batches", nreq, req_off, req_off[nreq], op, src, dst, nullptr, nq, qids,
                    out_pos, out_neg, nullptr);
}

int gamma_fetch_matches(gamma_ctx *ctx, gamma_matches *out) {
  if (!ctx) return GAMMA_EINVAL;
  ctx->err.clear();
  if (!ctx->staged) return ctx->fail(GAMMA_ESTATE, "gamma_fetch_matches: no staged batch");
  if (!out) return ctx->fail(GAMMA_EINVAL, "gamma_fetch_matches: null output");
  cudaSetDevice(ctx->device);
  int rc = match_with_rows(ctx, out);
  if (rc != GAMMA_OK && rc != GAMMA_EOVERFLOW) return rc;
  if (ctx->h_st->err) return ctx->fail(ctx->h_st->err, "gamma_fetch_matches: matching failed (code %d)", ctx->h_st->err);
  if (rc == GAMMA_EOVERFLOW)
    return ctx->fail(GAMMA_EOVERFLOW, "gamma_fetch_matches: %lld rows do not fit in %lld",
                     (long long)out->required, (long long)out->capacity);
  return GAMMA_OK;
}

int gamma_autotune(gamma_ctx *ctx, int32_t npoints, gamma_tune_point *points, int32_t repeats,
                   gamma_tune_point *best) {
  if (!ctx) return GAMMA_EINVAL;
  ctx->err.clear();
  if (!ctx->staged) return ctx->fail(GAMMA_ESTATE, "gamma_autotune: no staged batch");
  if (npoints < 1 || !points || !best || repeats < 1) return ctx->fail(GAMMA_EINVAL, "gamma_autotune: bad arguments");
  cudaSetDevice(ctx->device);
  const int wpb0 = ctx->wpb, tile0 = ctx->tile, grain0 = ctx->grain;
  int bi = -1;
  for (int i = 0; i < npoints; i++) {
    gamma_tune_point &pt = points[i];
    pt.ms = -1.f;
    if (pt.warps_per_block < 1 || pt.warps_per_block > 16 || pt.frontier_tile < 32 || pt.frontier_tile > 4096 ||
        pt.steal_grain < 1)
      continue;
    ctx->wpb = pt.warps_per_block;
    ctx->tile = pt.frontier_tile;
    ctx->grain = pt.steal_grain;
    std::vector<float> t;
    bool ok = true;
    for (int r = 0; r < repeats && ok; r++) {
      int rc = run_match(ctx, nullptr, 0, 0);
      if (rc || ctx->h_st->err) { ok = false; cudaGetLastError(); break; }
      t.push_back((float)(ctx->stats.ms_seed + ctx->stats.ms_match));
    }
    if (!ok) continue;
    std::sort(t.begin(), t.end());
    pt.ms = t[t.size() / 2];
    if (bi < 0 || pt.ms < points[bi].ms) bi = i;
  }
  if (bi < 0) {
    ctx->wpb = wpb0; ctx->tile = tile0; ctx->grain = grain0;
    return ctx->fail(GAMMA_EINVAL, "gamma_autotune: no point could run");
  }
  ctx->wpb = points[bi].warps_per_block;
  ctx->tile = points[bi].frontier_tile;
  ctx->grain = points[bi].steal_grain;
  *best = points[bi];
  return GAMMA_OK;
}

int gamma_update_counts(gamma_ctx *ctx, int32_t j, uint64_t *out) {
  if (!ctx) return GAMMA_EINVAL;
  ctx->err.clear();
  if (!ctx->staged) return ctx->fail(GAMMA_ESTATE, "gamma_update_counts: no staged batch");
  if (!(ctx->flags & GAMMA_F_PER_UPDATE)) return ctx->fail(GAMMA_ESTATE, "gamma_update_counts: GAMMA_F_PER_UPDATE not set");
  if (j < 0 || j >= (int)ctx->qids.size() || !out) return ctx->fail(GAMMA_EINVAL, "gamma_update_counts: bad query slot");
  if (ctx->b == 0) return GAMMA_OK;
  cudaSetDevice(ctx->device);
  CKC(cudaMemcpy(out, ctx->d_per_upd + (size_t)j * ctx->b, sizeof(uint64_t) * ctx->b, cudaMemcpyDeviceToHost));
  return GAMMA_OK;
}

int gamma_commit(gamma_ctx *ctx) {
  if (!ctx) return GAMMA_EINVAL;
  ctx->err.clear();
  if (!ctx->staged) return ctx->fail(GAMMA_ESTATE, "gamma_commit: no staged batch");
  cudaSetDevice(ctx->device);
  cudaStream_t s = ctx->stream;
  CKC(cudaMemsetAsync(&ctx->d_st->live, 0, sizeof(uint64_t), s));
  CKC(cudaEventRecord(ctx->ev[6], s));
  if (ctx->b > 0) CK(gm_commit(ctx->gd(), ctx->sb, ctx->b, ctx->nreq > 1, ctx->d_st, s));
  CKC(cudaEventRecord(ctx->ev[7], s));
  CKC(cudaMemcpyAsync(ctx->h_st, ctx->d_st, sizeof(GmStatus), cudaMemcpyDeviceToHost, s));
  CKC(cudaStreamSynchronize(s));
  ctx->live += (int64_t)ctx->h_st->live;  // signed change, two's complement
  ctx->hub_top = ctx->h_st->hub_top;
  ctx->stats.ms_commit = ev_ms(ctx->ev[6], ctx->ev[7]);
  ctx->staged = false;
  return GAMMA_OK;
}

int gamma_export_adjacency(gamma_ctx *ctx, int64_t *off, int32_t *nbr, int32_t *tag, int64_t cap) {
  if (!ctx) return GAMMA_EINVAL;
  ctx->err.clear();
  if (!ctx->loaded) return ctx->fail(GAMMA_ESTATE, "gamma_export_adjacency: no graph loaded");
  if (!off || (cap > 0 && (!nbr || !tag))) return ctx->fail(GAMMA_EINVAL, "gamma_export_adjacency: null arrays");
  cudaSetDevice(ctx->device);
  CKC(cudaStreamSynchronize(ctx->stream));
  std::vector<uint2> adj(ctx->n);
  std::vector<uint32_t> col(ctx->pool_top), etag(ctx->pool_top);
  CKC(cudaMemcpy(adj.data(), ctx->d_adj, sizeof(uint2) * ctx->n, cudaMemcpyDeviceToHost));
  if (ctx->pool_top) {
    CKC(cudaMemcpy(col.data(), ctx->d_col, sizeof(uint32_t) * ctx->pool_top, cudaMemcpyDeviceToHost));
    CKC(cudaMemcpy(etag.data(), ctx->d_etag, sizeof(uint32_t) * ctx->pool_top, cudaMemcpyDeviceToHost));
  }
  const uint32_t idmask = ctx->gd().idmask;
  int64_t k = 0;
  off[0] = 0;
  for (int32_t v = 0; v < ctx->n; v++) {
    for (uint32_t i = 0; i < adj[v].y; i++, k++) {
      if (k < cap) {
        uint32_t x = col[adj[v].x + i];
        nbr[k] = (int32_t)((x >> 1) & idmask);
        tag[k] = (x & 1u) ? (int32_t)etag[adj[v].x + i] : -1;
      }
    }
    off[v + 1] = k;
  }
  return k > cap ? ctx->fail(GAMMA_EOVERFLOW, "gamma_export_adjacency: %lld entries > cap", (long long)k) : GAMMA_OK;
}

// checkpoint layout (little-endian int32 words unless noted):
//   "GMCK" (4 bytes), version 1, n, n_cap, m (int64), labels[n], src[m], dst[m],
//   nq, then per query: q, eq, labels[q], src[eq], dst[eq]
namespace {
struct CkWriter {
  uint8_t *buf;
  int64_t cap, pos = 0;
  void bytes(const void *p, int64_t n) {
    if (buf && pos + n <= cap) memcpy(buf + pos, p, (size_t)n);
    pos += n;
  }
  void i32(int32_t v) { bytes(&v, 4); }
  void i64(int64_t v) { bytes(&v, 8); }
};
struct CkReader {
  const uint8_t *buf;
  int64_t size, pos = 0;
  bool ok = true;
  void bytes(void *p, int64_t n) {
    if (n < 0 || pos + n > size) { ok = false; return; }
    memcpy(p, buf + pos, (size_t)n);
    pos += n;
  }
  int32_t i32() { int32_t v = 0; bytes(&v, 4); return v; }
  int64_t i64() { int64_t v = 0; bytes(&v, 8); return v; }
};
}  // namespace

int gamma_plan_order(int32_t q, const int32_t *qlabels, int32_t eq, const int32_t *qsrc, const int32_t *qdst,
                     int32_t a, int32_t b, int32_t nlab, const int64_t *label_freq, int32_t *out_order,
                     uint16_t *out_bwd) {
  if (q < 2 || q > GM_MAXQ || eq < 1 || !qlabels || !qsrc || !qdst || !out_order || a < 0 || a >= q || b < 0 ||
      b >= q || a == b || nlab < 0 || (nlab > 0 && !label_freq))
    return GAMMA_EINVAL;
  HostQuery Q;
  Q.q = q;
  Q.lab.assign(qlabels, qlabels + q);
  std::vector<std::vector<char>> adjq(q, std::vector<char>(q, 0));
  for (int32_t e = 0; e < eq; e++) {
    const int32_t u = qsrc[e], w = qdst[e];
    if (u < 0 || u >= q || w < 0 || w >= q || u == w || adjq[u][w]) return GAMMA_EINVAL;
    adjq[u][w] = adjq[w][u] = 1;
    Q.edges.push_back({u, w});
  }
  if (!adjq[a][b]) return GAMMA_EINVAL;
  // connected (as gamma_register_query requires), so every step of the order has a choice
  std::vector<char> seen(q, 0);
  std::vector<int> stack = {0};
  seen[0] = 1;
  while (!stack.empty()) {
    const int u = stack.back();
    stack.pop_back();
    for (int w = 0; w < q; w++) if (adjq[u][w] && !seen[w]) { seen[w] = 1; stack.push_back(w); }
  }
  for (int u = 0; u < q; u++) if (!seen[u]) return GAMMA_EINVAL;
  std::vector<int64_t> freq(label_freq, label_freq + nlab);
  Plan P;
  make_plan(Q, 0, a, b, freq, P);
  for (int32_t l = 0; l < q; l++) {
    out_order[l] = P.qv[l];
    if (out_bwd) out_bwd[l] = P.bwd[l];
  }
  return GAMMA_OK;
}

int gamma_checkpoint(gamma_ctx *ctx, void *buf, int64_t cap, int64_t *size) {
  if (!ctx) return GAMMA_EINVAL;
  ctx->err.clear();
  if (!ctx->loaded) return ctx->fail(GAMMA_ESTATE, "gamma_checkpoint: no graph loaded");
  if (ctx->staged) return ctx->fail(GAMMA_ESTATE, "gamma_checkpoint: a batch is staged; commit it first");
  if (ctx->d_elab) return ctx->fail(GAMMA_EINVAL, "gamma_checkpoint: edge labels are not checkpointed");
  if (!size || (cap > 0 && !buf)) return ctx->fail(GAMMA_EINVAL, "gamma_checkpoint: null output");
  cudaSetDevice(ctx->device);
  CKC(cudaStreamSynchronize(ctx->stream));
  const int32_t n = ctx->n;
  std::vector<int32_t> lab(n);
  std::vector<uint2> adj(n);
  std::vector<uint32_t> col(ctx->pool_top);
  CKC(cudaMemcpy(lab.data(), ctx->d_label, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
  CKC(cudaMemcpy(adj.data(), ctx->d_adj, sizeof(uint2) * n, cudaMemcpyDeviceToHost));
  if (ctx->pool_top) CKC(cudaMemcpy(col.data(), ctx->d_col, sizeof(uint32_t) * ctx->pool_top, cudaMemcpyDeviceToHost));
  const uint32_t idmask = ctx->gd().idmask;
  std::vector<int32_t> es, ed;  // each undirected edge once, from its smaller end
  for (int32_t v = 0; v < n; v++)
    for (uint32_t i = 0; i < adj[v].y; i++) {
      const int32_t u = (int32_t)((col[adj[v].x + i] >> 1) & idmask);
      if (v < u) { es.push_back(v); ed.push_back(u); }
    }
  CkWriter w{reinterpret_cast<uint8_t *>(buf), cap};
  w.bytes("GMCK", 4);
  w.i32(1);
  w.i32(n);
  w.i32(ctx->n_cap);
  w.i64((int64_t)es.size());
  w.bytes(lab.data(), 4 * (int64_t)n);
  w.bytes(es.data(), 4 * (int64_t)es.size());
  w.bytes(ed.data(), 4 * (int64_t)ed.size());
  w.i32((int32_t)ctx->queries.size());
  for (const HostQuery &Q : ctx->queries) {
    w.i32(Q.q);
    w.i32((int32_t)Q.edges.size());
    w.bytes(Q.lab.data(), 4 * (int64_t)Q.q);
    for (auto &e : Q.edges) w.i32(e.first);
    for (auto &e : Q.edges) w.i32(e.second);
  }
  *size = w.pos;
  return w.pos > cap ? ctx->fail(GAMMA_EOVERFLOW, "gamma_checkpoint: %lld bytes > cap", (long long)w.pos) : GAMMA_OK;
}

int gamma_restore(gamma_ctx *ctx, const void *buf, int64_t size) {
  if (!ctx) return GAMMA_EINVAL;
  ctx->err.clear();
  if (!buf || size < 24) return ctx->fail(GAMMA_EINVAL, "gamma_restore: no checkpoint");
  CkReader r{reinterpret_cast<const uint8_t *>(buf), size};
  char magic[4];
  r.bytes(magic, 4);
  if (memcmp(magic, "GMCK", 4) != 0 || r.i32() != 1) return ctx->fail(GAMMA_EINVAL, "gamma_restore: not a checkpoint");
  const int32_t n = r.i32(), n_cap = r.i32();
  const int64_t m = r.i64();
  if (!r.ok || n <= 0 || n_cap < 0 || m < 0 || m > size) return ctx->fail(GAMMA_EINVAL, "gamma_restore: bad header");
  std::vector<int32_t> lab(n), es(m), ed(m);
  r.bytes(lab.data(), 4 * (int64_t)n);
  r.bytes(es.data(), 4 * m);
  r.bytes(ed.data(), 4 * m);
  const int32_t nq = r.i32();
  if (!r.ok || nq < 0) return ctx->fail(GAMMA_EINVAL, "gamma_restore: truncated checkpoint");
  std::vector<std::vector<int32_t>> ql(nq), qs(nq), qd(nq);
  for (int32_t j = 0; j < nq; j++) {
    const int32_t q = r.i32(), eq = r.i32();
    if (!r.ok || q < 2 || q > GM_MAXQ || eq < 0 || eq > q * (q - 1) / 2)
      return ctx->fail(GAMMA_EINVAL, "gamma_restore: bad query %d", j);
    ql[j].resize(q); qs[j].resize(eq); qd[j].resize(eq);
    r.bytes(ql[j].data(), 4 * (int64_t)q);
    r.bytes(qs[j].data(), 4 * (int64_t)eq);
    r.bytes(qd[j].data(), 4 * (int64_t)eq);
  }
  if (!r.ok) return ctx->fail(GAMMA_EINVAL, "gamma_restore: truncated checkpoint");
  // the graph and queries go through the ordinary validated calls; queries
  // are registered in their original order, so they get their original ids
  const int32_t keep_reserve = ctx->n_reserve;
  ctx->n_reserve = n_cap;
  int rc = gamma_load_graph(ctx, n, lab.data(), m, es.data(), ed.data());
  ctx->n_reserve = keep_reserve;
  if (rc != GAMMA_OK) return rc;
  for (int32_t j = 0; j < nq; j++) {
    int32_t qid = -1;
    rc = gamma_register_query(ctx, (int32_t)ql[j].size(), ql[j].data(), (int32_t)qs[j].size(), qs[j].data(),
                              qd[j].data(), &qid);
    if (rc != GAMMA_OK) return rc;
    if (qid != j) return ctx->fail(GAMMA_ESTATE, "gamma_restore: query %d came back as %d", j, qid);
  }
  return GAMMA_OK;
}

int gamma_reserve_vertices(gamma_ctx *ctx, int32_t n_max) {
  if (!ctx) return GAMMA_EINVAL;
  ctx->err.clear();
  if (n_max < 0) return ctx->fail(GAMMA_EINVAL, "gamma_reserve_vertices: negative size");
  ctx->n_reserve = n_max;
  return GAMMA_OK;
}

int gamma_add_vertices(gamma_ctx *ctx, int32_t k, const int32_t *labels, int32_t *out_first) {
  if (!ctx) return GAMMA_EINVAL;
  ctx->err.clear();
  if (!ctx->loaded) return ctx->fail(GAMMA_ESTATE, "gamma_add_vertices: no graph loaded");
  if (ctx->staged) return ctx->fail(GAMMA_ESTATE, "gamma_add_vertices: a batch is staged; commit it first");
  if (k < 0 || (k > 0 && !labels)) return ctx->fail(GAMMA_EINVAL, "gamma_add_vertices: bad size or null labels");
  if (out_first) *out_first = ctx->n;
  if (k == 0) return GAMMA_OK;
  const int64_t n2 = (int64_t)ctx->n + k;
  if (n2 > ctx->n_cap)
    return ctx->fail(GAMMA_EINVAL, "gamma_add_vertices: %lld vertices exceed the %d reserved "
                     "(call gamma_reserve_vertices before gamma_load_graph)", (long long)n2, ctx->n_cap);
  cudaSetDevice(ctx->device);
  std::vector<int32_t> hl(k);
  CKC(cudaMemcpy(hl.data(), labels, sizeof(int32_t) * k, cudaMemcpyDefault));
  for (int32_t i = 0; i < k; i++)
    if (hl[i] < 0 || hl[i] >= ctx->nlab)
      return ctx->fail(GAMMA_EINVAL, "gamma_add_vertices: label %d of new vertex %d is outside the graph's "
                       "labels [0, %d)", hl[i], i, ctx->nlab);
  const int32_t n = ctx->n, m2 = (int32_t)n2;
  drop_graph_exec(ctx);
  CKC(cudaStreamSynchronize(ctx->stream));
  // new vertices: no entries and no slot (their first insertion moves them to
  // the pool), zero label counts, not hubs, in no staged group
  CK(grow_vertex_array(ctx, &ctx->d_label, sizeof(int32_t), n, m2, 0));
  CKC(cudaMemcpy(ctx->d_label + n, hl.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice));
  CK(grow_vertex_array(ctx, &ctx->d_adj, sizeof(uint2), n, m2, 0));
  CK(grow_vertex_array(ctx, &ctx->d_cap, sizeof(uint32_t), n, m2, 0));
  CK(grow_vertex_array(ctx, &ctx->d_nlf, (size_t)ctx->nlfw, n, m2, 0));
  CK(grow_vertex_array(ctx, &ctx->d_vgroup, sizeof(int32_t), n, m2, 0xff));
  CK(grow_vertex_array(ctx, &ctx->d_hub_id, sizeof(int32_t), n, m2, 0xff));
  CK(grow_vertex_array(ctx, &ctx->d_hub_tab, sizeof(uint2), n, m2, 0));
  for (int32_t i = 0; i < k; i++) ctx->label_freq[hl[i]]++;
  ctx->n = m2;
  return GAMMA_OK;
}

int gamma_vertex_neighbors(gamma_ctx *ctx, int32_t v, int32_t *out, int64_t cap, int64_t *count) {
  if (!ctx) return GAMMA_EINVAL;
  ctx->err.clear();
  if (!ctx->loaded) return ctx->fail(GAMMA_ESTATE, "gamma_vertex_neighbors: no graph loaded");
  if (ctx->staged) return ctx->fail(GAMMA_ESTATE, "gamma_vertex_neighbors: a batch is staged; commit it first");
  if (v < 0 || v >= ctx->n || !count || (cap > 0 && !out))
    return ctx->fail(GAMMA_EINVAL, "gamma_vertex_neighbors: vertex out of range or null output");
  cudaSetDevice(ctx->device);
  CKC(cudaStreamSynchronize(ctx->stream));
  uint2 a;
  CKC(cudaMemcpy(&a, ctx->d_adj + v, sizeof(uint2), cudaMemcpyDeviceToHost));
  *count = a.y;
  if (a.y == 0) return GAMMA_OK;
  std::vector<uint32_t> keys(a.y);
  CKC(cudaMemcpy(keys.data(), ctx->d_col + a.x, sizeof(uint32_t) * a.y, cudaMemcpyDeviceToHost));
  const uint32_t idmask = ctx->gd().idmask;
  for (int64_t i = 0; i < (int64_t)a.y && i < cap; i++) out[i] = (int32_t)((keys[i] >> 1) & idmask);
  return (int64_t)a.y > cap ? ctx->fail(GAMMA_EOVERFLOW, "gamma_vertex_neighbors: %u neighbours > cap", a.y)
                            : GAMMA_OK;
}

int gamma_get_stats(gamma_ctx *ctx, gamma_stats *out) {
  if (!ctx || !out) return GAMMA_EINVAL;
  *out = ctx->stats;
  out->pool_used = (int64_t)ctx->pool_top;
  out->pool_cap = ctx->pool_cap;
  out->live_edges = ctx->live;
  out->kernel_launches = __atomic_load_n(&gm_launch_count, __ATOMIC_RELAXED);
  out->graph_captures = ctx->graph_captures;
  return GAMMA_OK;
}

}  // extern "C"
