// gm_server.cu -- the served form: a host worker thread that keeps the graph
// on the device and applies a stream of update requests in arrival order.
//
// Continuous batching: requests that arrive while a group is on the GPU wait
// in a FIFO; when the GPU is free, the worker takes every waiting request it
// can admit -- in order, until the group would exceed the update / request
// caps or its estimated device memory would exceed a fraction of the free
// HBM -- and stages them together with gamma_apply_batches, so their seeding
// and DFS run in the same launches while each request still gets exactly the
// result it would get on its own (request r sees the graph after requests
// 0..r-1; requests may touch the same edges).  The group is then committed.
// A request is copied into pinned host memory by the submitting thread, which
// overlaps with the GPU work of the current group.
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gm_common.cuh"

namespace {

struct Request {
  int64_t ticket = 0;
  int64_t b = 0;
  int8_t *op = nullptr;  // pinned
  int32_t *src = nullptr, *dst = nullptr;
  double arrival_ms = 0, start_ms = 0, done_ms = 0;
  int32_t group = 0;
  int status = GAMMA_OK;
  bool done = false;
  std::vector<uint64_t> pos, neg;
};

double now_ms(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

void free_request(Request *r) {
  if (r->op) cudaFreeHost(r->op);
  if (r->src) cudaFreeHost(r->src);
  if (r->dst) cudaFreeHost(r->dst);
  r->op = nullptr; r->src = nullptr; r->dst = nullptr;
}

}  // namespace

struct gamma_server {
  gamma_ctx *ctx = nullptr;
  std::vector<int32_t> qids;
  gamma_server_options opt{};
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request *> pending;
  std::unordered_map<int64_t, Request *> all;
  int64_t next_ticket = 0;
  bool stopping = false;
  std::thread worker;
  // group staging (pinned, grown on demand)
  int8_t *g_op = nullptr;
  int32_t *g_src = nullptr, *g_dst = nullptr;
  int64_t g_cap = 0;
  gamma_server_stats stats{};

  int ensure_group(int64_t n) {
    if (n <= g_cap) return GAMMA_OK;
    if (g_op) cudaFreeHost(g_op);
    if (g_src) cudaFreeHost(g_src);
    if (g_dst) cudaFreeHost(g_dst);
    g_op = nullptr; g_src = nullptr; g_dst = nullptr;
    int64_t c = n + n / 2 + 1024;
    if (cudaMallocHost((void **)&g_op, c) != cudaSuccess || cudaMallocHost((void **)&g_src, 4 * c) != cudaSuccess ||
        cudaMallocHost((void **)&g_dst, 4 * c) != cudaSuccess) {
      g_cap = 0;
      return GAMMA_ENOMEM;
    }
    g_cap = c;
    return GAMMA_OK;
  }

  // device bytes a group of n updates may need beyond the resident graph:
  // the staging buffers (inputs 9 B, canonical endpoints and op 9 B, sort keys
  // and values with their alternates 48 B, vertex groups 32 B, sorted batch
  // keys 8 B, request and chain links 9 B per update), the DFS work items
  // (up to 8 per update at 16 B) and the adjacency pool's growth when touched
  // lists outgrow their slack (a moved list takes 1.25x its entries; about 2
  // entries of 4 B per update on average, counted at 4x for skewed lists),
  // plus the fixed task ring, counts and status (64 MiB)
  static uint64_t est_bytes(int64_t n) {
    const uint64_t per_update = 9 + 9 + 48 + 32 + 8 + 9 + 8 * 16 + 4 * 2 * 4;
    return (uint64_t)n * per_update + (64ull << 20);
  }

  void run() {
    cudaSetDevice(ctx_device());
    std::vector<Request *> group;
    for (;;) {
      group.clear();
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return stopping || !pending.empty(); });
        if (pending.empty() && stopping) return;
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        const double budget = opt.hbm_fraction * (double)free_b;
        int64_t nupd = 0;
        while (!pending.empty()) {
          Request *r = pending.front();
          if (!group.empty()) {
            if ((int)group.size() >= opt.max_requests || nupd + r->b > opt.max_updates) break;
            if ((double)est_bytes(nupd + r->b) > budget) break;
          }
          nupd += r->b;
          group.push_back(r);
          pending.pop_front();
        }
      }
      run_group(group);
    }
  }

  int ctx_device();

  // stage requests [i0, i1) of the group together and commit them; returns
  // the status, counts in pos/neg at the requests' positions
  int apply_range(std::vector<Request *> &group, size_t i0, size_t i1, std::vector<uint64_t> &pos,
                  std::vector<uint64_t> &neg) {
    int64_t n = 0;
    for (size_t i = i0; i < i1; i++) n += group[i]->b;
    int rc = ensure_group(n);
    if (rc != GAMMA_OK) return rc;
    const int nq = (int)qids.size();
    std::vector<int64_t> off(i1 - i0 + 1, 0);
    for (size_t i = i0; i < i1; i++) {
      Request *r = group[i];
      const int64_t o = off[i - i0];
      memcpy(g_op + o, r->op, r->b);
      memcpy(g_src + o, r->src, 4 * r->b);
      memcpy(g_dst + o, r->dst, 4 * r->b);
      off[i - i0 + 1] = o + r->b;
    }
    rc = gamma_apply_batches(ctx, (int32_t)(i1 - i0), off.data(), g_op, g_src, g_dst, nq, qids.data(),
                             pos.data() + i0 * nq, neg.data() + i0 * nq);
    if (rc == GAMMA_OK || rc == GAMMA_ETIMEOUT) {
      int rc2 = gamma_commit(ctx);
      if (rc == GAMMA_OK) rc = rc2;
    }
    return rc;
  }

  void run_group(std::vector<Request *> &group) {
    const double start = now_ms(t0);
    int64_t n = 0;
    for (Request *r : group) n += r->b;
    const int nq = (int)qids.size();
    std::vector<uint64_t> pos(group.size() * std::max(nq, 1)), neg(pos.size());
    std::vector<int> status(group.size(), GAMMA_OK);
    int rc = apply_range(group, 0, group.size(), pos, neg);
    if (rc == GAMMA_EINVAL && group.size() > 1) {
      // some request is invalid (the whole group was rejected, the graph is
      // unchanged): serve the requests one by one, in order, so that only the
      // invalid ones fail and every other request meets the graph left by
      // the valid requests before it, as one-at-a-time serving would give
      for (size_t i = 0; i < group.size(); i++) status[i] = apply_range(group, i, i + 1, pos, neg);
    } else {
      for (auto &x : status) x = rc;
    }
    const double done = now_ms(t0);
    std::lock_guard<std::mutex> lk(mu);
    for (size_t i = 0; i < group.size(); i++) {
      Request *r = group[i];
      r->start_ms = start;
      r->done_ms = done;
      r->group = (int32_t)group.size();
      r->status = status[i];
      r->pos.assign(pos.begin() + i * nq, pos.begin() + (i + 1) * nq);
      r->neg.assign(neg.begin() + i * nq, neg.begin() + (i + 1) * nq);
      r->done = true;
      free_request(r);
    }
    stats.groups++;
    stats.requests += (int64_t)group.size();
    stats.updates += n;
    stats.busy_ms += done - start;
    if ((int64_t)group.size() > stats.max_group) stats.max_group = (int64_t)group.size();
    cv_done.notify_all();
  }
};

// the context's device (gm_api.cu owns the context layout)
int gm_ctx_device(gamma_ctx *ctx);
int gamma_server::ctx_device() { return gm_ctx_device(ctx); }

extern "C" {

int gamma_server_start(gamma_ctx *ctx, int32_t nq, const int32_t *qids, const gamma_server_options *options,
                       gamma_server **out) {
  if (!ctx || !out || nq < 0 || (nq > 0 && !qids)) return GAMMA_EINVAL;
  gamma_server *s = new gamma_server();
  s->ctx = ctx;
  s->qids.assign(qids, qids + nq);
  if (options) s->opt = *options;
  if (s->opt.max_updates <= 0) s->opt.max_updates = 1 << 21;
  if (s->opt.max_requests <= 0) s->opt.max_requests = 256;
  if (s->opt.hbm_fraction <= 0) s->opt.hbm_fraction = 0.5;
  s->t0 = std::chrono::steady_clock::now();
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return GAMMA_OK;
}

int gamma_server_submit(gamma_server *s, int64_t b, const int8_t *op, const int32_t *src, const int32_t *dst,
                        int64_t *ticket) {
  if (!s || b < 0 || (b > 0 && (!op || !src || !dst)) || !ticket) return GAMMA_EINVAL;
  Request *r = new Request();
  r->b = b;
  const int64_t c = b > 0 ? b : 1;
  if (cudaMallocHost((void **)&r->op, c) != cudaSuccess || cudaMallocHost((void **)&r->src, 4 * c) != cudaSuccess ||
      cudaMallocHost((void **)&r->dst, 4 * c) != cudaSuccess) {
    free_request(r);
    delete r;
    return GAMMA_ENOMEM;
  }
  if (b > 0) {
    memcpy(r->op, op, b);
    memcpy(r->src, src, 4 * b);
    memcpy(r->dst, dst, 4 * b);
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stopping) {
    free_request(r);
    delete r;
    return GAMMA_ESTATE;
  }
  r->ticket = s->next_ticket++;
  r->arrival_ms = now_ms(s->t0);
  s->all[r->ticket] = r;
  s->pending.push_back(r);
  *ticket = r->ticket;
  s->cv_work.notify_one();
  return GAMMA_OK;
}

int gamma_server_wait(gamma_server *s, int64_t ticket, uint64_t *out_pos, uint64_t *out_neg,
                      gamma_request_info *info) {
  if (!s) return GAMMA_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return GAMMA_EINVAL;
  Request *r = it->second;
  s->cv_done.wait(lk, [&] { return r->done; });
  const int nq = (int)s->qids.size();
  for (int j = 0; j < nq; j++) {
    if (out_pos) out_pos[j] = r->pos[j];
    if (out_neg) out_neg[j] = r->neg[j];
  }
  if (info) {
    info->arrival_ms = r->arrival_ms;
    info->start_ms = r->start_ms;
    info->done_ms = r->done_ms;
    info->group_size = r->group;
    info->status = r->status;
  }
  int rc = r->status;
  s->all.erase(it);
  delete r;
  return rc;
}

int gamma_server_stats_get(gamma_server *s, gamma_server_stats *out) {
  if (!s || !out) return GAMMA_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  return GAMMA_OK;
}

int gamma_server_stop(gamma_server *s) {
  if (!s) return GAMMA_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (auto &kv : s->all) {
    free_request(kv.second);
    delete kv.second;
  }
  if (s->g_op) cudaFreeHost(s->g_op);
  if (s->g_src) cudaFreeHost(s->g_src);
  if (s->g_dst) cudaFreeHost(s->g_dst);
  delete s;
  return GAMMA_OK;
}

}  // extern "C"
