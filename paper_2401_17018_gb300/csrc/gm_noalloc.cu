// gm_noalloc.cu -- gamma_recount_noalloc: the DFS kernel re-run over the
// staged batch without allocating anything.
//
// Who needs it: callers that cannot allocate device memory when they want
// the counts -- an application whose device memory is entirely reserved by
// another allocator (a framework's caching allocator or a preallocated
// arena, so cudaMalloc would fail), or a latency-critical loop that may not
// pay for cudaMalloc / cudaFree, which can synchronize the whole device.
// The DFS normally takes its scratch (donated-task queue, scheduling
// counters, count accumulators) from buffers the context allocates; here
// that scratch lives in one file-scope device array.
//
// The array is part of the library image: every GPU that loads the library
// holds it (about 1.2 MB) until the process exits.  All calls share it and it
// keeps the last call's contents, so each call clears what must start at zero;
// two calls whose work overlaps on the GPU (different streams or threads)
// would race on it and must not be issued.
#include <mutex>

#include "gm_graph.cuh"

#define GM_NOALLOC_SLOTS 256    // requests x queries of the staged batch, at most
#define GM_NOALLOC_TASKS 16384  // donated-task slots

namespace {

struct NoallocScratch {
  unsigned long long cnt[2 * GM_NOALLOC_SLOTS];
  uint32_t sched[GM_SCHED_WORDS];
  uint32_t task_seq[GM_NOALLOC_TASKS];
  Task tasks[GM_NOALLOC_TASKS];
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

std::mutex g_mu;
void *g_addr[128];  // device address of the array, per device ordinal (set up once)

}  // namespace

int gm_recount_prepare(gamma_ctx *ctx, MatchArgs *a, int *nslots, int *num_sms, cudaStream_t *stream);
int gm_ctx_device(gamma_ctx *ctx);
int gm_ctx_fail(gamma_ctx *ctx, int code, const char *msg);
void gm_recount_done(gamma_ctx *ctx, uint64_t expansions, uint32_t donated);

extern "C" int gamma_recount_noalloc(gamma_ctx *ctx, int32_t cap, uint64_t *out_pos, uint64_t *out_neg) {
  if (!ctx) return GAMMA_EINVAL;
  if (!out_pos || !out_neg || cap < 1) return gm_ctx_fail(ctx, GAMMA_EINVAL, "gamma_recount_noalloc: no output arrays");
  MatchArgs a;
  int nslots = 0, num_sms = 0;
  cudaStream_t s = nullptr;
  int rc = gm_recount_prepare(ctx, &a, &nslots, &num_sms, &s);
  if (rc) return rc;
  if (nslots > GM_NOALLOC_SLOTS)
    return gm_ctx_fail(ctx, GAMMA_EINVAL, "gamma_recount_noalloc: more than 256 request x query slots");
  if (nslots > cap)
    return gm_ctx_fail(ctx, GAMMA_EINVAL, "gamma_recount_noalloc: the output arrays hold fewer entries than "
                                          "requests x queries of the staged batch");
  const int dev = gm_ctx_device(ctx);
  if (dev < 0 || dev >= 128) return gm_ctx_fail(ctx, GAMMA_EINVAL, "gamma_recount_noalloc: device ordinal >= 128");
  if (cudaSetDevice(dev) != cudaSuccess) return gm_ctx_fail(ctx, GAMMA_ECUDA, "gamma_recount_noalloc: cudaSetDevice failed");
  void *base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {  // once per device, with that device current
      cudaError_t e = cudaGetSymbolAddress(&g_addr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_addr[dev] = nullptr;
        return gm_ctx_fail(ctx, GAMMA_ECUDA, "gamma_recount_noalloc: cudaGetSymbolAddress failed");
      }
    }
    base = g_addr[dev];
  }
  NoallocScratch *sc = reinterpret_cast<NoallocScratch *>(base);
  a.cnt = reinterpret_cast<uint64_t *>(sc->cnt);
  a.sched = sc->sched;
  a.task_seq = sc->task_seq;
  a.tasks = sc->tasks;
  a.task_cap = GM_NOALLOC_TASKS;
  // zero what the kernel accumulates into; restart the work-item cursor
  if (cudaMemsetAsync(sc->cnt, 0, sizeof(unsigned long long) * 2 * nslots, s) != cudaSuccess ||
      cudaMemsetAsync(sc->task_seq, 0, sizeof(sc->task_seq), s) != cudaSuccess ||
      cudaMemsetAsync(&a.st->next_item, 0, sizeof(uint64_t), s) != cudaSuccess ||
      cudaMemsetAsync(&a.st->expansions, 0, sizeof(uint64_t), s) != cudaSuccess ||
      cudaMemsetAsync(&a.st->abort, 0, sizeof(int32_t), s) != cudaSuccess)
    return gm_ctx_fail(ctx, GAMMA_ECUDA, "gamma_recount_noalloc: cudaMemsetAsync failed");
  rc = gm_dfs(a, num_sms, s);  // clears the scheduling counters, then launches the DFS
  if (rc) return gm_ctx_fail(ctx, rc, "gamma_recount_noalloc: DFS launch failed");
  int32_t err = 0;
  uint64_t expansions = 0;
  uint32_t donated = 0;
  uint64_t tmp[2 * GM_NOALLOC_SLOTS];
  if (cudaMemcpyAsync(tmp, sc->cnt, sizeof(uint64_t) * 2 * nslots, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&err, &a.st->err, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&expansions, &a.st->expansions, sizeof(uint64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&donated, &a.st->tasks_donated, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return gm_ctx_fail(ctx, GAMMA_ECUDA, "gamma_recount_noalloc: copy failed");
  gm_recount_done(ctx, expansions, donated);
  for (int j = 0; j < nslots; j++) {
    out_pos[j] = tmp[2 * j];
    out_neg[j] = tmp[2 * j + 1];
  }
  if (err) return gm_ctx_fail(ctx, err, "gamma_recount_noalloc: the DFS reported an error");
  return GAMMA_OK;
}
