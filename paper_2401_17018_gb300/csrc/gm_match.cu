// gm_match.cu -- seeding (Alg. 1, lines 2-6) and the DFS extension kernel
// (Alg. 1 with GenCandidates and the duplicate-free total order of Sec. IV-C).
//
// Seeding: one thread per update looks up the plans whose first two labels
// equal the labels of the update's endpoints (min, max), applies the
// neighbour-label-count filter to both, picks the shorter of the label-L(pi[2])
// segments of their lists as the level-2 driver and writes work items of at
// most `grain` level-2 candidates each.
//
// DFS: persistent warps pull work items from a global cursor.  Each warp runs
// a depth-first search whose unit is a tile: for every stored level it keeps
// up to `tile` partial matches (vertex + parent index).  Expanding a level
// maps the 32 lanes onto the next 32 (partial match, driver-segment slot)
// pairs of the whole tile, so lanes stay busy even when single segments are
// short; survivors are compacted with a ballot into the next level's tile,
// and the warp descends when that tile is full or the parent is exhausted.
// A candidate c for position l, drawn from the label-L(pi[l]) segment of the
// neighbour list of its driver (the backward neighbour with the fewest such
// neighbours), must: be visible in the seed's view with the charging rule
// (untagged edge, or a same-sign update edge of larger index), differ from
// the already-matched vertices of its label (injectivity), be adjacent in the
// same sense to every other backward neighbour (binary search of its key in
// that neighbour's sorted list), and, below the last level, pass the
// neighbour-label-count filter.  The last level is only counted (and
// optionally written out).
#include <atomic>

#include "gm_graph.cuh"

namespace {

// a flag read by lane 0 and broadcast, so the whole warp takes the same branch
__device__ __forceinline__ int warp_read(const int32_t *p) {
  int v = 0;
  if ((threadIdx.x & 31) == 0) v = *(const volatile int32_t *)p;
  return __shfl_sync(GM_FULL, v, 0);
}

// Visibility of a batch-tagged edge (tag = update index << 1 | deletion) to a
// seed of update `upd` with sign `sdel` from request `r`.  Same request: the
// seed's view (G' for insertions, G for deletions) plus the charging rule
// (only same-sign updates of larger index).  Several requests staged together
// are applied in order: the tag is the first update of the edge's chain, the
// later ones follow through cnext; an earlier request's insertion is already
// present and its deletion already gone, a later request's update has not
// happened yet (so the edge is there exactly when the chain's first update is
// a deletion, or the last earlier request inserted it).
__device__ __forceinline__ bool tag_ok(uint32_t t, uint32_t sdel, uint32_t upd, const uint32_t *req,
                                       uint32_t r, const uint32_t *cnext, const int8_t *op) {
  uint32_t k = t >> 1, d = t & 1u;
  if (!req) return d == sdel && k > upd;
  bool present = d == 1u;  // before the chain's first update
  while (true) {
    const uint32_t rk = __ldg(req + k);
    if (rk == r) return d == sdel && k > upd;
    if (rk > r) return present;
    present = d == 0u;  // after an earlier request's update
    const uint32_t nx = cnext ? __ldg(cnext + k) : ~0u;
    if (nx == ~0u) return present;
    k = nx;
    d = __ldg(op + k) < 0 ? 1u : 0u;
  }
}

// Algorithmic-byte accumulator: counts only in the instrumented build of the
// DFS kernel (C = true); in the timed build every update compiles away.
template <bool C>
struct ByteCount {
  uint64_t v = 0;
  __device__ __forceinline__ void operator+=(uint64_t x) {
    if (C) v += x;
  }
};

// algorithmic bytes of one binary search over a list of d entries: one 32-B
// sector per halving step, never more than the whole list
__device__ __forceinline__ uint32_t probe_bytes(uint32_t d) {
  uint32_t steps = 32u - __clz(d | 1u);
  return min(4u * d, 32u * steps) + 8u;
}

// A list's membership index in 8 bytes: {first hash slot, log2 capacity} for
// a hash-indexed list, else {list offset, length | GM_DESC_LIST}.
#define GM_DESC_LIST 0x80000000u
__device__ __forceinline__ uint2 edge_desc(const GraphDev &g, uint32_t w) {
  const uint2 t = g.elab ? make_uint2(0, 0) : __ldg(g.hub_tab + w);  // hash sets hold keys only, not labels
  if (t.y) return t;
  const uint2 a = __ldg(reinterpret_cast<const uint2 *>(g.adj) + w);
  return make_uint2(a.x, a.y | GM_DESC_LIST);
}

// is the edge (w, c) visible in the seed's view under the charging rule, and,
// in an edge-labelled graph, labelled el?  x = adjacency key of c (flag bit
// ignored), D = edge_desc(g, w)
template <bool C>
__device__ __forceinline__ bool edge_ok_d(const GraphDev &g, uint32_t w, uint2 D, uint32_t x, uint32_t el,
                                          uint32_t sdel, uint32_t upd, const uint32_t *req, uint32_t r,
                                          const uint32_t *cnext, const int8_t *op, ByteCount<C> &bytes) {
  const uint32_t key = x & ~1u;
  uint2 a;
  if (!(D.y & GM_DESC_LIST)) {
    // hash-indexed list: probe its set; a flagged key still needs the tag from the list
    const uint32_t mask = (1u << D.y) - 1u;
    const uint32_t *T = g.hub_keys + D.x;
    uint32_t p = gm_hash(key >> 1) & mask;
    bytes += 12;
    for (uint32_t probe = 0; probe <= mask; probe++) {
      const uint32_t e = __ldg(T + p);
      bytes += (probe == 0 || (p & 7u) == 0) ? 32 : 0;
      if (e == GM_EMPTY) return false;
      if ((e | 1u) == (key | 1u)) {
        if (!(e & 1u)) return true;
        break;  // batch edge: fetch its tag below
      }
      p = (p + 1) & mask;
    }
    a = __ldg(reinterpret_cast<const uint2 *>(g.adj) + w);
  } else {
    a = make_uint2(D.x, D.y & ~GM_DESC_LIST);
  }
  if (a.y <= GM_SCAN_MAX) {
    // a short list is read whole: independent 16-byte loads from the aligned
    // word before it (the pool is padded), one memory round trip instead of
    // a chain of binary-search steps
    const uint32_t b0 = a.x & ~3u, off = a.x - b0, end = off + a.y;
    const uint4 *P4 = reinterpret_cast<const uint4 *>(g.col + b0);
    int hit = -1;
    uint32_t hy = 0;
#pragma unroll
    for (int j = 0; j < (GM_SCAN_MAX + 3) / 4 + 1; j++) {
      if (4u * j < end) {
        const uint4 q4 = __ldg(P4 + j);
        const uint32_t wv[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
        for (int t = 0; t < 4; t++) {
          const uint32_t idx = 4u * j + t;
          if (idx >= off && idx < end && (wv[t] | 1u) == (key | 1u)) { hit = (int)(idx - off); hy = wv[t]; }
        }
      }
    }
    bytes += 16u * ((end + 3) / 4) + 8u;
    if (hit < 0) return false;
    if (g.elab && __ldg(g.elab + a.x + hit) != el) return false;
    if (hy & 1u) return tag_ok(__ldg(g.etag + a.x + hit), sdel, upd, req, r, cnext, op);
    return true;
  }
  bytes += probe_bytes(a.y);
  const uint32_t *L = g.col + a.x;
  uint32_t p = gm_lower_bound(L, a.y, key);
  if (p >= a.y) return false;
  uint32_t y = __ldg(L + p);
  if ((y | 1u) != (key | 1u)) return false;
  if (g.elab && __ldg(g.elab + a.x + p) != el) return false;
  if (y & 1u) return tag_ok(__ldg(g.etag + a.x + p), sdel, upd, req, r, cnext, op);
  return true;
}

template <bool C>
__device__ __forceinline__ bool edge_ok(const GraphDev &g, uint32_t w, uint32_t x, uint32_t el, uint32_t sdel,
                                        uint32_t upd, const uint32_t *req, uint32_t r, const uint32_t *cnext,
                                        const int8_t *op, ByteCount<C> &bytes) {
  return edge_ok_d(g, w, edge_desc(g, w), x, el, sdel, upd, req, r, cnext, op, bytes);
}

// size of N^lab(v) for choosing a driver: the per-label count, exact below
// 255; a saturated count is made exact from the hash index's label-segment
// starts, or, for a vertex without one, ranked after every exact size
__device__ __forceinline__ uint32_t seg_size(const GraphDev &g, uint32_t v, int lab) {
  const uint32_t c = __ldg(g.nlf + (size_t)v * g.nlfw + lab);
  if (c < 255u) return c;
  const int32_t h = __ldg(g.hub_id + v);
  if (h < 0) return 1u << 30;
  const uint32_t *o = g.hub_lofs + (size_t)h * (g.nlab + 1) + lab;
  return __ldg(o + 1) - __ldg(o);
}

__device__ __forceinline__ bool nlf_ok(const GraphDev &g, uint32_t v, const Plan &P, int pos) {
  const uint8_t *row = g.nlf + (size_t)v * g.nlfw;
  int nr = P.nreq[pos];
  for (int r = 0; r < nr; r++)
    if (__ldg(row + P.req_lab[pos][r]) < P.req_cnt[pos][r]) return false;
  return true;
}

// [lo, hi) of the label-`lab` segment of list L (len entries)
__device__ __forceinline__ void seg_bounds(const GraphDev &g, const uint32_t *L, uint32_t len, int lab,
                                           uint32_t &lo, uint32_t &hi) {
  const int s = g.idb + 1;
  lo = gm_lower_bound(L, len, (uint32_t)lab << s);
  uint64_t up = (uint64_t)(lab + 1) << s;
  hi = (up >> 32) ? len : gm_lower_bound(L, len, (uint32_t)up);
}

// absolute col slot and length of N^lab(v): from the hub offset table, else
// from the prefix of v's per-label counts when none of them is saturated,
// else by binary search
template <bool C>
__device__ __forceinline__ void label_segment(const GraphDev &g, uint32_t v, int lab, uint32_t &lo,
                                              uint32_t &len, ByteCount<C> &bytes) {
  const uint2 a = __ldg(reinterpret_cast<const uint2 *>(g.adj) + v);
  const int32_t h = __ldg(g.hub_id + v);
  bytes += 12;
  if (h >= 0) {
    const uint32_t *o = g.hub_lofs + (size_t)h * (g.nlab + 1) + lab;
    const uint32_t s0 = __ldg(o), s1 = __ldg(o + 1);
    lo = a.x + s0;
    len = s1 - s0;
    bytes += 8;
    return;
  }
  const uint8_t *row = g.nlf + (size_t)v * g.nlfw;
  uint32_t pre = 0, sat = 0;
  for (int l = 0; l < lab; l++) {
    const uint32_t c = __ldg(row + l);
    pre += c;
    sat |= (c == 255u);
  }
  const uint32_t c = __ldg(row + lab);
  bytes += lab + 1;
  if (!sat && c < 255u) {
    lo = a.x + pre;
    len = c;
    return;
  }
  uint32_t slo, shi;
  seg_bounds(g, g.col + a.x, a.y, lab, slo, shi);
  bytes += 2u * probe_bytes(a.y);
  lo = a.x + slo;
  len = shi - slo;
}

// ------------------------------------------------------------------ seeding
__global__ void k_seed(MatchArgs a) {
  const GraphDev &g = a.g;
  GmStatus *st = a.st;
  if (*(volatile int32_t *)&st->err) return;
  const int lane = threadIdx.x & 31;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // Work items come out in seeding order, and the DFS warps take them in
  // that order.  With seed_sorted, thread t takes entry t of the batch sorted
  // by vertex and seeds the update there only if that vertex is the
  // update's endpoint of higher degree (ties: smaller id): the updates at one
  // hub then sit together, so warps that run at the same time search around
  // the same hub and share its lists and hash set in L2.
  const int64_t nit = a.seed_sorted ? (int64_t)a.n2 : a.b;
  // grid-stride loop with a warp-uniform trip count for the warp-aggregated atomics
  int64_t b_round = ((nit + 31) / 32) * 32;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < b_round; t += stride) {
    bool act = t < nit;
    int64_t k = t;
    if (act && a.seed_sorted) {
      const uint64_t key = a.bkeys[t];
      if (key == ~0ull) {
        act = false;
      } else {
        k = (int64_t)(a.bvals[t] >> 1);
        const uint32_t x = (uint32_t)(key >> 33);
        const uint32_t y = (a.cu[k] == x) ? a.cv[k] : a.cu[k];
        const uint32_t dx = a.g.adj[x].y, dy = a.g.adj[y].y;
        act = dx > dy || (dx == dy && x < y);
      }
    }
    uint32_t v1 = 0, v2 = 0, sdel = 0;
    uint32_t p0 = 0, p1 = 0;
    if (act) {
      v1 = a.cu[k]; v2 = a.cv[k];
      sdel = a.op[k] < 0 ? 1u : 0u;
      int l1 = __ldg(g.label + v1), l2 = __ldg(g.label + v2);
      uint32_t pr = (uint32_t)l1 * g.nlab + l2;
      p0 = a.pair_off[pr]; p1 = a.pair_off[pr + 1];
    }
    uint32_t my_items = 0, my_seeds = 0;
    // pass 1: count items; pass 2: write them at a warp-aggregated offset
    for (int pass = 0; pass < 2; pass++) {
      uint64_t base = 0;
      if (pass == 1) {
        uint32_t inc = my_items;
        for (int d = 1; d < 32; d <<= 1) {
          uint32_t y = __shfl_up_sync(GM_FULL, inc, d);
          if (lane >= d) inc += y;
        }
        uint32_t wtot = __shfl_sync(GM_FULL, inc, 31);
        uint64_t wb = 0;
        if (lane == 31 && wtot) wb = atomicAdd((unsigned long long *)&st->nitems, (unsigned long long)wtot);
        wb = __shfl_sync(GM_FULL, wb, 31);
        base = wb + inc - my_items;
        uint32_t sd = my_seeds;
        for (int d = 16; d > 0; d >>= 1) sd += __shfl_down_sync(GM_FULL, sd, d);
        if (lane == 0 && sd) atomicAdd((unsigned long long *)&st->nseeds, (unsigned long long)sd);
      }
      for (uint32_t pi = p0; pi < p1; pi++) {
        const int pidx = a.pair_plans[pi];
        const Plan &P = a.plans[pidx];
        if (a.qfilter >= 0 && P.qslot != a.qfilter) continue;
        if (a.use_filter && !(nlf_ok(g, v1, P, 0) && nlf_ok(g, v2, P, 1))) continue;
        if (g.elab && a.ulab[k] != P.el[1][0]) continue;  // the update's edge label against the query edge's
        if (P.q == 2) {
          if (pass == 0) {
            my_seeds++;
            const uint32_t rq = a.req ? a.req[k] : 0u;
            atomicAdd((unsigned long long *)&a.cnt[((uint64_t)rq * a.nq + P.qslot) * 2 + sdel], 1ull);
            if (a.per_upd) atomicAdd((unsigned long long *)&a.per_upd[(uint64_t)P.qslot * a.b + k], 1ull);
            if (a.rows) {
              uint64_t r = atomicAdd((unsigned long long *)&st->rows, 1ull);
              if (r < a.row_cap) {
                int32_t *row = a.rows + r * a.row_stride;
                row[0] = P.qid; row[1] = (int32_t)k; row[2] = sdel ? -1 : 1;
                for (int c = 3; c < a.row_stride; c++) row[c] = -1;
                row[3 + P.qv[0]] = (int32_t)v1;
                row[3 + P.qv[1]] = (int32_t)v2;
              }
            }
          }
          continue;
        }
        // level-2 driver: the backward neighbour (position 0 or 1) of pi[2]
        // whose label-L(pi[2]) segment is shorter
        const int lab2 = P.lab[2];
        const uint16_t bw = P.bwd[2];
        uint32_t best_len = 0xffffffffu, best_lo = 0;
        int drv = 0;
        ByteCount<false> nb;
        for (int pos = 0; pos < 2; pos++) {
          if (!((bw >> pos) & 1)) continue;
          uint32_t lo, len;
          label_segment(g, pos ? v2 : v1, lab2, lo, len, nb);
          if (len < best_len) { best_len = len; best_lo = lo; drv = pos; }
        }
        if (best_len == 0 || best_len == 0xffffffffu) continue;
        uint32_t nit = (best_len + a.grain - 1) / a.grain;
        if (pass == 0) {
          my_items += nit;
          my_seeds++;
        } else {
          for (uint32_t j = 0; j < nit; j++) {
            uint64_t slot = base + j;
            if (slot < a.item_cap) {
              WorkItem w;
              w.upd = (uint32_t)k;
              w.plan = (uint16_t)pidx;
              w.drv = (uint8_t)drv;
              w.pad = 0;
              w.lo = best_lo + j * a.grain;
              w.len = min((uint32_t)a.grain, best_len - j * a.grain);
              a.items[slot] = w;
            }
          }
          base += nit;
        }
      }
    }
  }
}

// ------------------------------------------------------------------ DFS
struct WarpHdr {
  Plan plan;
  uint32_t cnt[GM_MAXQ];   // entries stored per level
  uint32_t cur[GM_MAXQ];   // expansion pairs consumed per level
  uint32_t tot[GM_MAXQ];   // expansion pairs this warp still owns per level
  uint32_t full[GM_MAXQ];  // expansion pairs of the level before any donation
  uint32_t coll;           // bit L: level L's entries share their last-position candidates by sibling run
  int32_t hoist;           // level whose entries carry HO (the last level, prepared), else -1
};

__host__ __device__ inline size_t smem_per_warp(int tile, int nlev) {
  size_t b = sizeof(WarpHdr);
  b = (b + 15) & ~(size_t)15;
  size_t lt = (size_t)nlev * tile;
  b += lt * 4 * 3;              // V, LO, EX
  b += lt * 2;                  // PAR
  b += lt * 2;                  // MUL
  b += lt;                      // DRV
  b = (b + 15) & ~(size_t)15;
  b += (size_t)tile * 16;       // HO: the last level's first membership test per entry
  return b;
}

constexpr uint32_t GM_RING_LARGE = 1u << 20;  // task rings this large take reservations without a retry loop
constexpr uint32_t DONATE_EVERY = 16;  // expansion steps between looks at the waiting tickets
constexpr uint32_t DONATE_MIN = 64;    // pairs a level must still own to be split

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int32_t vload(const int32_t *p) { return *(const volatile int32_t *)p; }
__device__ __forceinline__ uint32_t vload(const uint32_t *p) { return *(const volatile uint32_t *)p; }

// lane 0 of a warp without work: take a ticket and wait (bounded) until the
// slot with that number is donated, or until no warp holds work any more.
// Returns true with the slot to run (already counted busy by its donor).
__device__ bool idle_wait(const MatchArgs &a, uint64_t &slot) {
  uint32_t *sched = a.sched;
  const uint32_t t = atomicAdd(sched + GM_SCHED_TICKET, 1u);
  const uint64_t t0 = global_ns();
  uint32_t ns = 128;
  for (uint32_t poll = 0;; poll++) {
    if (t < vload(sched + GM_SCHED_RESERVE)) {
      slot = t;
      return true;
    }
    if ((poll & 7u) == 0) {
      if (vload(&a.st->abort)) return false;
      if (vload(sched + GM_SCHED_BUSY) == 0u) {
        __threadfence();
        if (t >= vload(sched + GM_SCHED_RESERVE)) return false;
        continue;
      }
      if (global_ns() - t0 > a.idle_limit_ns) {  // nothing arrived for too long: report, do not hang
        gm_set_err(a.st, GAMMA_ETIMEOUT);
        atomicExch(&a.st->abort, 1);
        return false;
      }
    }
    __nanosleep(ns);
    if (ns < 4096) ns <<= 1;
  }
}

// lane 0 of a busy warp: reserve up to n consecutive task numbers, no more
// than the tickets of idle warps not yet matched with a task, and count
// their future runners as busy.  Returns the number granted (0: none).
// Every granted number is below the tickets taken, so each has a waiting
// receiver: donors that read the same demand at once cannot flood the queue
// with tasks nobody waits for, and task r's ring slot (r mod capacity) was
// freed by task r - capacity, whose receiver already holds its ticket.
__device__ uint32_t reserve_tasks(const MatchArgs &a, uint32_t n, uint32_t &base) {
  uint32_t *sched = a.sched;
  if (n == 0 || n > a.task_cap) return 0;
  atomicAdd(sched + GM_SCHED_BUSY, n);  // the donor itself is busy, so no warp can see zero meanwhile
  if (a.task_cap >= GM_RING_LARGE) {
    // a large ring: one atomic, no retries under contention.  The caller
    // asked for no more than the waiting tickets it read, so donors reading
    // at once overshoot by at most 32 tasks each, far below the ring's
    // capacity, and every slot's previous task was read long before.
    base = atomicAdd(sched + GM_SCHED_RESERVE, n);
    return n;
  }
  uint32_t r = vload(sched + GM_SCHED_RESERVE);
  while (true) {
    const int32_t waiting = (int32_t)(vload(sched + GM_SCHED_TICKET) - r);
    const uint32_t g = waiting > 0 ? min(n, (uint32_t)waiting) : 0u;
    if (g == 0) {
      atomicSub(sched + GM_SCHED_BUSY, n);
      return 0;
    }
    const uint32_t old = atomicCAS(sched + GM_SCHED_RESERVE, r, r + g);
    if (old == r) {
      if (g < n) atomicSub(sched + GM_SCHED_BUSY, n - g);
      base = r;
      return g;
    }
    r = old;
  }
}

// write task number r into its ring slot: wait (bounded) until the slot's
// previous task has been read, then publish r + 1 in the slot's word
__device__ bool publish_task(const MatchArgs &a, uint32_t r, const Task &t) {
  const uint32_t ph = r & (a.task_cap - 1u);
  const uint64_t t0 = global_ns();
  while (vload(&a.task_seq[ph]) != 0u) {
    if (global_ns() - t0 > a.handoff_limit_ns) {
      gm_set_err(a.st, GAMMA_ETIMEOUT);
      atomicExch(&a.st->abort, 1);
      return false;
    }
    __nanosleep(64);
  }
  a.tasks[ph] = t;
  __threadfence();
  *(volatile uint32_t *)&a.task_seq[ph] = r + 1u;
  return true;
}

// tickets waiting for a slot (warp-uniform)
__device__ __forceinline__ uint32_t demand(const MatchArgs &a) {
  int32_t d = 0;
  if ((threadIdx.x & 31) == 0)
    d = (int32_t)(vload(a.sched + GM_SCHED_TICKET) - vload(a.sched + GM_SCHED_RESERVE));
  d = __shfl_sync(GM_FULL, d, 0);
  return d > 0 ? (uint32_t)d : 0u;
}

// 64 registers a thread: 32 resident warps per SM at any block size (the
// uncapped build needs 72 and fits only 24 warps of 256-thread blocks, 15%
// slower on the mid workload; caps of 56 and 48 spill without gaining)
template <bool kCountBytes>
__global__ void __maxnreg__(64) k_dfs(MatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const GraphDev &g = a.g;
  GmStatus *st = a.st;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int T = a.tile, NL = a.nlev;
  const uint32_t lt_mask = (1u << lane) - 1u;
  unsigned char *wbase = smem + (size_t)wib * smem_per_warp(T, NL);
  WarpHdr *H = reinterpret_cast<WarpHdr *>(wbase);
  size_t o = (sizeof(WarpHdr) + 15) & ~(size_t)15;
  uint32_t *V = reinterpret_cast<uint32_t *>(wbase + o);
  uint32_t *LO = V + (size_t)NL * T;
  uint32_t *EX = LO + (size_t)NL * T;
  uint16_t *PAR = reinterpret_cast<uint16_t *>(EX + (size_t)NL * T);
  uint16_t *MUL = PAR + (size_t)NL * T;  // sibling-run length at the run's first entry
  uint8_t *DRV = reinterpret_cast<uint8_t *>(MUL + (size_t)NL * T);
  // per entry of the last level: {vertex w, its index descriptor, position} of
  // the first membership test, read once at prepare instead of per candidate
  uint4 *HO = reinterpret_cast<uint4 *>(wbase + ((o + (size_t)NL * T * 17 + 15) & ~(size_t)15));  // after DRV

  if (warp_read(&st->err)) return;
  const uint64_t nitems = min(*(volatile uint64_t *)&st->nitems, a.item_cap);
  const uint32_t ntouched = *(volatile uint32_t *)&st->ntouched;
  int cur_plan = -1;
  bool items_done = false;

  while (true) {
    // ---------------- acquire work: a seed item, else a donated task, else wait
    int kind = 0;  // 1 item, 2 task, 0 finished
    uint64_t slot = 0;
    if (lane == 0) {
      atomicAdd(a.sched + GM_SCHED_BUSY, 1u);
      if (!items_done && !vload(&st->abort)) {
        uint64_t it = atomicAdd((unsigned long long *)&st->next_item, 1ull);
        if (it < nitems) { kind = 1; slot = it; } else items_done = true;
      }
      if (!kind) {
        atomicSub(a.sched + GM_SCHED_BUSY, 1u);
        if (a.tasks && idle_wait(a, slot)) kind = 2;
      }
      if (kind == 2) {  // the donor publishes right after reserving; wait for it (bounded)
        const uint64_t t0 = global_ns();
        while (vload(&a.task_seq[slot & (a.task_cap - 1u)]) != (uint32_t)slot + 1u) {
          if (global_ns() - t0 > a.handoff_limit_ns) {
            gm_set_err(st, GAMMA_ETIMEOUT);
            atomicExch(&st->abort, 1);
            atomicSub(a.sched + GM_SCHED_BUSY, 1u);
            kind = 0;
            break;
          }
          __nanosleep(32);
        }
        __threadfence();
      }
    }
    kind = __shfl_sync(GM_FULL, kind, 0);
    if (!kind) break;
    slot = __shfl_sync(GM_FULL, slot, 0);

    // ---------------- the unit of work as (update, plan, depth, drv, lo, len, m[])
    uint32_t word = 0;  // lane j holds word j of the task record
    if (kind == 1) {
      const uint32_t *src = reinterpret_cast<const uint32_t *>(a.items + slot);
      if (lane < 4) word = src[lane];
      // WorkItem {upd, plan|drv<<16|pad<<24, lo, len} -> task words {upd, plan|depth|drv, lo, len}
      if (lane == 1) word = (word & 0xffffu) | (0xffu << 16) | (((word >> 16) & 0xffu) << 24);
    } else {
      const uint32_t ph = (uint32_t)slot & (a.task_cap - 1u);
      const uint32_t *src = reinterpret_cast<const uint32_t *>(a.tasks + ph);
      if (lane < 16) word = __ldcg(src + lane);
      __syncwarp();
      __threadfence();
      if (lane == 0) *(volatile uint32_t *)&a.task_seq[ph] = 0u;  // the ring slot is free again
    }
    const uint32_t upd = __shfl_sync(GM_FULL, word, 0);
    const uint32_t w1 = __shfl_sync(GM_FULL, word, 1);
    const uint32_t wlo = __shfl_sync(GM_FULL, word, 2);
    const uint32_t wlen = __shfl_sync(GM_FULL, word, 3);
    const int plan = (int)(w1 & 0xffffu);
    const int depth = (int)(int8_t)((w1 >> 16) & 0xffu);
    const uint32_t wdrv = (w1 >> 24) & 0xffu;
    const uint32_t mword = __shfl_sync(GM_FULL, word, (lane + 4) & 31);  // m[lane]

    if (plan != cur_plan) {
      const uint32_t *src = reinterpret_cast<const uint32_t *>(a.plans + plan);
      uint32_t *dst = reinterpret_cast<uint32_t *>(&H->plan);
      for (int i = lane; i < (int)(sizeof(Plan) / 4); i += 32) dst[i] = __ldg(src + i);
      cur_plan = plan;
    }
    if (lane < GM_MAXQ) H->cnt[lane] = 0;
    if (lane == 0) { H->coll = 0; H->hoist = -1; }
    __syncwarp();
    int lev;
    uint32_t root_lo = wlo, root_len = wlen, root_cur = 0, root_drv = wdrv;
    if (depth >= 0) {
      // levels 0..depth hold the donated partial match; only level `depth` has pairs left
      if (lane <= depth) {
        H->cnt[lane] = 1;
        V[lane * T] = mword;
        PAR[lane * T] = 0;
        H->cur[lane] = 0;
        H->tot[lane] = (lane == depth) ? wlen : 0u;
        H->full[lane] = H->tot[lane];
      }
      if (lane == depth) {
        LO[depth * T] = wlo;
        EX[depth * T] = 0;
        DRV[depth * T] = (uint8_t)wdrv;
      }
      __syncwarp();
      lev = depth;
      root_len = 0;
    } else {
      lev = -1;
    }
    const Plan &P = H->plan;
    const int q = P.q, last = q - 1;
    const uint32_t m0 = __ldg(a.cu + upd), m1 = __ldg(a.cv + upd);
    const uint32_t sdel = a.op[upd] < 0 ? 1u : 0u;
    const uint32_t rq = a.req ? __ldg(a.req + upd) : 0u;
    uint64_t wcount = 0;
    ByteCount<kCountBytes> lbytes;  // this lane's algorithmic bytes (instrumented build only)
    uint32_t chunks = 0, flushed = 0;  // expansion steps of this unit; those already added to the total

    // prepare level L (position L+2): driver segment of every entry for position L+3
    // Shared-prefix coalescing: when the last query vertex is not adjacent to
    // the one before it, the children of one partial match (a run of
    // siblings, consecutive and sorted by id in the level) have the same
    // last-position candidates.  Only the run's first entry then gets a
    // driver range; each candidate it finds counts once per sibling, minus
    // the sibling it would coincide with (same label).  Counts only.
    auto prepare = [&](int L) {
      const int p = L + 2, np = p + 1;
      const uint16_t bw = P.bwd[np];
      const int lab = P.lab[np];
      const uint32_t n = H->cnt[L];
      const bool coll = a.share && np == last && !((bw >> p) & 1u) && !(a.leaf && __popc((uint32_t)bw) == 1);
      const uint16_t *par = PAR + L * T;
      uint32_t carry = 0;
      for (uint32_t base = 0; base < n; base += 32) {
        uint32_t i = base + lane;
        uint32_t len = 0, lo = 0, v2 = 0;
        int drv = 0, drv2 = -1;
        bool first = true;
        if (coll && i < n) {
          first = i == 0 || par[i] != par[i - 1];
          uint32_t j = i + 1;
          if (first)
            while (j < n && par[j] == par[i]) j++;
          MUL[L * T + i] = (uint16_t)(j - i);
        }
        if (i < n && first) {
          // the backward neighbour with the fewest label-lab neighbours
          // drives; the one with the next fewest is tested first
          uint32_t best = 0xffffffffu, bestv = 0, best2 = 0xffffffffu;
          uint32_t e = i;
          auto consider = [&](uint32_t vv, int pos) {
            const uint32_t c = seg_size(g, vv, lab);
            if (c < best) {
              if (best != 0xffffffffu) { best2 = best; v2 = bestv; drv2 = drv; }  // the old driver is now second
              best = c; bestv = vv; drv = pos;
            } else if (c < best2) {
              best2 = c; v2 = vv; drv2 = pos;
            }
          };
          for (int l2 = L; l2 >= 0; l2--) {
            int pos = l2 + 2;
            if ((bw >> pos) & 1) consider(V[l2 * T + e], pos);
            e = PAR[l2 * T + e];
          }
          if ((bw >> 1) & 1) consider(m1, 1);
          if (bw & 1) consider(m0, 0);
          lbytes += 4u * __popc(bw);
          if (best > 0) label_segment(g, bestv, lab, lo, len, lbytes);
        }
        if (i < n) {
          LO[L * T + i] = lo;
          DRV[L * T + i] = (uint8_t)drv;
        }
        if (np == last && i < n && first) {
          // the first membership test of the last position (the backward
          // neighbour other than the driver with the fewest label-lab
          // neighbours, the likeliest to reject), looked up once here
          uint32_t hp = 0xFFu;
          uint2 D = make_uint2(0, 0);
          if (drv2 >= 0 && len) {
            hp = (uint32_t)drv2;
            D = edge_desc(g, v2);
          }
          HO[i] = make_uint4(hp == 0xFFu ? 0u : v2, D.x, D.y, hp);
        }
        uint32_t inc = len;
        for (int d = 1; d < 32; d <<= 1) {
          uint32_t y = __shfl_up_sync(GM_FULL, inc, d);
          if (lane >= d) inc += y;
        }
        if (i < n) EX[L * T + i] = carry + inc - len;
        carry += __shfl_sync(GM_FULL, inc, 31);
      }
      if (lane == 0) {
        H->tot[L] = carry; H->full[L] = carry; H->cur[L] = 0;
        H->coll = coll ? (H->coll | (1u << L)) : (H->coll & ~(1u << L));
        if (np == last) H->hoist = L;
      }
      __syncwarp();
    };

    // split off the second half of the shallowest level that still owns
    // enough pairs and publish it as tasks for idle warps
    auto donate = [&](uint32_t want) {
      int L = -2;
      if (root_len > root_cur && root_len - root_cur >= DONATE_MIN) L = -1;
      for (int l = 0; L == -2 && l <= lev; l++)
        if (H->tot[l] > H->cur[l] && H->tot[l] - H->cur[l] >= DONATE_MIN && l < GM_TASK_M && !((H->coll >> l) & 1u))
          L = l;  // a shared level stays: a task could not carry its sibling runs
      if (L == -2) return;
      const uint32_t c0 = (L < 0) ? root_cur : H->cur[L];
      const uint32_t t0 = (L < 0) ? root_len : H->tot[L];
      const uint32_t s = c0 + max(32u, ((t0 - c0) / 2) & ~31u);
      if (s >= t0) return;
      if (L < 0) {
        uint32_t base = 0;
        int ok = 0;
        if (lane == 0 && reserve_tasks(a, 1, base) == 1) {
          Task t;
          t.upd = upd; t.plan = (uint16_t)plan; t.depth = -1; t.drv = (uint8_t)root_drv;
          t.lo = root_lo + s; t.len = t0 - s;
          publish_task(a, base, t);
          ok = 1;
        }
        if (__shfl_sync(GM_FULL, ok, 0)) root_len = s;
        return;
      }
      // entries covering [s, t0): donate at most 32 of them, always the tail
      const uint32_t n = H->cnt[L];
      const uint32_t *ex = EX + L * T;
      auto entry_of = [&](uint32_t x) {  // last entry with ex <= x
        uint32_t lo = 0, hi = n;
        while (hi - lo > 1) {
          uint32_t mid = (lo + hi) >> 1;
          if (ex[mid] <= x) lo = mid; else hi = mid;
        }
        return lo;
      };
      const uint32_t e_s = entry_of(s), e_end = entry_of(t0 - 1);
      const uint32_t most = min(32u, max(want, 1u));
      uint32_t nt = min(e_end - e_s + 1, most);
      uint32_t base = 0;
      if (lane == 0) nt = reserve_tasks(a, nt, base);  // the tail entries, as many as were granted
      nt = __shfl_sync(GM_FULL, nt, 0);
      if (nt == 0) return;
      base = __shfl_sync(GM_FULL, base, 0);
      const uint32_t e_first = e_end - (nt - 1);
      const uint32_t s2 = (e_first == e_s) ? s : ex[e_first];
      if ((uint32_t)lane < nt) {
        const uint32_t e = e_first + lane;
        const uint32_t elen = ((e + 1 < n) ? ex[e + 1] : H->full[L]) - ex[e];
        const uint32_t a0 = max(s2, ex[e]), a1 = min(t0, ex[e] + elen);
        Task t;
        t.upd = upd; t.plan = (uint16_t)plan; t.depth = (int8_t)L; t.drv = DRV[L * T + e];
        t.lo = LO[L * T + e] + (a0 - ex[e]);
        t.len = a1 - a0;
        uint32_t ee = e;
        for (int l2 = L; l2 >= 0; l2--) {
          t.m[l2] = V[l2 * T + ee];
          ee = PAR[l2 * T + ee];
        }
        publish_task(a, base + lane, t);
      }
      __syncwarp();
      if (lane == 0) H->tot[L] = s2;
      __syncwarp();
    };

    while (true) {
      const int c = lev + 3;  // position of the candidates produced from level lev
      uint32_t total, cur;
      if (lev < 0) { total = root_len; cur = root_cur; }
      else { total = H->tot[lev]; cur = H->cur[lev]; }
      if (cur >= total) {
        if (lev < 0) break;
        __syncwarp();
        if (lane == 0) H->cnt[lev] = 0;
        __syncwarp();
        lev--;
        continue;
      }
      const bool stored = (c != last);
      if (!stored && a.leaf && !a.rows && __popc((uint32_t)P.bwd[c]) == 1) {
        // The last vertex hangs on a single earlier vertex (a degree-1 query
        // vertex, Sec. V-B Remark): every slot of its driver slice is a match
        // except batch-tagged entries this seed must not see and vertices the
        // partial match already uses, so count the slice instead of visiting it.
        const int lab = P.lab[c];
        const uint16_t same = P.samelab[c];
        uint64_t add = 0;
        uint32_t nent = 1;
        // drop from len the slots of [lo, lo + len) in N^lab(v) the seed cannot use
        auto slice_count = [&](uint32_t v, uint32_t lo, uint32_t len, uint32_t k_lo, uint32_t k_hi) -> uint64_t {
          uint64_t cntv = len;
          const int32_t gi = __ldg(g.vgroup + v);
          lbytes += 12;
          if (gi >= 0) {  // v's batch entries: insertions, then deletions, each sorted by key
            const uint32_t s0 = __ldg(a.gstart + gi), ni = __ldg(a.gins + gi);
            const uint32_t e1 = ((uint32_t)gi + 1 < ntouched) ? __ldg(a.gstart + gi + 1) : a.n2;
            for (int part = 0; part < 2; part++) {
              const uint32_t pb = part ? s0 + ni : s0, pe = part ? e1 : s0 + ni;
              uint32_t l2 = pb, h2 = pe;
              while (l2 < h2) {
                const uint32_t mid = (l2 + h2) >> 1;
                if (((uint32_t)__ldg(a.bkeys + mid) & ~1u) < k_lo) l2 = mid + 1; else h2 = mid;
              }
              lbytes += 32u * (32u - __clz((pe - pb) | 1u));
              for (uint32_t j = l2; j < pe; j++) {
                const uint32_t kj = (uint32_t)__ldg(a.bkeys + j) & ~1u;
                lbytes += 12;
                if (kj > k_hi) break;
                if (!tag_ok(__ldg(a.bvals + j), sdel, upd, a.req, rq, a.cnext, a.op)) cntv--;
              }
            }
          }
          return cntv;
        };
        // a same-label vertex of the partial match inside the slice is not a new match
        auto conflict = [&](uint32_t v, uint32_t mv, uint32_t k_lo, uint32_t k_hi) -> uint32_t {
          const uint32_t kj = gm_key(lab, mv, g.idb);
          if (kj < k_lo || kj > k_hi) return 0u;
          return edge_ok(g, v, kj, 0u, sdel, upd, a.req, rq, a.cnext, a.op, lbytes) ? 1u : 0u;  // unlabelled graphs only
        };
        if (lev < 0) {
          if (lane == 0) {
            const uint32_t v = root_drv ? m1 : m0, lo = root_lo + cur, len = total - cur;
            const uint32_t k_lo = __ldg(g.col + lo) & ~1u, k_hi = __ldg(g.col + lo + len - 1) & ~1u;
            uint64_t cv = slice_count(v, lo, len, k_lo, k_hi);
            if (root_drv != 0 && (same & 1u)) cv -= conflict(v, m0, k_lo, k_hi);
            if (root_drv != 1 && (same & 2u)) cv -= conflict(v, m1, k_lo, k_hi);
            add = cv;
          }
        } else {
          const uint32_t n = H->cnt[lev];
          const uint32_t *ex = EX + lev * T;
          auto entry_of = [&](uint32_t x) {  // last entry with ex <= x
            uint32_t lo = 0, hi = n;
            while (hi - lo > 1) {
              uint32_t mid = (lo + hi) >> 1;
              if (ex[mid] <= x) lo = mid; else hi = mid;
            }
            return lo;
          };
          const uint32_t e0 = entry_of(cur), e1 = entry_of(total - 1);
          nent = e1 - e0 + 1;
          for (uint32_t e = e0 + lane; e <= e1; e += 32) {
            const uint32_t elen = ((e + 1 < n) ? ex[e + 1] : H->full[lev]) - ex[e];
            const uint32_t a0 = max(cur, ex[e]), a1 = min(total, ex[e] + elen);
            if (a1 <= a0) continue;
            const uint32_t lo = LO[lev * T + e] + (a0 - ex[e]), len = a1 - a0;
            const int dp = DRV[lev * T + e];
            // the driver's vertex, from the chain of entry e
            uint32_t v = (dp == 0) ? m0 : m1;
            {
              uint32_t ee = e;
              for (int l2 = lev; l2 >= 0; l2--) {
                if (l2 + 2 == dp) v = V[l2 * T + ee];
                ee = PAR[l2 * T + ee];
              }
            }
            const uint32_t k_lo = __ldg(g.col + lo) & ~1u, k_hi = __ldg(g.col + lo + len - 1) & ~1u;
            uint64_t cv = slice_count(v, lo, len, k_lo, k_hi);
            uint32_t ee = e;
            for (int l2 = lev; l2 >= 0; l2--) {
              const int pos = l2 + 2;
              if (pos != dp && ((same >> pos) & 1u)) cv -= conflict(v, V[l2 * T + ee], k_lo, k_hi);
              ee = PAR[l2 * T + ee];
            }
            if (dp != 1 && ((same >> 1) & 1u)) cv -= conflict(v, m1, k_lo, k_hi);
            if (dp != 0 && (same & 1u)) cv -= conflict(v, m0, k_lo, k_hi);
            add += cv;
          }
        }
        for (int d = 16; d > 0; d >>= 1) add += __shfl_xor_sync(GM_FULL, add, d);
        wcount += add;
        chunks += (nent + 31) / 32;
        if (lev < 0) root_cur = total;
        else if (lane == 0) H->cur[lev] = total;
        __syncwarp();
        continue;
      }
      if (stored && H->cnt[lev + 1] + 32 > (uint32_t)T) {
        prepare(lev + 1);
        lev++;
        continue;
      }
      // ---- one 32-wide expansion step
      const uint32_t gidx = cur + lane;
      bool ok = gidx < total;
      uint32_t e = 0, slot2 = 0;
      int drv;
      if (lev < 0) {
        slot2 = root_lo + gidx;
        drv = root_drv;
      } else {
        const uint32_t n = H->cnt[lev];
        const uint32_t *ex = EX + lev * T;
        uint32_t lo = 0, hi = n;  // last entry with ex <= gidx
        while (hi - lo > 1) {
          uint32_t mid = (lo + hi) >> 1;
          if (ex[mid] <= gidx) lo = mid; else hi = mid;
        }
        e = lo;
        slot2 = LO[lev * T + e] + (gidx - ex[e]);
        drv = DRV[lev * T + e];
      }
      chunks++;
      uint32_t x = ok ? __ldg(g.col + slot2) : 0u;
      if (ok && g.elab && __ldg(g.elab + slot2) != P.el[c][drv]) ok = false;  // the driver edge's label
      const uint32_t id = (x >> 1) & g.idmask;
      if (ok && (x & 1u)) ok = tag_ok(__ldg(g.etag + slot2), sdel, upd, a.req, rq, a.cnext, a.op);
      uint32_t hp = 0xFFu;  // position whose membership test was looked up at prepare
      if (!stored && lev >= 0 && H->hoist == lev) {
        const uint4 h = HO[e];
        hp = h.w;
        if (ok && hp != 0xFFu)
          ok = edge_ok_d(g, h.x, make_uint2(h.y, h.z), x, P.el[c][hp], sdel, upd, a.req, rq, a.cnext, a.op, lbytes);
      }
      const uint16_t chk_edge = P.bwd[c] & (uint16_t)~(1u << drv) & (uint16_t)~(hp < 16u ? (1u << hp) : 0u);
      const bool shared = !stored && lev >= 0 && ((H->coll >> lev) & 1u);
      // shared: the run's siblings differ at position lev + 2 only; that
      // position is no backward neighbour of c, and equality with it is
      // settled per sibling below
      const uint16_t chk_neq = shared ? (uint16_t)(P.samelab[c] & ~(1u << (lev + 2))) : P.samelab[c];
      if (ok && (chk_edge | chk_neq)) {
        uint32_t ee = e;
        // walk the stored positions only down to the lowest one with a check
        const uint32_t need_hi = (uint32_t)(chk_edge | chk_neq) & ~3u;
        const int stop = need_hi ? __ffs(need_hi) - 3 : lev + 1;
        for (int l2 = lev; l2 >= stop && ok; l2--) {
          const int pos = l2 + 2;
          const uint32_t vv = V[l2 * T + ee];
          if ((chk_neq >> pos) & 1) ok = (vv != id);
          if (ok && ((chk_edge >> pos) & 1))
            ok = edge_ok(g, vv, x, P.el[c][pos], sdel, upd, a.req, rq, a.cnext, a.op, lbytes);
          ee = PAR[l2 * T + ee];
        }
        if (ok && ((chk_neq >> 1) & 1)) ok = (m1 != id);
        if (ok && ((chk_edge >> 1) & 1)) ok = edge_ok(g, m1, x, P.el[c][1], sdel, upd, a.req, rq, a.cnext, a.op, lbytes);
        if (ok && (chk_neq & 1)) ok = (m0 != id);
        if (ok && (chk_edge & 1)) ok = edge_ok(g, m0, x, P.el[c][0], sdel, upd, a.req, rq, a.cnext, a.op, lbytes);
      }
      if (ok && stored && a.use_filter) ok = nlf_ok(g, id, P, c);
      if (gidx < total) lbytes += ((x & 1u) ? 8u : 4u) + (ok ? 8u : 0u);
      const unsigned mask = __ballot_sync(GM_FULL, ok);
      if (shared) {
        uint32_t add = 0;
        if (ok) {
          const uint32_t m = MUL[lev * T + e];
          add = m;
          if ((P.samelab[c] >> (lev + 2)) & 1u) {  // is the candidate one of the siblings (sorted by id)?
            const uint32_t *sv = V + lev * T + e;
            uint32_t l2 = 0, h2 = m;
            while (l2 < h2) {
              const uint32_t mid = (l2 + h2) >> 1;
              if (sv[mid] < id) l2 = mid + 1; else h2 = mid;
            }
            if (l2 < m && sv[l2] == id) add--;
            lbytes += 4u * (32u - __clz(m));
          }
        }
        wcount += __reduce_add_sync(GM_FULL, add);
      } else if (!stored) {
        wcount += __popc(mask);
        if (a.rows && mask) {
          uint64_t rb = 0;
          if (lane == 0) rb = atomicAdd((unsigned long long *)&st->rows, (unsigned long long)__popc(mask));
          rb = __shfl_sync(GM_FULL, rb, 0);
          if (ok) {
            uint64_t r = rb + __popc(mask & lt_mask);
            if (r < a.row_cap) {
              int32_t *row = a.rows + r * a.row_stride;
              row[0] = P.qid; row[1] = (int32_t)upd; row[2] = sdel ? -1 : 1;
              for (int cc = 3 + q; cc < a.row_stride; cc++) row[cc] = -1;
              row[3 + P.qv[c]] = (int32_t)id;
              uint32_t ee = e;
              for (int l2 = lev; l2 >= 0; l2--) {
                row[3 + P.qv[l2 + 2]] = (int32_t)V[l2 * T + ee];
                ee = PAR[l2 * T + ee];
              }
              row[3 + P.qv[1]] = (int32_t)m1;
              row[3 + P.qv[0]] = (int32_t)m0;
            }
          }
        }
      } else if (mask) {
        const uint32_t nb = H->cnt[lev + 1];
        if (ok) {
          uint32_t r = nb + __popc(mask & lt_mask);
          V[(lev + 1) * T + r] = id;
          PAR[(lev + 1) * T + r] = (uint16_t)e;
        }
        __syncwarp();
        if (lane == 0) H->cnt[lev + 1] = nb + __popc(mask);
      }
      const uint32_t ncur = cur + 32;
      if (lev < 0) root_cur = ncur;
      else if (lane == 0) H->cur[lev] = ncur;
      __syncwarp();
      if (stored && ncur >= total && H->cnt[lev + 1] > 0) {
        prepare(lev + 1);
        lev++;
      }
      if (a.tasks && (chunks % DONATE_EVERY) == 0) {
        const uint32_t want = demand(a);
        if (want) donate(want);
      }
      if (chunks - flushed >= 1024u) {  // add to the total as we go, so a budget stops a long unit too
        if (lane == 0) {
          const unsigned long long d = chunks - flushed;
          const unsigned long long ex = atomicAdd((unsigned long long *)&st->expansions, d) + d;
          if (a.budget && ex > a.budget) {
            atomicExch(&st->abort, 1);
            gm_set_err(st, GAMMA_ETIMEOUT);
          }
        }
        flushed = chunks;
        if (warp_read(&st->abort)) break;
      }
    }
    if (kCountBytes) {
      uint64_t tb = lbytes.v + ((lane == 0) ? 16u : 0u);
      for (int d = 16; d > 0; d >>= 1) tb += __shfl_down_sync(GM_FULL, tb, d);
      if (lane == 0) atomicAdd((unsigned long long *)&st->alg_bytes, (unsigned long long)tb);
    }
    if (lane == 0) {
      if (wcount) {
        atomicAdd((unsigned long long *)&a.cnt[((uint64_t)rq * a.nq + P.qslot) * 2 + sdel], (unsigned long long)wcount);
        if (a.per_upd)
          atomicAdd((unsigned long long *)&a.per_upd[(uint64_t)P.qslot * a.b + upd], (unsigned long long)wcount);
      }
      const unsigned long long d = chunks - flushed;
      unsigned long long ex = atomicAdd((unsigned long long *)&st->expansions, d);
      if (a.budget && ex + d > a.budget) {
        atomicExch(&st->abort, 1);
        gm_set_err(st, GAMMA_ETIMEOUT);
      }
      __threadfence();
      atomicSub(a.sched + GM_SCHED_BUSY, 1u);
    }
    __syncwarp();
  }
}

}  // namespace

size_t gm_dfs_smem_per_warp(int tile, int nlev) { return smem_per_warp(tile, nlev); }

int gm_seed(const MatchArgs &a, cudaStream_t s) {
  if (a.b <= 0 || a.nplans <= 0) return GAMMA_OK;
  int threads = 256;
  const int64_t nit = a.seed_sorted ? (int64_t)a.n2 : a.b;
  int64_t blocks = (nit + threads - 1) / threads;
  if (blocks > 65536) blocks = 65536;
  k_seed<<<(int)blocks, threads, 0, s>>>(a);
  GM_LAUNCHED();
  GM_CUDA(cudaGetLastError());
  return GAMMA_OK;
}

template <bool kCountBytes>
static int launch_dfs(const MatchArgs &a, int num_sms, cudaStream_t s) {
  const int wpb = a.warps_per_block;
  const size_t smem = smem_per_warp(a.tile, a.nlev) * wpb;
  // the dynamic shared-memory limit is a per-device property of the kernel:
  // remember, per device ordinal, the largest size already allowed
  static std::atomic<size_t> configured[GM_MAX_DEVICES];
  int dev = 0;
  GM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= GM_MAX_DEVICES) return GAMMA_EINVAL;
  if (smem > 48 * 1024 && smem > configured[dev].load()) {
    GM_CUDA(cudaFuncSetAttribute(k_dfs<kCountBytes>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    size_t prev = configured[dev].load();
    while (prev < smem && !configured[dev].compare_exchange_weak(prev, smem)) {
    }
  }
  int per_sm = 0;
  GM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfs<kCountBytes>, wpb * 32, smem));
  if (per_sm < 1) return GAMMA_EINVAL;
  GM_CUDA(cudaMemsetAsync(a.sched, 0, GM_SCHED_WORDS * sizeof(uint32_t), s));
  k_dfs<kCountBytes><<<num_sms * per_sm, wpb * 32, smem, s>>>(a);
  GM_LAUNCHED();
  GM_CUDA(cudaGetLastError());
  GM_CUDA(cudaMemcpyAsync(&a.st->tasks_donated, a.sched + GM_SCHED_RESERVE, sizeof(uint32_t),
                          cudaMemcpyDeviceToDevice, s));
  return GAMMA_OK;
}

int gm_dfs(const MatchArgs &a, int num_sms, cudaStream_t s) {
  return a.count_bytes ? launch_dfs<true>(a, num_sms, s) : launch_dfs<false>(a, num_sms, s);
}
