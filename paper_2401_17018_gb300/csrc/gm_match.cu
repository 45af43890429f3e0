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
#include "gm_graph.cuh"

namespace {

// a flag read by lane 0 and broadcast, so the whole warp takes the same branch
__device__ __forceinline__ int warp_read(const int32_t *p) {
  int v = 0;
  if ((threadIdx.x & 31) == 0) v = *(const volatile int32_t *)p;
  return __shfl_sync(GM_FULL, v, 0);
}

__device__ __forceinline__ bool tag_ok(uint32_t t, uint32_t sdel, uint32_t upd) {
  return ((t & 1u) == sdel) && ((t >> 1) > upd);
}

// is the edge (w, c) visible in the seed's view under the charging rule?
// x = adjacency key of c (flag bit ignored)
// algorithmic bytes of one binary search over a list of d entries: one 32-B
// sector per halving step, never more than the whole list
__device__ __forceinline__ uint32_t probe_bytes(uint32_t d) {
  uint32_t steps = 32u - __clz(d | 1u);
  return min(4u * d, 32u * steps) + 8u;
}

__device__ __forceinline__ bool edge_ok(const GraphDev &g, uint32_t w, uint32_t x, uint32_t sdel,
                                        uint32_t upd, uint64_t &bytes) {
  const uint2 a = __ldg(reinterpret_cast<const uint2 *>(g.adj) + w);
  bytes += probe_bytes(a.y);
  const uint32_t *L = g.col + a.x;
  const uint32_t key = x & ~1u;
  uint32_t p = gm_lower_bound(L, a.y, key);
  if (p >= a.y) return false;
  uint32_t y = __ldg(L + p);
  if ((y | 1u) != (key | 1u)) return false;
  if (y & 1u) return tag_ok(__ldg(g.etag + a.x + p), sdel, upd);
  return true;
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

// ------------------------------------------------------------------ seeding
__global__ void k_seed(MatchArgs a) {
  const GraphDev &g = a.g;
  GmStatus *st = a.st;
  if (*(volatile int32_t *)&st->err) return;
  const int lane = threadIdx.x & 31;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // grid-stride loop with a warp-uniform trip count for the warp-aggregated atomics
  int64_t b_round = ((a.b + 31) / 32) * 32;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < b_round; k += stride) {
    const bool act = k < a.b;
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
        if (a.use_filter && !(nlf_ok(g, v1, P, 0) && nlf_ok(g, v2, P, 1))) continue;
        if (P.q == 2) {
          if (pass == 0) {
            my_seeds++;
            atomicAdd((unsigned long long *)&a.cnt[P.qslot * 2 + sdel], 1ull);
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
        for (int pos = 0; pos < 2; pos++) {
          if (!((bw >> pos) & 1)) continue;
          uint32_t w = pos ? v2 : v1;
          uint2 ad = __ldg(reinterpret_cast<const uint2 *>(g.adj) + w);
          uint32_t lo, hi;
          seg_bounds(g, g.col + ad.x, ad.y, lab2, lo, hi);
          if (hi - lo < best_len) { best_len = hi - lo; best_lo = ad.x + lo; drv = pos; }
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
  uint32_t cnt[GM_MAXQ];
  uint32_t cur[GM_MAXQ];
  uint32_t tot[GM_MAXQ];
};

__host__ __device__ inline size_t smem_per_warp(int tile, int nlev) {
  size_t b = sizeof(WarpHdr);
  b = (b + 15) & ~(size_t)15;
  size_t lt = (size_t)nlev * tile;
  b += lt * 4 * 3;              // V, LO, EX
  b += lt * 2;                  // PAR
  b += lt;                      // DRV
  return (b + 15) & ~(size_t)15;
}

__global__ void k_dfs(MatchArgs a) {
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
  uint8_t *DRV = reinterpret_cast<uint8_t *>(PAR + (size_t)NL * T);

  if (warp_read(&st->err)) return;
  const uint64_t nitems = min(*(volatile uint64_t *)&st->nitems, a.item_cap);
  int cur_plan = -1;

  while (true) {
    uint64_t it = 0;
    if (lane == 0) it = atomicAdd((unsigned long long *)&st->next_item, 1ull);
    it = __shfl_sync(GM_FULL, it, 0);
    if (it >= nitems) break;
    if (warp_read(&st->abort)) break;
    const WorkItem w = a.items[it];
    if ((int)w.plan != cur_plan) {
      const uint32_t *src = reinterpret_cast<const uint32_t *>(a.plans + w.plan);
      uint32_t *dst = reinterpret_cast<uint32_t *>(&H->plan);
      for (int i = lane; i < (int)(sizeof(Plan) / 4); i += 32) dst[i] = __ldg(src + i);
      cur_plan = w.plan;
    }
    if (lane < GM_MAXQ) H->cnt[lane] = 0;
    __syncwarp();
    const Plan &P = H->plan;
    const int q = P.q, last = q - 1;
    const uint32_t upd = w.upd;
    const uint32_t m0 = __ldg(a.cu + upd), m1 = __ldg(a.cv + upd);
    const uint32_t sdel = a.op[upd] < 0 ? 1u : 0u;
    uint64_t wcount = 0;
    uint64_t lbytes = 0;  // this lane's algorithmic bytes (only reported with count_bytes)
    uint32_t chunks = 0;
    int lev = -1;            // parent level (-1 = the seed itself)
    uint32_t root_cur = 0;

    // prepare level L (position L+2): driver segment of every entry for position L+3
    auto prepare = [&](int L) {
      const int p = L + 2, np = p + 1;
      const uint16_t bw = P.bwd[np];
      const int lab = P.lab[np];
      const uint32_t n = H->cnt[L];
      uint32_t carry = 0;
      for (uint32_t base = 0; base < n; base += 32) {
        uint32_t i = base + lane;
        uint32_t len = 0, lo = 0;
        int drv = 0;
        if (i < n) {
          // walk the chain of entry i, keep the backward neighbour with the
          // smallest label-lab count (driver choice only; exact bounds below)
          uint32_t best = 0xffffffffu, bestv = 0;
          uint32_t e = i;
          for (int l2 = L; l2 >= 0; l2--) {
            int pos = l2 + 2;
            uint32_t vv = V[l2 * T + e];
            if ((bw >> pos) & 1) {
              uint32_t c = __ldg(g.nlf + (size_t)vv * g.nlfw + lab);
              if (c < best) { best = c; bestv = vv; drv = pos; }
            }
            e = PAR[l2 * T + e];
          }
          if ((bw >> 1) & 1) {
            uint32_t c = __ldg(g.nlf + (size_t)m1 * g.nlfw + lab);
            if (c < best) { best = c; bestv = m1; drv = 1; }
          }
          if (bw & 1) {
            uint32_t c = __ldg(g.nlf + (size_t)m0 * g.nlfw + lab);
            if (c < best) { best = c; bestv = m0; drv = 0; }
          }
          lbytes += 4u * __popc(bw);
          if (best > 0) {
            uint2 ad = __ldg(reinterpret_cast<const uint2 *>(g.adj) + bestv);
            uint32_t slo, shi;
            seg_bounds(g, g.col + ad.x, ad.y, lab, slo, shi);
            lbytes += 2u * probe_bytes(ad.y);
            lo = ad.x + slo;
            len = shi - slo;
          }
          LO[L * T + i] = lo;
          DRV[L * T + i] = (uint8_t)drv;
        }
        uint32_t inc = len;
        for (int d = 1; d < 32; d <<= 1) {
          uint32_t y = __shfl_up_sync(GM_FULL, inc, d);
          if (lane >= d) inc += y;
        }
        if (i < n) EX[L * T + i] = carry + inc - len;
        carry += __shfl_sync(GM_FULL, inc, 31);
      }
      if (lane == 0) { H->tot[L] = carry; H->cur[L] = 0; }
      __syncwarp();
    };

    while (true) {
      const int c = lev + 3;  // position of the candidates produced from level lev
      uint32_t total, cur;
      if (lev < 0) { total = w.len; cur = root_cur; }
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
      if (stored && H->cnt[lev + 1] + 32 > (uint32_t)T) {
        prepare(lev + 1);
        lev++;
        continue;
      }
      // ---- one 32-wide expansion step
      const uint32_t gidx = cur + lane;
      bool ok = gidx < total;
      uint32_t e = 0, slot = 0;
      int drv;
      if (lev < 0) {
        slot = w.lo + gidx;
        drv = w.drv;
      } else {
        const uint32_t n = H->cnt[lev];
        const uint32_t *ex = EX + lev * T;
        uint32_t lo = 0, hi = n;  // last entry with ex <= gidx
        while (hi - lo > 1) {
          uint32_t mid = (lo + hi) >> 1;
          if (ex[mid] <= gidx) lo = mid; else hi = mid;
        }
        e = lo;
        slot = LO[lev * T + e] + (gidx - ex[e]);
        drv = DRV[lev * T + e];
      }
      chunks++;
      uint32_t x = ok ? __ldg(g.col + slot) : 0u;
      const uint32_t id = (x >> 1) & g.idmask;
      if (ok && (x & 1u)) ok = tag_ok(__ldg(g.etag + slot), sdel, upd);
      const uint16_t chk_edge = P.bwd[c] & (uint16_t)~(1u << drv);
      const uint16_t chk_neq = P.samelab[c];
      if (ok && (chk_edge | chk_neq)) {
        uint32_t ee = e;
        for (int l2 = lev; l2 >= 0 && ok; l2--) {
          const int pos = l2 + 2;
          const uint32_t vv = V[l2 * T + ee];
          if ((chk_neq >> pos) & 1) ok = (vv != id);
          if (ok && ((chk_edge >> pos) & 1)) ok = edge_ok(g, vv, x, sdel, upd, lbytes);
          ee = PAR[l2 * T + ee];
        }
        if (ok && ((chk_neq >> 1) & 1)) ok = (m1 != id);
        if (ok && ((chk_edge >> 1) & 1)) ok = edge_ok(g, m1, x, sdel, upd, lbytes);
        if (ok && (chk_neq & 1)) ok = (m0 != id);
        if (ok && (chk_edge & 1)) ok = edge_ok(g, m0, x, sdel, upd, lbytes);
      }
      if (ok && stored && a.use_filter) ok = nlf_ok(g, id, P, c);
      if (gidx < total) lbytes += ((x & 1u) ? 8u : 4u) + (ok ? 8u : 0u);
      const unsigned mask = __ballot_sync(GM_FULL, ok);
      if (!stored) {
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
      if ((chunks & 1023u) == 0 && warp_read(&st->abort)) break;
    }
    if (a.count_bytes) {
      lbytes += (lane == 0) ? sizeof(WorkItem) : 0;
      for (int d = 16; d > 0; d >>= 1) lbytes += __shfl_down_sync(GM_FULL, lbytes, d);
      if (lane == 0) atomicAdd((unsigned long long *)&st->alg_bytes, (unsigned long long)lbytes);
    }
    if (lane == 0) {
      if (wcount) {
        atomicAdd((unsigned long long *)&a.cnt[P.qslot * 2 + sdel], (unsigned long long)wcount);
        if (a.per_upd)
          atomicAdd((unsigned long long *)&a.per_upd[(uint64_t)P.qslot * a.b + upd], (unsigned long long)wcount);
      }
      unsigned long long ex = atomicAdd((unsigned long long *)&st->expansions, (unsigned long long)chunks);
      if (a.budget && ex + chunks > a.budget) {
        atomicExch(&st->abort, 1);
        gm_set_err(st, GAMMA_ETIMEOUT);
      }
    }
    __syncwarp();
  }
}

}  // namespace

size_t gm_dfs_smem_per_warp(int tile, int nlev) { return smem_per_warp(tile, nlev); }

int gm_seed(const MatchArgs &a, cudaStream_t s) {
  if (a.b <= 0 || a.nplans <= 0) return GAMMA_OK;
  int threads = 256;
  int64_t blocks = (a.b + threads - 1) / threads;
  if (blocks > 65536) blocks = 65536;
  k_seed<<<(int)blocks, threads, 0, s>>>(a);
  GM_LAUNCHED();
  GM_CUDA(cudaGetLastError());
  return GAMMA_OK;
}

int gm_dfs(const MatchArgs &a, int num_sms, cudaStream_t s) {
  const int wpb = a.warps_per_block;
  const size_t smem = smem_per_warp(a.tile, a.nlev) * wpb;
  static size_t configured = 0;
  if (smem > 48 * 1024 && smem > configured) {
    GM_CUDA(cudaFuncSetAttribute(k_dfs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured = smem;
  }
  int per_sm = 0;
  GM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfs, wpb * 32, smem));
  if (per_sm < 1) return GAMMA_EINVAL;
  k_dfs<<<num_sms * per_sm, wpb * 32, smem, s>>>(a);
  GM_LAUNCHED();
  GM_CUDA(cudaGetLastError());
  return GAMMA_OK;
}
