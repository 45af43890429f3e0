// gm_graph.cu -- the device-resident dynamic CSR: bulk load, batch staging
// (validate the batch, merge insertions into the sorted lists, tag
// deletions), commit (drop deleted entries, clear tags) and the per-label
// neighbour counts of the union graph G u G' used by the candidate filter
// (the neighbourhood-label-frequency test of Sec. IV-B, as counts).
//
// Lists keep slack (cap >= len); a list that outgrows its slot is moved to a
// fresh slot at the top of the pool.  The graph update of the paper is a GPMA
// (Sec. V-C); here each touched list is rewritten by one warp with a
// merge-path merge, in place from the back when it fits.
#include "gm_graph.cuh"

namespace {

// lower bound that reads through the coherent path (lists change in-kernel)
__device__ __forceinline__ uint32_t lb_coherent(const uint32_t *a, uint32_t len, uint32_t key) {
  uint32_t lo = 0, hi = len;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint32_t slack_cap(uint32_t len) {
  if (len == 0) return 0;
  uint32_t s = len / 4;
  if (s < 4) s = 4;
  return (len + s + 3u) & ~3u;
}

// ------------------------------- load ---------------------------------------
__global__ void k_load_validate(const int32_t *__restrict__ labels, int32_t n,
                                const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                                const int32_t *__restrict__ elabels, int64_t m, GmStatus *st) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)n || i < m; i += stride) {
    if (i < n) {
      int32_t l = labels[i];
      if (l < 0) { gm_set_err(st, GAMMA_EINVAL); }
      else atomicMax(&st->max_label, (uint32_t)l);
    }
    if (i < m) {
      int32_t s = src[i], d = dst[i];
      const bool bad_label = elabels && (elabels[i] < 0 || elabels[i] > 255);
      if (s < 0 || s >= n || d < 0 || d >= n || s == d || bad_label) {
        gm_set_err(st, GAMMA_EINVAL);
        gm_bad_index(st, i);
      }
    }
  }
}

// vals (edge-labelled graphs, else null): each directed entry carries its edge's label through the sort
__global__ void k_load_keys(const int32_t *__restrict__ src, const int32_t *__restrict__ dst,
                            const int32_t *__restrict__ elabels, int64_t m, const int32_t *__restrict__ label, int idb,
                            uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    uint32_t s = (uint32_t)src[e], d = (uint32_t)dst[e];
    keys[2 * e] = ((uint64_t)s << 32) | gm_key(label[d], d, idb);
    keys[2 * e + 1] = ((uint64_t)d << 32) | gm_key(label[s], s, idb);
    if (vals) vals[2 * e] = vals[2 * e + 1] = (uint32_t)elabels[e];
  }
}

// a repeated edge is merged; with edge labels its copies must agree
__global__ void k_load_uniq(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t n2,
                            uint32_t *__restrict__ flag, uint32_t *__restrict__ deg, GmStatus *st) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
    uint64_t k = keys[i];
    uint32_t f = (i == 0 || keys[i - 1] != k) ? 1u : 0u;
    if (!f && vals && vals[i - 1] != vals[i]) gm_set_err(st, GAMMA_EINVAL);
    flag[i] = f;
    if (f) atomicAdd(&deg[k >> 32], 1u);
  }
}

__global__ void k_load_caps(const uint32_t *__restrict__ deg, int32_t n, uint32_t *__restrict__ cap) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) cap[v] = slack_cap(deg[v]);
}

__global__ void k_load_scatter(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t n2,
                               const uint32_t *__restrict__ flag, const uint32_t *__restrict__ pos,
                               const uint32_t *__restrict__ rowstart, const uint32_t *__restrict__ off,
                               uint32_t *__restrict__ col, uint8_t *__restrict__ elab) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
    if (!flag[i]) continue;
    uint64_t k = keys[i];
    uint32_t s = (uint32_t)(k >> 32);
    const uint32_t slot = off[s] + pos[i] - rowstart[s];
    col[slot] = (uint32_t)k;
    if (elab) elab[slot] = (uint8_t)vals[i];
  }
}

__global__ void k_load_adj(const uint32_t *__restrict__ off, const uint32_t *__restrict__ deg,
                           const uint32_t *__restrict__ cap, int32_t n, uint2 *__restrict__ adj, GmStatus *st) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    adj[v] = make_uint2(off[v], deg[v]);
    if (v == n - 1) st->pool_top = off[v] + cap[v];
  }
}

// per-label neighbour counts: one warp per vertex, lane l finds where label
// l0 + l starts in the sorted list; counts are differences of those starts.
__global__ void k_nlf(GraphDev g, const uint32_t *__restrict__ verts, const uint32_t *__restrict__ nverts_dev,
                      uint32_t nverts) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  uint32_t nv = nverts_dev ? *nverts_dev : nverts;
  const int s = g.idb + 1;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nv; w += nw) {
    uint32_t v = verts ? verts[w] : (uint32_t)w;
    uint2 a = g.adj[v];
    const uint32_t *L = g.col + a.x;
    for (int l0 = 0; l0 < g.nlab; l0 += 31) {
      int l = l0 + lane;
      uint32_t bnd = (l >= g.nlab) ? a.y : lb_coherent(L, a.y, (uint32_t)l << s);
      uint32_t nb = __shfl_down_sync(GM_FULL, bnd, 1);
      if (lane < 31 && l < g.nlab) {
        uint32_t c = nb - bnd;
        g.nlf[(size_t)v * g.nlfw + l] = (uint8_t)(c > 255u ? 255u : c);
      }
    }
  }
}

// hub index rebuild: one warp per listed vertex that is a hub.  Label-segment
// starts come from lower bounds (lane l -> label l); the hash set is cleared
// and refilled from the list, moving to a larger slot range (from the hub
// pool) when the list outgrew half of the table; if the pool is exhausted the
// vertex keeps no table and lookups fall back to binary search.
__global__ void k_hub(GraphDev g, const uint32_t *__restrict__ verts, const uint32_t *__restrict__ nverts_dev,
                      uint32_t nverts, GmStatus *st) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const uint32_t nv = nverts_dev ? *nverts_dev : nverts;
  const int s = g.idb + 1;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nv; w += nw) {
    const uint32_t v = verts ? verts[w] : (uint32_t)w;
    const int32_t h = g.hub_id[v];
    if (h < 0) continue;
    const uint2 a = g.adj[v];
    const uint32_t *L = g.col + a.x;
    uint32_t *lofs = g.hub_lofs + (size_t)h * (g.nlab + 1);
    for (int l0 = 0; l0 <= g.nlab; l0 += 32) {
      int l = l0 + lane;
      if (l <= g.nlab) lofs[l] = (l >= g.nlab) ? a.y : lb_coherent(L, a.y, (uint32_t)l << s);
    }
    if (g.hub_keys == nullptr) continue;
    uint2 t = g.hub_tab[v];
    uint32_t cap = t.y ? (1u << t.y) : 0u;
    if (2ull * a.y + 2 > cap) {
      uint32_t bits = 3;
      while ((1ull << bits) < 3ull * a.y + 8) bits++;
      uint32_t off = 0;
      int ok = 0;
      if (lane == 0) {
        off = atomicAdd(&st->hub_top, 1u << bits);
        ok = (uint64_t)off + (1ull << bits) <= g.hub_keys_cap;
      }
      off = __shfl_sync(GM_FULL, off, 0);
      ok = __shfl_sync(GM_FULL, ok, 0);
      t = ok ? make_uint2(off, bits) : make_uint2(0, 0);
      if (lane == 0) g.hub_tab[v] = t;
      cap = t.y ? (1u << t.y) : 0u;
    }
    if (!cap) continue;
    uint32_t *T = g.hub_keys + t.x;
    for (uint32_t i = lane; i < cap; i += 32) T[i] = GM_EMPTY;
    __syncwarp();
    const uint32_t mask = cap - 1;
    for (uint32_t i = lane; i < a.y; i += 32) {
      const uint32_t key = L[i];
      uint32_t p = gm_hash(key >> 1) & mask;
      for (uint32_t probe = 0; probe < cap; probe++) {
        if (atomicCAS(T + p, GM_EMPTY, key) == GM_EMPTY) break;
        p = (p + 1) & mask;
      }
    }
    __syncwarp();
  }
}

// ------------------------------- request chains -----------------------------
// Several requests staged together may touch the same edge: request r sees
// the graph the requests before it leave.  The updates of one edge, in index
// order, form a chain; a valid chain alternates insertion and deletion and
// holds at most one update per request (its head must also agree with G,
// which the stage checks like any single update).

// edge key (u << idb | v) of every update, with the first checks of an update
// on its own; an invalid update gets the key ~0 (it sorts last)
__global__ void k_chain_keys(const int8_t *__restrict__ op, const int32_t *__restrict__ src,
                             const int32_t *__restrict__ dst, int64_t b, GraphDev g, uint64_t *__restrict__ keys,
                             uint32_t *__restrict__ idx, GmStatus *st) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < b; k += stride) {
    const int o = op[k];
    const int32_t s = src[k], d = dst[k];
    const bool bad = (o != 1 && o != -1) || s < 0 || s >= g.n || d < 0 || d >= g.n || s == d;
    if (bad) {
      gm_set_err(st, GAMMA_EINVAL);
      gm_bad_index(st, k);
    }
    const uint64_t u = (uint64_t)min(s, d), v = (uint64_t)max(s, d);
    keys[k] = bad ? ~0ull : ((u << g.idb) | v);
    idx[k] = (uint32_t)k;
  }
}

// after the stable sort by edge key: link each update to the next one of the
// same edge, mark heads, check the chains, and record at each head whether
// the edge exists once the whole chain is applied
__global__ void k_chain_link(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ idx, int64_t b,
                             const int8_t *__restrict__ op, const uint32_t *__restrict__ req,
                             uint32_t *__restrict__ cnext, uint8_t *__restrict__ cinfo, GmStatus *st) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < b; j += stride) {
    const uint64_t key = keys[j];
    const uint32_t k = idx[j];
    if (key == ~0ull) {  // invalid on its own (already reported)
      cnext[k] = ~0u;
      cinfo[k] = GM_CHAIN_HEAD;
      continue;
    }
    const bool has_prev = j > 0 && keys[j - 1] == key;
    const bool has_next = j + 1 < b && keys[j + 1] == key;
    cnext[k] = has_next ? idx[j + 1] : ~0u;
    if (has_prev) {
      const uint32_t kp = idx[j - 1];
      if (op[kp] == op[k] || req[kp] == req[k]) {  // not alternating, or one request touches the edge twice
        gm_set_err(st, GAMMA_EINVAL);
        gm_bad_index(st, (int64_t)k);
      }
      cinfo[k] = 0;
      continue;
    }
    int64_t e = j;
    while (e + 1 < b && keys[e + 1] == key) e++;  // chains are short: one update per request at most
    uint8_t info = GM_CHAIN_HEAD;
    if (e > j) info |= GM_CHAIN_LONG;
    if (op[idx[e]] > 0) info |= GM_CHAIN_PRESENT;
    cinfo[k] = info;
  }
}

// at commit: a chain's head entry carries the head's tag; turn its deletion
// bit into "absent after the whole chain" so the commit keeps or drops the
// edge by the chain's last update
__global__ void k_chain_final(GraphDev g, const uint32_t *__restrict__ cu, const uint32_t *__restrict__ cv, int64_t b,
                              const uint8_t *__restrict__ cinfo) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < b; k += stride) {
    const uint8_t info = cinfo[k];
    if (!(info & GM_CHAIN_LONG)) continue;
    const uint32_t gone = (info & GM_CHAIN_PRESENT) ? 0u : 1u;
    for (int side = 0; side < 2; side++) {
      const uint32_t v = side ? cv[k] : cu[k], w = side ? cu[k] : cv[k];
      const uint2 a = g.adj[v];
      const uint32_t k32 = gm_key(g.label[w], w, g.idb);
      const uint32_t p = lb_coherent(g.col + a.x, a.y, k32);
      if (p < a.y && (g.col[a.x + p] >> 1) == (k32 >> 1)) g.etag[a.x + p] = (g.etag[a.x + p] & ~1u) | gone;
    }
  }
}

// ------------------------------- stage --------------------------------------
// sort key: (vertex << 33) | (deletion << 32) | adjacency key with flag set,
// so a vertex's group lists its insertions (sorted) before its deletions.
// cinfo (chains of several requests, else null): an update that is not the
// head of its edge's chain enters no list; its entries get the key ~0
__global__ void k_stage_prep(const int8_t *__restrict__ op, const int32_t *__restrict__ src,
                             const int32_t *__restrict__ dst, int64_t b, GraphDev g,
                             uint32_t *__restrict__ cu, uint32_t *__restrict__ cv, int8_t *__restrict__ cop,
                             uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
                             const uint8_t *__restrict__ cinfo, const int32_t *__restrict__ elab_in,
                             uint8_t *__restrict__ ulab, GmStatus *st) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < b; k += stride) {
    int o = op[k];
    int32_t s = src[k], d = dst[k];
    // edge-labelled graph: an insertion's label (a deletion's is read while merging)
    const int32_t el = (g.elab && elab_in && o == 1) ? elab_in[k] : 0;
    if (g.elab) ulab[k] = (uint8_t)el;
    bool bad = (o != 1 && o != -1) || s < 0 || s >= g.n || d < 0 || d >= g.n || s == d || el < 0 || el > 255;
    if (bad) {
      gm_set_err(st, GAMMA_EINVAL);
      gm_bad_index(st, k);
      keys[2 * k] = keys[2 * k + 1] = ~0ull;
      vals[2 * k] = vals[2 * k + 1] = 0;
      cu[k] = cv[k] = 0;
      cop[k] = 1;
      continue;
    }
    uint32_t u = (uint32_t)min(s, d), v = (uint32_t)max(s, d);
    uint64_t del = (o < 0) ? 1ull : 0ull;
    cu[k] = u; cv[k] = v; cop[k] = (int8_t)o;
    if (cinfo && !(cinfo[k] & GM_CHAIN_HEAD)) {
      keys[2 * k] = keys[2 * k + 1] = ~0ull;
      vals[2 * k] = vals[2 * k + 1] = 0;
      continue;
    }
    keys[2 * k] = ((uint64_t)u << 33) | (del << 32) | gm_key(g.label[v], v, g.idb) | 1u;
    keys[2 * k + 1] = ((uint64_t)v << 33) | (del << 32) | gm_key(g.label[u], u, g.idb) | 1u;
    uint32_t val = ((uint32_t)k << 1) | (uint32_t)del;
    vals[2 * k] = val; vals[2 * k + 1] = val;
  }
}

// after the sort: duplicate and existence checks, group heads
__global__ void k_stage_check(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t n2,
                              GraphDev g, uint32_t *__restrict__ head, GmStatus *st) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n2; j += stride) {
    uint64_t key = keys[j];
    if (key == ~0ull) { head[j] = 0; continue; }
    uint32_t vtx = (uint32_t)(key >> 33);
    uint32_t h = (j == 0 || (keys[j - 1] >> 33) != vtx) ? 1u : 0u;
    head[j] = h;
    uint32_t k = vals[j] >> 1;
    bool del = (key >> 32) & 1ull;
    if (j > 0 && (keys[j - 1] >> 1) == (key >> 1)) {  // same edge, same op, twice
      uint32_t kp = vals[j - 1] >> 1;
      gm_set_err(st, GAMMA_EINVAL);
      gm_bad_index(st, (int64_t)max(k, kp));
    }
    uint32_t k32 = (uint32_t)key & ~1u;
    uint32_t other = (k32 >> 1) & g.idmask;
    if (vtx < other) {  // check each undirected edge once
      uint2 a = g.adj[vtx];
      const uint32_t *L = g.col + a.x;
      uint32_t p = lb_coherent(L, a.y, k32);
      bool found = p < a.y && (L[p] >> 1) == (k32 >> 1);
      if (found != del) {
        gm_set_err(st, GAMMA_EINVAL);
        gm_bad_index(st, (int64_t)k);
      }
    }
  }
}

__global__ void k_stage_groups(const uint64_t *__restrict__ keys, int64_t n2, const uint32_t *__restrict__ head,
                               const uint32_t *__restrict__ gid, uint32_t *__restrict__ gv,
                               uint32_t *__restrict__ gstart, uint32_t *__restrict__ gins, GmStatus *st) {
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n2; j += stride) {
    uint64_t key = keys[j];
    if (j == n2 - 1) st->ntouched = gid[j] + head[j];
    if (key == ~0ull) continue;
    if (j == n2 - 1 || keys[j + 1] == ~0ull) st->n2_valid = (uint32_t)(j + 1);  // unused entries sort last
    uint32_t gi = gid[j] + head[j] - 1;  // gid is the exclusive scan of the head flags
    if (head[j]) { gv[gi] = (uint32_t)(key >> 33); gstart[gi] = (uint32_t)j; }
    if (!((key >> 32) & 1ull)) atomicAdd(&gins[gi], 1u);
  }
}

__global__ void k_stage_plan(GraphDev g, const uint32_t *__restrict__ gv, const uint32_t *__restrict__ gins,
                             uint32_t *__restrict__ greloc, GmStatus *st) {
  uint32_t nt = st->ntouched;
  uint64_t local = 0;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nt; i += stride) {
    uint32_t v = gv[i];
    uint32_t nl = g.adj[v].y + gins[i];
    uint32_t r = 0;
    if (nl > g.cap[v]) r = slack_cap(nl);
    greloc[i] = r;
    local += r;
  }
  for (int d = 16; d > 0; d >>= 1) local += __shfl_down_sync(GM_FULL, local, d);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd((unsigned long long *)&st->reloc_total, (unsigned long long)local);
}

__global__ void k_stage_alloc(GraphDev g, GmStatus *st) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    if (st->err == 0 && (uint64_t)st->pool_top + st->reloc_total > (uint64_t)g.pool_cap)
      gm_set_err(st, GAMMA_ENOMEM);
  }
}

// number of A elements among the first `diag` outputs of merge(A, B)
__device__ __forceinline__ uint32_t merge_path(const uint32_t *A, uint32_t na, const uint32_t *B, uint32_t nb,
                                               uint32_t diag) {
  uint32_t lo = diag > nb ? diag - nb : 0, hi = diag < na ? diag : na;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (A[mid] < B[diag - 1 - mid]) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// one warp per touched vertex: merge the sorted insertions into the list
// (backwards in place, or forwards into a new slot), then tag the deletions.
__global__ void k_stage_merge(GraphDev g, const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                              int64_t n2, const uint32_t *__restrict__ gv, const uint32_t *__restrict__ gstart,
                              const uint32_t *__restrict__ gins, const uint32_t *__restrict__ greloc,
                              uint32_t *__restrict__ bkeys, uint8_t *__restrict__ ulab, GmStatus *st) {
  if (*(volatile int32_t *)&st->err) return;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const uint32_t nt = st->ntouched;
  for (int64_t gi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; gi < nt; gi += nw) {
    const uint32_t v = gv[gi];
    const uint32_t start = gstart[gi];
    const uint32_t end = (gi + 1 < nt) ? gstart[gi + 1] : st->n2_valid;
    const uint32_t ni = gins[gi];
    const uint2 a = g.adj[v];
    const uint32_t na = a.y, tot = na + ni;
    // insertion keys of this group as a contiguous array
    uint32_t *B = bkeys + start;
    for (uint32_t i = lane; i < ni; i += 32) B[i] = (uint32_t)keys[start + i];
    __syncwarp();
    uint32_t off = a.x;
    const uint32_t *A = g.col + a.x;
    uint32_t r = greloc[gi];
    if (r) {
      uint32_t no = 0;
      if (lane == 0) {
        no = atomicAdd(&st->pool_top, r);
        atomicAdd((unsigned long long *)&st->garbage, (unsigned long long)g.cap[v]);
        g.cap[v] = r;
      }
      off = __shfl_sync(GM_FULL, no, 0);
      uint32_t *O = g.col + off;
      for (uint32_t base = 0; base < tot; base += 32) {
        uint32_t d = base + lane;
        if (d < tot) {
          uint32_t i = merge_path(A, na, B, ni, d), j = d - i;
          if (i < na && (j >= ni || A[i] < B[j])) {
            O[d] = A[i];
            if (g.elab) g.elab[off + d] = g.elab[a.x + i];
          } else {
            O[d] = B[j];
            g.etag[off + d] = vals[start + j];
            if (g.elab) g.elab[off + d] = ulab[vals[start + j] >> 1];
          }
        }
      }
    } else if (ni) {
      uint32_t *O = g.col + off;
      for (uint32_t base = 0; base < tot; base += 32) {
        // outputs tot-1-base-lane, descending: read everything, then write
        int64_t dd = (int64_t)tot - 1 - base - lane;
        bool act = dd >= 0;
        uint32_t val = 0, tag = 0;
        uint8_t lab = 0;
        bool fromB = false;
        if (act) {
          uint32_t d = (uint32_t)dd;
          uint32_t i = merge_path(A, na, B, ni, d), j = d - i;
          if (i < na && (j >= ni || A[i] < B[j])) {
            val = A[i];
            if (g.elab) lab = g.elab[a.x + i];
          } else {
            val = B[j]; tag = vals[start + j]; fromB = true;
            if (g.elab) lab = ulab[tag >> 1];
          }
        }
        __syncwarp();
        if (act) {
          O[dd] = val;
          if (fromB) g.etag[off + dd] = tag;
          if (g.elab) g.elab[off + dd] = lab;
        }
        __syncwarp();
      }
    }
    __syncwarp();
    // tag deletions in the merged list
    const uint32_t *L = g.col + off;
    for (uint32_t j = start + ni + lane; j < end; j += 32) {
      uint32_t k32 = (uint32_t)keys[j] & ~1u;
      uint32_t p = lb_coherent(L, tot, k32);
      if (p < tot && (L[p] >> 1) == (k32 >> 1)) {  // always true for a validated batch
        g.col[off + p] = k32 | 1u;
        g.etag[off + p] = vals[j];
        if (g.elab) ulab[vals[j] >> 1] = g.elab[off + p];  // the deleted edge's label
      }
    }
    __syncwarp();
    if (lane == 0) {
      g.adj[v] = make_uint2(off, tot);
      g.vgroup[v] = (int32_t)gi;
    }
  }
}

// ------------------------------- commit -------------------------------------
__global__ void k_commit(GraphDev g, const uint32_t *__restrict__ gv, const uint32_t *__restrict__ gins,
                         GmStatus *st) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const uint32_t nt = st->ntouched;
  for (int64_t gi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; gi < nt; gi += nw) {
    const uint32_t v = gv[gi];
    const uint2 a = g.adj[v];
    uint32_t *L = g.col + a.x;
    uint32_t out = 0;
    for (uint32_t base = 0; base < a.y; base += 32) {
      uint32_t i = base + lane;
      uint32_t e = 0;
      uint8_t lab = 0;
      bool keep = false;
      if (i < a.y) {
        e = L[i];
        keep = !((e & 1u) && (g.etag[a.x + i] & 1u));
        if (g.elab) lab = g.elab[a.x + i];
      }
      unsigned mask = __ballot_sync(GM_FULL, keep);
      __syncwarp();
      if (keep) {
        const uint32_t to = out + __popc(mask & ((1u << lane) - 1u));
        L[to] = e & ~1u;
        if (g.elab) g.elab[a.x + to] = lab;
      }
      out += __popc(mask);
      __syncwarp();
    }
    if (lane == 0) {
      g.adj[v] = make_uint2(a.x, out);
      g.vgroup[v] = -1;
      // change of this list's committed length: insertions - deletions
      int64_t delta = (int64_t)gins[gi] - (int64_t)(a.y - out);
      if (delta) atomicAdd((unsigned long long *)&st->live, (unsigned long long)delta);
    }
  }
}

__global__ void k_begin_group(GmStatus *st) {
  if (threadIdx.x == 0 && blockIdx.x == 0) st->next_item = st->nitems;
}

inline int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 1 << 20) b = 1 << 20;
  return (int)b;
}

}  // namespace

// --------------------------------------------------------------------------
// host wrappers
// --------------------------------------------------------------------------
int gm_load_validate(const int32_t *labels, int32_t n, const int32_t *src, const int32_t *dst,
                     const int32_t *elabels, int64_t m, GmStatus *st, cudaStream_t s) {
  k_load_validate<<<grid_for(n > m ? n : m, 256), 256, 0, s>>>(labels, n, src, dst, elabels, m, st);
  GM_LAUNCHED();
  GM_CUDA(cudaGetLastError());
  return GAMMA_OK;
}

int gm_load_build(GraphDev g, const int32_t *src, const int32_t *dst, const int32_t *elabels, int64_t m,
                  uint32_t **col_out, uint32_t **etag_out, uint8_t **elab_out, uint32_t *pool_cap_out,
                  double pool_factor, uint64_t pool_reserve, GmStatus *st, GmStatus *h_st, cudaStream_t s) {
  const int64_t n2 = 2 * m;
  uint64_t *keys = nullptr, *tk = nullptr;
  uint32_t *flag = nullptr, *pos = nullptr, *deg = nullptr, *rowstart = nullptr, *off = nullptr;
  uint32_t *vals = nullptr, *tv = nullptr;  // edge labels riding with the keys (labelled graphs)
  if (elabels) {
    GM_CUDA(cudaMallocAsync((void **)&vals, sizeof(uint32_t) * (n2 + 1), s));
    GM_CUDA(cudaMallocAsync((void **)&tv, sizeof(uint32_t) * (n2 + 1), s));
  }
  GM_CUDA(cudaMallocAsync((void **)&keys, sizeof(uint64_t) * (n2 + 1), s));
  GM_CUDA(cudaMallocAsync((void **)&tk, sizeof(uint64_t) * (n2 + 1), s));
  GM_CUDA(cudaMallocAsync((void **)&flag, sizeof(uint32_t) * (n2 + 1), s));
  GM_CUDA(cudaMallocAsync((void **)&pos, sizeof(uint32_t) * (n2 + 1), s));
  GM_CUDA(cudaMallocAsync((void **)&deg, sizeof(uint32_t) * (g.n + 1), s));
  GM_CUDA(cudaMallocAsync((void **)&rowstart, sizeof(uint32_t) * (g.n + 1), s));
  GM_CUDA(cudaMallocAsync((void **)&off, sizeof(uint32_t) * (g.n + 1), s));
  GM_CUDA(cudaMemsetAsync(deg, 0, sizeof(uint32_t) * (g.n + 1), s));
  if (m > 0) {
    k_load_keys<<<grid_for(m, 256), 256, 0, s>>>(src, dst, elabels, m, g.label, g.idb, keys, vals);
    GM_LAUNCHED();
    GM_CUDA(cudaGetLastError());
    int rc = gm_radix_sort(keys, vals, tk, tv, n2, 1, 32 + g.idb, s);
    if (rc) return rc;
    k_load_uniq<<<grid_for(n2, 256), 256, 0, s>>>(keys, vals, n2, flag, deg, st);
    GM_LAUNCHED();
    GM_CUDA(cudaGetLastError());
    rc = gm_scan_excl_u32(flag, pos, n2, s);
    if (rc) return rc;
  }
  int rc = gm_scan_excl_u32(deg, rowstart, g.n, s);
  if (rc) return rc;
  k_load_caps<<<grid_for(g.n, 256), 256, 0, s>>>(deg, g.n, g.cap);
  GM_LAUNCHED();
  GM_CUDA(cudaGetLastError());
  rc = gm_scan_excl_u32(g.cap, off, g.n, s);
  if (rc) return rc;
  k_load_adj<<<grid_for(g.n, 256), 256, 0, s>>>(off, deg, g.cap, g.n, g.adj, st);
  GM_LAUNCHED();
  GM_CUDA(cudaGetLastError());
  GM_CUDA(cudaMemcpyAsync(h_st, st, sizeof(GmStatus), cudaMemcpyDeviceToHost, s));
  GM_CUDA(cudaStreamSynchronize(s));
  uint64_t used = h_st->pool_top;
  uint64_t cap = (uint64_t)(used * pool_factor) + pool_reserve + 64;
  if (cap >= (1ull << 32) - 64) return GAMMA_ENOMEM;
  uint32_t *col = nullptr, *etag = nullptr;
  uint8_t *elab = nullptr;
  GM_CUDA(cudaMalloc((void **)&col, sizeof(uint32_t) * (cap + GM_COL_PAD)));  // padded: short lists are read in 16-byte words
  GM_CUDA(cudaMalloc((void **)&etag, sizeof(uint32_t) * cap));
  if (elabels) GM_CUDA(cudaMalloc((void **)&elab, cap + GM_COL_PAD));
  if (m > 0) {
    k_load_scatter<<<grid_for(n2, 256), 256, 0, s>>>(keys, vals, n2, flag, pos, rowstart, off, col, elab);
    GM_LAUNCHED();
    GM_CUDA(cudaGetLastError());
  }
  GM_CUDA(cudaFreeAsync(keys, s));
  GM_CUDA(cudaFreeAsync(tk, s));
  GM_CUDA(cudaFreeAsync(flag, s));
  GM_CUDA(cudaFreeAsync(pos, s));
  GM_CUDA(cudaFreeAsync(deg, s));
  GM_CUDA(cudaFreeAsync(rowstart, s));
  GM_CUDA(cudaFreeAsync(off, s));
  if (vals) GM_CUDA(cudaFreeAsync(vals, s));
  if (tv) GM_CUDA(cudaFreeAsync(tv, s));
  *col_out = col;
  *etag_out = etag;
  *elab_out = elab;
  *pool_cap_out = (uint32_t)cap;
  return GAMMA_OK;
}

int gm_nlf(GraphDev g, const uint32_t *verts, const uint32_t *nverts_dev, uint32_t nverts_max, cudaStream_t s) {
  if (nverts_max == 0) return GAMMA_OK;
  int threads = 256;
  int64_t blocks = ((int64_t)nverts_max * 32 + threads - 1) / threads;
  if (blocks > 8192) blocks = 8192;
  k_nlf<<<(int)blocks, threads, 0, s>>>(g, verts, nverts_dev, nverts_max);
  GM_LAUNCHED();
  GM_CUDA(cudaGetLastError());
  return GAMMA_OK;
}

int gm_hub(GraphDev g, const uint32_t *verts, const uint32_t *nverts_dev, uint32_t nverts_max, GmStatus *st,
           cudaStream_t s) {
  if (nverts_max == 0 || g.nhub == 0) return GAMMA_OK;
  int threads = 256;
  int64_t blocks = ((int64_t)nverts_max * 32 + threads - 1) / threads;
  if (blocks > 8192) blocks = 8192;
  k_hub<<<(int)blocks, threads, 0, s>>>(g, verts, nverts_dev, nverts_max, st);
  GM_LAUNCHED();
  GM_CUDA(cudaGetLastError());
  return GAMMA_OK;
}

int gm_stage(GraphDev g, const int8_t *op, const int32_t *src, const int32_t *dst, const int32_t *elab_in, int64_t b,
             const uint32_t *req, StageBufs &sb, GmStatus *st, cudaStream_t s) {
  const int64_t n2 = 2 * b;
  int rc = GAMMA_OK;
  if (req) {  // chains of updates on one edge across requests (the sort buffers serve as scratch)
    k_chain_keys<<<grid_for(b, 256), 256, 0, s>>>(op, src, dst, b, g, sb.keys, sb.vals, st);
    GM_LAUNCHED();
    GM_CUDA(cudaGetLastError());
    rc = gm_radix_sort(sb.keys, sb.vals, sb.tk, sb.tv, b, 0, 2 * g.idb, s);
    if (rc) return rc;
    k_chain_link<<<grid_for(b, 256), 256, 0, s>>>(sb.keys, sb.vals, b, op, req, sb.cnext, sb.cinfo, st);
    GM_LAUNCHED();
    GM_CUDA(cudaGetLastError());
  }
  k_stage_prep<<<grid_for(b, 256), 256, 0, s>>>(op, src, dst, b, g, sb.cu, sb.cv, sb.cop, sb.keys, sb.vals,
                                                req ? sb.cinfo : nullptr, elab_in, sb.ulab, st);
  GM_LAUNCHED();
  GM_CUDA(cudaGetLastError());
  rc = gm_radix_sort(sb.keys, sb.vals, sb.tk, sb.tv, n2, 1, 33 + g.idb, s);
  if (rc) return rc;
  k_stage_check<<<grid_for(n2, 256), 256, 0, s>>>(sb.keys, sb.vals, n2, g, sb.head, st);
  GM_LAUNCHED();
  GM_CUDA(cudaGetLastError());
  rc = gm_scan_excl_u32(sb.head, sb.gid, n2, s);
  if (rc) return rc;
  GM_CUDA(cudaMemsetAsync(sb.gins, 0, sizeof(uint32_t) * n2, s));
  k_stage_groups<<<grid_for(n2, 256), 256, 0, s>>>(sb.keys, n2, sb.head, sb.gid, sb.gv, sb.gstart, sb.gins, st);
  GM_LAUNCHED();
  GM_CUDA(cudaGetLastError());
  k_stage_plan<<<grid_for(n2, 256), 256, 0, s>>>(g, sb.gv, sb.gins, sb.greloc, st);
  GM_LAUNCHED();
  GM_CUDA(cudaGetLastError());
  k_stage_alloc<<<1, 32, 0, s>>>(g, st);
  GM_LAUNCHED();
  GM_CUDA(cudaGetLastError());
  int64_t mb = (n2 * 32 + 255) / 256;
  if (mb > 16384) mb = 16384;
  if (mb < 1) mb = 1;
  k_stage_merge<<<(int)mb, 256, 0, s>>>(g, sb.keys, sb.vals, n2, sb.gv, sb.gstart, sb.gins, sb.greloc, sb.bkeys,
                                        sb.ulab, st);
  GM_LAUNCHED();
  GM_CUDA(cudaGetLastError());
  rc = gm_nlf(g, sb.gv, &st->ntouched, (uint32_t)n2, s);
  if (rc) return rc;
  return gm_hub(g, sb.gv, &st->ntouched, (uint32_t)n2, st, s);
}

int gm_commit(GraphDev g, const StageBufs &sb, int64_t b, bool chains, GmStatus *st, cudaStream_t s) {
  const int64_t n2 = 2 * b;
  if (chains) {
    k_chain_final<<<grid_for(b, 256), 256, 0, s>>>(g, sb.cu, sb.cv, b, sb.cinfo);
    GM_LAUNCHED();
    GM_CUDA(cudaGetLastError());
  }
  int64_t mb = (n2 * 32 + 255) / 256;
  if (mb > 16384) mb = 16384;
  if (mb < 1) mb = 1;
  k_commit<<<(int)mb, 256, 0, s>>>(g, sb.gv, sb.gins, st);
  GM_LAUNCHED();
  GM_CUDA(cudaGetLastError());
  int rc = gm_nlf(g, sb.gv, &st->ntouched, (uint32_t)n2, s);
  if (rc) return rc;
  return gm_hub(g, sb.gv, &st->ntouched, (uint32_t)n2, st, s);
}

int gm_begin_group(GmStatus *st, cudaStream_t s) {
  k_begin_group<<<1, 32, 0, s>>>(st);
  GM_LAUNCHED();
  GM_CUDA(cudaGetLastError());
  return GAMMA_OK;
}
