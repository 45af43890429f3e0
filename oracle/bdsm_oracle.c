/*
 * bdsm_oracle.c -- plain, slow, single-threaded CPU oracle for batch-dynamic
 * subgraph matching (BDSM).  TEST INFRASTRUCTURE ONLY: it exists to check the
 * CUDA path and is never part of it.  It shares no code with the library.
 *
 * What it computes (Sec. II-A, Def. 1 and Def. 2, Problem Statement):
 *   G' = (E(G) \ D) u I for a batch with insertions I and deletions D.
 *   An embedding (Def. 2) is an injective map phi: V(Q) -> V(G) with
 *   L(phi(u)) = L(u) for every query vertex and (phi(u), phi(u')) an edge for
 *   every query edge (non-induced).  The incremental matches are
 *     positive: Emb(Q, G') \ Emb(Q, G)   (embeddings using >= 1 inserted edge)
 *     negative: Emb(Q, G)  \ Emb(Q, G')  (embeddings using >= 1 deleted edge)
 *   and each one is charged to the lowest-indexed update of its own sign among
 *   the update edges that are images of query edges (Sec. IV-C, the total
 *   order over updates used to remove duplicates).
 *
 * How: for each update i (sign s, view V = G' if s = + else G), for each
 * query edge (a, b) and each of the two orientations of the undirected update
 * edge, fix phi(a), phi(b) to its endpoints when the labels agree, then
 * backtrack over the other query vertices in a fixed order in which every
 * vertex has an already-assigned query neighbour (the query is connected),
 * trying every V-neighbour carrying the vertex's label of the image of one
 * assigned query neighbour (the one whose image has the fewest such
 * neighbours; lists are sorted by label, then id).  A candidate
 * is kept when its label matches, it is not already used, and for EVERY query
 * edge to an assigned vertex the image edge is in V and is not an update of
 * sign s with index < i.  No filter, no encoding, no reordering: membership is
 * a hash-set lookup.
 *
 * Edge labels (Sec. II-A: the label function covers edges too): optional.
 * With them, an embedding must also map every query edge onto a data edge
 * of the same label; an inserted edge carries the label its update gives, a
 * deletion removes the edge whatever its label.  Without them every edge
 * has label 0.
 *
 * Batch validity (a reading: the paper is silent): a batch is rejected as a
 * whole when any update has an out-of-range id, a self-loop, an op other than
 * +1/-1, repeats an edge already in the batch, inserts an edge present in G
 * or deletes one absent from G.  The reported offender is the smallest index
 * k such that update k is invalid on its own or repeats an earlier update.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_EBUDGET (-2)
#define OR_ENOMEM (-3)

/* ---------------- open-addressing hash map: edge key -> int64 value ------ */
typedef struct {
  uint64_t *keys; /* 0 = empty; stored key = real key + 1 */
  int64_t *vals;
  uint64_t mask;
} hmap;

static uint64_t hmix(uint64_t z) {
  z ^= z >> 33; z *= 0xff51afd7ed558ccdULL;
  z ^= z >> 33; z *= 0xc4ceb9fe1a85ec53ULL;
  z ^= z >> 33; return z;
}

static int hmap_init(hmap *h, int64_t n) {
  uint64_t cap = 16;
  while (cap < (uint64_t)(2 * n + 16)) cap <<= 1;
  h->keys = (uint64_t *)calloc(cap, sizeof(uint64_t));
  h->vals = (int64_t *)malloc(cap * sizeof(int64_t));
  h->mask = cap - 1;
  return (h->keys && h->vals) ? 0 : -1;
}

static void hmap_free(hmap *h) { free(h->keys); free(h->vals); }

/* returns 1 if inserted, 0 if present (value untouched) */
static int hmap_put(hmap *h, uint64_t key, int64_t val) {
  uint64_t k = key + 1, i = hmix(k) & h->mask;
  while (h->keys[i]) {
    if (h->keys[i] == k) return 0;
    i = (i + 1) & h->mask;
  }
  h->keys[i] = k; h->vals[i] = val; return 1;
}

static int hmap_get(const hmap *h, uint64_t key, int64_t *val) {
  uint64_t k = key + 1, i = hmix(k) & h->mask;
  while (h->keys[i]) {
    if (h->keys[i] == k) { if (val) *val = h->vals[i]; return 1; }
    i = (i + 1) & h->mask;
  }
  return 0;
}

static uint64_t ekey(int32_t a, int32_t b) {
  uint32_t lo = (uint32_t)(a < b ? a : b), hi = (uint32_t)(a < b ? b : a);
  return ((uint64_t)lo << 32) | hi;
}

/* ---------------- adjacency lists (for iteration only) -------------------- */
/* Each vertex's neighbours are kept sorted by (label, id), so the neighbours
 * that carry one label form one run, found by two binary searches. */
typedef struct { int64_t *off; int32_t *nbr; const int32_t *lab; } adj;

static const int32_t *g_sort_lab; /* labels for the qsort comparator (single-threaded build) */

static int by_label_then_id(const void *x, const void *y) {
  const int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
  const int32_t la = g_sort_lab[a], lb = g_sort_lab[b];
  if (la != lb) return la < lb ? -1 : 1;
  return (a > b) - (a < b);
}

/* [*lo, *hi) = the run of x's neighbours with label lab */
static void label_run(const adj *A, int32_t x, int32_t lab, int64_t *lo, int64_t *hi) {
  int64_t a = A->off[x], b = A->off[x + 1];
  while (a < b) { /* first neighbour with label >= lab */
    int64_t m = a + (b - a) / 2;
    if (A->lab[A->nbr[m]] < lab) a = m + 1; else b = m;
  }
  *lo = a;
  b = A->off[x + 1];
  while (a < b) { /* first neighbour with label > lab */
    int64_t m = a + (b - a) / 2;
    if (A->lab[A->nbr[m]] <= lab) a = m + 1; else b = m;
  }
  *hi = a;
}

static int adj_build(adj *A, int32_t n, int64_t m, const int32_t *s, const int32_t *d, const int32_t *lab) {
  A->lab = lab;
  A->off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  A->nbr = (int32_t *)malloc((size_t)(2 * m + 1) * sizeof(int32_t));
  if (!A->off || !A->nbr) return -1;
  for (int64_t e = 0; e < m; e++) { A->off[s[e] + 1]++; A->off[d[e] + 1]++; }
  for (int32_t v = 0; v < n; v++) A->off[v + 1] += A->off[v];
  int64_t *fill = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!fill) return -1;
  memcpy(fill, A->off, ((size_t)n + 1) * sizeof(int64_t));
  for (int64_t e = 0; e < m; e++) {
    A->nbr[fill[s[e]]++] = d[e];
    A->nbr[fill[d[e]]++] = s[e];
  }
  free(fill);
  g_sort_lab = lab;
  for (int32_t v = 0; v < n; v++)
    qsort(A->nbr + A->off[v], (size_t)(A->off[v + 1] - A->off[v]), sizeof(int32_t), by_label_then_id);
  return 0;
}

static void adj_free(adj *A) { free(A->off); free(A->nbr); }

/* ---------------- search state --------------------------------------------- */
typedef struct {
  int32_t q;
  const int32_t *qlab;
  int32_t eq;
  const int32_t *qs, *qd;
  const int32_t *lab;
  const hmap *gset;   /* edges of G -> edge label */
  const hmap *bmap;   /* batch edge -> update index */
  const int32_t *qel; /* query edge labels (NULL: all 0) */
  const int32_t *uel; /* labels of inserted edges by update (NULL: all 0) */
  const int8_t *op;
  const adj *view;
  int sign;           /* +1 / -1 of the seeding update */
  int64_t upd;        /* index of the seeding update */
  int32_t order[32];  /* search order after the two seeded vertices */
  int32_t anchor[32]; /* an assigned query neighbour of order[t] */
  int32_t phi[32];
  uint8_t used_q[32];
  uint64_t count;
  uint64_t nodes, budget;
  int32_t *tuples; int64_t tuple_cap; int64_t *n_tuples;
  int over_budget;
  int32_t shard, nshards; /* this call enumerates the shard-th of nshards disjoint parts */
} srch;

/* label of the data edge (x, y) as the update k that touches it leaves or
 * finds it: an insertion's own label, else the label in G */
static int64_t touched_label(const srch *S, int64_t k, uint64_t key) {
  if (S->op[k] == 1) return S->uel ? S->uel[k] : 0;
  int64_t l = 0;
  hmap_get(S->gset, key, &l);
  return l;
}

/* Is data edge (x, y) an edge of the seed's view with label lab, and not an
 * update of the seed's sign with a smaller index (charging rule)? */
static int edge_ok(const srch *S, int32_t x, int32_t y, int64_t lab) {
  uint64_t k = ekey(x, y);
  int64_t bi;
  if (hmap_get(S->bmap, k, &bi)) {
    int bs = S->op[bi];
    if (bs != S->sign) return 0;      /* +: deleted edge not in G'; -: inserted edge not in G */
    if (touched_label(S, bi, k) != lab) return 0;
    return bi >= S->upd;              /* same sign: only later-or-equal updates */
  }
  int64_t l;
  return hmap_get(S->gset, k, &l) && l == lab;  /* untouched edge: in G iff in G' */
}

/* every query edge between u and an assigned query vertex maps into the view */
static int all_edges_ok(const srch *S, int32_t u, int32_t c) {
  for (int32_t e = 0; e < S->eq; e++) {
    int32_t a = S->qs[e], b = S->qd[e], w;
    if (a == u) w = b; else if (b == u) w = a; else continue;
    if (!S->used_q[w]) continue;
    if (!edge_ok(S, c, S->phi[w], S->qel ? S->qel[e] : 0)) return 0;
  }
  return 1;
}

static void emit(srch *S) {
  S->count++;
  if (S->tuples && S->n_tuples) {
    int64_t t = *S->n_tuples;
    if (t < S->tuple_cap) {
      int32_t *r = S->tuples + t * (2 + S->q);
      r[0] = (int32_t)S->upd; r[1] = S->sign;
      for (int32_t u = 0; u < S->q; u++) r[2 + u] = S->phi[u];
    }
    *S->n_tuples = t + 1;
  }
}

static void extend(srch *S, int32_t t) {
  if (S->over_budget) return;
  if (t == S->q) {
    /* a two-vertex query has no searched position: its match belongs to part 0 */
    if (t > 2 || S->shard == 0) emit(S);
    return;
  }
  int32_t u = S->order[t];
  const adj *A = S->view;
  /* every valid image of u carries u's label and is a view-neighbour of the
   * image of each assigned query neighbour of u; scan the shortest of those
   * neighbours' runs of u's label */
  int64_t lo = 0, hi = 0;
  label_run(A, S->phi[S->anchor[t]], S->qlab[u], &lo, &hi);
  for (int32_t e = 0; e < S->eq; e++) {
    int32_t a = S->qs[e], b = S->qd[e], w;
    if (a == u) w = b; else if (b == u) w = a; else continue;
    if (!S->used_q[w]) continue;
    int64_t l2, h2;
    label_run(A, S->phi[w], S->qlab[u], &l2, &h2);
    if (h2 - l2 < hi - lo) { lo = l2; hi = h2; }
  }
  for (int64_t p = lo; p < hi; p++) {
    /* parts: the first searched position's candidates are dealt round-robin by
     * their place in the scanned run, so the parts partition the matches */
    if (t == 2 && S->nshards > 1 && (p - lo) % S->nshards != S->shard) continue;
    int32_t c = A->nbr[p];
    if (++S->nodes > S->budget && S->budget) { S->over_budget = 1; return; }
    if (S->lab[c] != S->qlab[u]) continue;
    int dup = 0;
    for (int32_t w = 0; w < S->q; w++)
      if (S->used_q[w] && S->phi[w] == c) { dup = 1; break; }
    if (dup) continue;
    if (!all_edges_ok(S, u, c)) continue;
    S->phi[u] = c; S->used_q[u] = 1;
    extend(S, t + 1);
    S->used_q[u] = 0;
  }
}

/* order for a seeded query edge (a, b): repeatedly take the unassigned
 * vertex with the most assigned neighbours (ties: the smaller id); anchor =
 * its assigned neighbour with the smallest id.  Any order in which every
 * vertex has an assigned neighbour enumerates the same embeddings; this one
 * checks as many query edges as early as possible.  Returns 0 if Q is
 * disconnected. */
static int make_order(srch *S, int32_t a, int32_t b) {
  uint8_t in[32] = {0};
  in[a] = in[b] = 1;
  S->order[0] = a; S->order[1] = b;
  for (int32_t t = 2; t < S->q; t++) {
    int32_t pick = -1, anc = -1, best = 0;
    for (int32_t u = 0; u < S->q; u++) {
      if (in[u]) continue;
      int32_t nb = 0, first = -1;
      for (int32_t w = 0; w < S->q; w++) {
        if (!in[w]) continue;
        int adjq = 0;
        for (int32_t e = 0; e < S->eq; e++)
          if ((S->qs[e] == u && S->qd[e] == w) || (S->qs[e] == w && S->qd[e] == u)) { adjq = 1; break; }
        if (adjq) { nb++; if (first < 0) first = w; }
      }
      if (nb > best) { best = nb; pick = u; anc = first; }
    }
    if (pick < 0) return 0;
    in[pick] = 1; S->order[t] = pick; S->anchor[t] = anc;
  }
  return 1;
}

/* ---------------- a session: G, the batch and G' built once --------------- */
typedef struct {
  int32_t n;
  int32_t *labels;
  int64_t b;
  int8_t *op;
  int32_t *usrc, *udst, *uel; /* uel NULL: inserted edges have label 0 */
  hmap gset, bmap;
  adj AG, AP;
} oracle_session;

void oracle_session_close(oracle_session *z) {
  if (!z) return;
  adj_free(&z->AG); adj_free(&z->AP);
  hmap_free(&z->gset); hmap_free(&z->bmap);
  free(z->labels); free(z->op); free(z->usrc); free(z->udst); free(z->uel);
  free(z);
}

/*
 * oracle_session_open: validate and build G (n vertices with labels[n]; m
 * undirected edges (src[e], dst[e]) with labels elabel[m], NULL = all 0;
 * duplicates merged; a duplicate with a different label, a self-loop or a bad
 * id -> OR_EINVAL with bad_index = -1), the batch (b updates op[k] = +1/-1,
 * usrc[k], udst[k]; an insertion's edge gets label uelabel[k], NULL = 0) and
 * G'.  The arrays are copied; *out receives the session.  OR_EINVAL with
 * bad_index = the smallest offending update for an invalid batch.
 */
int oracle_session_open(int32_t n, const int32_t *labels, int64_t m, const int32_t *src, const int32_t *dst,
                        const int32_t *elabel, int64_t b, const int8_t *op, const int32_t *usrc,
                        const int32_t *udst, const int32_t *uelabel, oracle_session **out, int64_t *bad_index) {
  if (bad_index) *bad_index = -1;
  *out = NULL;
  oracle_session *z = (oracle_session *)calloc(1, sizeof(oracle_session));
  if (!z) return OR_ENOMEM;
  z->n = n; z->b = b;
  z->labels = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
  z->op = (int8_t *)malloc((size_t)b + 1);
  z->usrc = (int32_t *)malloc(((size_t)b + 1) * sizeof(int32_t));
  z->udst = (int32_t *)malloc(((size_t)b + 1) * sizeof(int32_t));
  if (uelabel) z->uel = (int32_t *)malloc(((size_t)b + 1) * sizeof(int32_t));
  if (!z->labels || !z->op || !z->usrc || !z->udst || (uelabel && !z->uel)) { oracle_session_close(z); return OR_ENOMEM; }
  memcpy(z->labels, labels, (size_t)n * sizeof(int32_t));
  if (b) {
    memcpy(z->op, op, (size_t)b);
    memcpy(z->usrc, usrc, (size_t)b * sizeof(int32_t));
    memcpy(z->udst, udst, (size_t)b * sizeof(int32_t));
    if (uelabel) memcpy(z->uel, uelabel, (size_t)b * sizeof(int32_t));
  }
  if (hmap_init(&z->gset, m) || hmap_init(&z->bmap, b)) { oracle_session_close(z); return OR_ENOMEM; }
  int32_t *gs = (int32_t *)malloc((size_t)(m + 1) * sizeof(int32_t));
  int32_t *gd = (int32_t *)malloc((size_t)(m + 1) * sizeof(int32_t));
  if (!gs || !gd) { free(gs); free(gd); oracle_session_close(z); return OR_ENOMEM; }
  int64_t mu = 0;
  for (int64_t e = 0; e < m; e++) {
    if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n || src[e] == dst[e]) {
      free(gs); free(gd); oracle_session_close(z); return OR_EINVAL;
    }
    const int64_t el = elabel ? elabel[e] : 0;
    if (hmap_put(&z->gset, ekey(src[e], dst[e]), el)) {
      gs[mu] = src[e]; gd[mu] = dst[e]; mu++;
    } else {
      int64_t had = 0;
      hmap_get(&z->gset, ekey(src[e], dst[e]), &had);
      if (had != el) { free(gs); free(gd); oracle_session_close(z); return OR_EINVAL; }
    }
  }
  /* batch validation, in index order */
  for (int64_t k = 0; k < b; k++) {
    int32_t x = usrc[k], y = udst[k];
    int bad = (op[k] != 1 && op[k] != -1) || x < 0 || x >= n || y < 0 || y >= n || x == y;
    if (!bad) {
      uint64_t kk = ekey(x, y);
      int ing = hmap_get(&z->gset, kk, NULL);
      if (!hmap_put(&z->bmap, kk, k)) bad = 1;
      else if (op[k] == 1 && ing) bad = 1;
      else if (op[k] == -1 && !ing) bad = 1;
    }
    if (bad) {
      if (bad_index) *bad_index = k;
      free(gs); free(gd); oracle_session_close(z); return OR_EINVAL;
    }
  }
  /* G' edge list */
  int32_t *ps = (int32_t *)malloc((size_t)(mu + b + 1) * sizeof(int32_t));
  int32_t *pd = (int32_t *)malloc((size_t)(mu + b + 1) * sizeof(int32_t));
  if (!ps || !pd) { free(ps); free(pd); free(gs); free(gd); oracle_session_close(z); return OR_ENOMEM; }
  int64_t mp = 0;
  for (int64_t e = 0; e < mu; e++) {
    int64_t bi;
    if (hmap_get(&z->bmap, ekey(gs[e], gd[e]), &bi) && op[bi] == -1) continue;
    ps[mp] = gs[e]; pd[mp] = gd[e]; mp++;
  }
  for (int64_t k = 0; k < b; k++)
    if (op[k] == 1) { ps[mp] = usrc[k]; pd[mp] = udst[k]; mp++; }
  int rc = (adj_build(&z->AG, n, mu, gs, gd, z->labels) || adj_build(&z->AP, n, mp, ps, pd, z->labels)) ? OR_ENOMEM
                                                                                                      : OR_OK;
  free(ps); free(pd); free(gs); free(gd);
  if (rc) { oracle_session_close(z); return rc; }
  *out = z;
  return OR_OK;
}

/*
 * oracle_session_eval: incremental matches of nq queries for the session's
 * batch.
 *   queries: query j has qn[j] <= 31 vertices with labels qlab + qlab_off[j],
 *            qe[j] edges (qsrc/qdst + qe_off[j]) with labels qelabel + qe_off[j]
 *            (NULL: all 0); each must be connected
 *   eval:    n_eval update indices to evaluate (eval_idx == NULL: all b, in order)
 *   out_count[j * ne + i]: matches of query j charged to update eval_idx[i]
 *   tuples:  (one query only) rows of (update, sign, phi[0..q-1]) up to tuple_cap
 *            rows; *n_tuples receives the number of rows produced
 *   node_budget: 0 = unlimited, else OR_EBUDGET once that many candidates were
 *            tried for one query
 *   update_budget: 0 = none, else each (query, update) evaluation may try that
 *            many candidates; one that needs more gets out_count = UINT64_MAX
 *            ("not computed") and the next one starts afresh
 *   shard, nshards: with nshards > 1, count only the part shard (0-based) of
 *            each (query, update) evaluation: the candidates of the first
 *            searched query vertex are dealt round-robin over nshards parts,
 *            so the parts' counts add up to the whole (nshards <= 1: all)
 * Returns OR_OK, OR_EINVAL, OR_EBUDGET.
 */
int oracle_session_eval(const oracle_session *z, int32_t nq, const int32_t *qn, const int32_t *qlab,
                        const int64_t *qlab_off, const int32_t *qe, const int32_t *qsrc, const int32_t *qdst,
                        const int64_t *qe_off, const int32_t *qelabel, int64_t n_eval, const int64_t *eval_idx,
                        uint64_t *out_count, int32_t *tuples, int64_t tuple_cap, int64_t *n_tuples,
                        uint64_t node_budget, uint64_t update_budget, int32_t shard, int32_t nshards) {
  if (n_tuples) *n_tuples = 0;
  if (!z || nq < 0 || (tuples && nq != 1)) return OR_EINVAL;
  if (nshards < 1) nshards = 1;
  if (shard < 0 || shard >= nshards) return OR_EINVAL;
  for (int32_t j = 0; j < nq; j++) {
    int32_t q = qn[j], eq = qe[j];
    const int32_t *qs = qsrc + qe_off[j], *qd = qdst + qe_off[j];
    if (q < 2 || q > 31 || eq < 1) return OR_EINVAL;
    for (int32_t e = 0; e < eq; e++)
      if (qs[e] < 0 || qs[e] >= q || qd[e] < 0 || qd[e] >= q || qs[e] == qd[e]) return OR_EINVAL;
  }
  const int32_t *labels = z->labels, *usrc = z->usrc, *udst = z->udst;
  const int8_t *op = z->op;
  const int64_t b = z->b;
  int rc = OR_OK;
  int64_t ne = eval_idx ? n_eval : b;
  for (int32_t j = 0; j < nq && rc == OR_OK; j++) {
    srch S;
    memset(&S, 0, sizeof(S));
    S.q = qn[j]; S.qlab = qlab + qlab_off[j]; S.eq = qe[j];
    S.qs = qsrc + qe_off[j]; S.qd = qdst + qe_off[j]; S.lab = labels;
    S.gset = &z->gset; S.bmap = &z->bmap; S.op = op; S.budget = node_budget;
    S.qel = qelabel ? qelabel + qe_off[j] : NULL; S.uel = z->uel;
    S.tuples = tuples; S.tuple_cap = tuple_cap; S.n_tuples = n_tuples;
    S.shard = shard; S.nshards = nshards;
    for (int64_t i = 0; i < ne && rc == OR_OK; i++) {
      int64_t k = eval_idx ? eval_idx[i] : i;
      if (k < 0 || k >= b) { rc = OR_EINVAL; break; }
      S.sign = op[k]; S.upd = k; S.view = (op[k] == 1) ? &z->AP : &z->AG;
      S.count = 0;
      if (update_budget) { S.nodes = 0; S.budget = update_budget; S.over_budget = 0; }
      for (int32_t e = 0; e < S.eq; e++) {
        for (int o = 0; o < 2; o++) {
          int32_t a = S.qs[e], bq = S.qd[e];
          int32_t x = o ? udst[k] : usrc[k], y = o ? usrc[k] : udst[k];
          if (labels[x] != S.qlab[a] || labels[y] != S.qlab[bq]) continue;
          if (touched_label(&S, k, ekey(x, y)) != (S.qel ? S.qel[e] : 0)) continue;
          if (!make_order(&S, a, bq)) { rc = OR_EINVAL; break; }
          memset(S.used_q, 0, sizeof(S.used_q));
          S.phi[a] = x; S.phi[bq] = y; S.used_q[a] = S.used_q[bq] = 1;
          extend(&S, 2);
          if (S.over_budget) { if (!update_budget) rc = OR_EBUDGET; break; }
        }
        if (rc != OR_OK || S.over_budget) break;
      }
      if (out_count) out_count[(int64_t)j * ne + i] = (update_budget && S.over_budget) ? UINT64_MAX : S.count;
    }
  }
  return rc;
}

/*
 * oracle_bdsm_multi_el: one call = open a session, evaluate, close it (the
 * arguments are those of oracle_session_open and oracle_session_eval, with
 * the whole search in one part).
 */
int oracle_bdsm_multi_el(int32_t n, const int32_t *labels, int64_t m, const int32_t *src, const int32_t *dst,
                         const int32_t *elabel, int32_t nq, const int32_t *qn, const int32_t *qlab,
                         const int64_t *qlab_off, const int32_t *qe, const int32_t *qsrc, const int32_t *qdst,
                         const int64_t *qe_off, const int32_t *qelabel, int64_t b, const int8_t *op,
                         const int32_t *usrc, const int32_t *udst, const int32_t *uelabel, int64_t n_eval,
                         const int64_t *eval_idx, uint64_t *out_count, int32_t *tuples, int64_t tuple_cap,
                         int64_t *n_tuples, uint64_t node_budget, uint64_t update_budget, int64_t *bad_index) {
  if (n_tuples) *n_tuples = 0;
  if (nq < 0 || (tuples && nq != 1)) { if (bad_index) *bad_index = -1; return OR_EINVAL; }
  for (int32_t j = 0; j < nq; j++) {  /* queries are checked before the graph is built */
    int32_t q = qn[j], eq = qe[j];
    const int32_t *qs = qsrc + qe_off[j], *qd = qdst + qe_off[j];
    if (q < 2 || q > 31 || eq < 1) { if (bad_index) *bad_index = -1; return OR_EINVAL; }
    for (int32_t e = 0; e < eq; e++)
      if (qs[e] < 0 || qs[e] >= q || qd[e] < 0 || qd[e] >= q || qs[e] == qd[e]) {
        if (bad_index) *bad_index = -1;
        return OR_EINVAL;
      }
  }
  oracle_session *z = NULL;
  int rc = oracle_session_open(n, labels, m, src, dst, elabel, b, op, usrc, udst, uelabel, &z, bad_index);
  if (rc != OR_OK) return rc;
  rc = oracle_session_eval(z, nq, qn, qlab, qlab_off, qe, qsrc, qdst, qe_off, qelabel, n_eval, eval_idx, out_count,
                           tuples, tuple_cap, n_tuples, node_budget, update_budget, 0, 1);
  oracle_session_close(z);
  return rc;
}

/* Vertex labels only: every edge has label 0. */
int oracle_bdsm_multi(int32_t n, const int32_t *labels, int64_t m, const int32_t *src, const int32_t *dst,
                      int32_t nq, const int32_t *qn, const int32_t *qlab, const int64_t *qlab_off,
                      const int32_t *qe, const int32_t *qsrc, const int32_t *qdst, const int64_t *qe_off,
                      int64_t b, const int8_t *op, const int32_t *usrc, const int32_t *udst,
                      int64_t n_eval, const int64_t *eval_idx, uint64_t *out_count,
                      int32_t *tuples, int64_t tuple_cap, int64_t *n_tuples,
                      uint64_t node_budget, uint64_t update_budget, int64_t *bad_index) {
  return oracle_bdsm_multi_el(n, labels, m, src, dst, NULL, nq, qn, qlab, qlab_off, qe, qsrc, qdst, qe_off, NULL, b,
                              op, usrc, udst, NULL, n_eval, eval_idx, out_count, tuples, tuple_cap, n_tuples,
                              node_budget, update_budget, bad_index);
}

/* One query: oracle_bdsm_multi with nq = 1. */
int oracle_bdsm(int32_t n, const int32_t *labels, int64_t m, const int32_t *src, const int32_t *dst,
                int32_t q, const int32_t *qlabels, int32_t eq, const int32_t *qsrc, const int32_t *qdst,
                int64_t b, const int8_t *op, const int32_t *usrc, const int32_t *udst,
                int64_t n_eval, const int64_t *eval_idx, uint64_t *out_count,
                int32_t *tuples, int64_t tuple_cap, int64_t *n_tuples,
                uint64_t node_budget, int64_t *bad_index) {
  int64_t zero = 0;
  return oracle_bdsm_multi(n, labels, m, src, dst, 1, &q, qlabels, &zero, &eq, qsrc, qdst, &zero, b, op, usrc,
                           udst, n_eval, eval_idx, out_count, tuples, tuple_cap, n_tuples, node_budget, 0,
                           bad_index);
}
