/*
 * rmat_gen.c -- the R-MAT edge draw of inputs.rmat_edges in C, for the
 * large synthetic graphs (the scale-23 graph takes minutes in numpy).  It is
 * part of the seeded input generator, not of the matching path, and gives
 * the same bytes as the numpy version (a CPU test compares them):
 *
 *   candidate i (i = 0, 1, ...): for level l = 0 .. scale-1 draw
 *     r = splitmix64(key + (i * scale + l + 1) * GOLD) >> 32
 *   and set bit (scale-1-l) of src when r >= t_ab, of dst when
 *   t_a <= r < t_ab or r >= t_abc;
 *   the edge is (min, max); self-loops are dropped; an edge already drawn
 *   is skipped; the first n_edges distinct edges are returned in draw order.
 *
 * splitmix64 is Steele, Lea and Flood's SplitMix64 output function
 * (OOPSLA 2014), the same constants as inputs._mix.
 */
#include <stdint.h>
#include <stdlib.h>

#define GOLD 0x9E3779B97F4A7C15ULL

static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* open addressing set of nonzero 64-bit keys */
typedef struct {
  uint64_t *k;
  uint64_t mask;
} kset;

static int kset_add(kset *s, uint64_t key) { /* 1 if new */
  uint64_t i = mix64(key) & s->mask;
  while (s->k[i]) {
    if (s->k[i] == key) return 0;
    i = (i + 1) & s->mask;
  }
  s->k[i] = key;
  return 1;
}

/* Returns the number of candidates drawn, or -1 when memory runs out.
 * out_src / out_dst receive n_edges endpoints (src < dst), before any
 * vertex relabelling. */
int64_t rmat_draw(int32_t scale, int64_t n_edges, uint64_t key, uint32_t t_a, uint32_t t_ab, uint32_t t_abc,
                  int32_t *out_src, int32_t *out_dst) {
  uint64_t cap = 16;
  while (cap < (uint64_t)(2 * n_edges + 16)) cap <<= 1;
  kset s;
  s.k = (uint64_t *)calloc(cap, sizeof(uint64_t));
  s.mask = cap - 1;
  if (!s.k) return -1;
  int64_t got = 0;
  uint64_t i = 0;
  for (; got < n_edges; i++) {
    uint64_t src = 0, dst = 0;
    for (int32_t l = 0; l < scale; l++) {
      const uint64_t idx = i * (uint64_t)scale + (uint64_t)l;
      const uint32_t r = (uint32_t)(mix64(key + (idx + 1) * GOLD) >> 32);
      const uint64_t bit = 1ULL << (scale - 1 - l);
      if (r >= t_ab) src |= bit;
      if ((r >= t_a && r < t_ab) || r >= t_abc) dst |= bit;
    }
    if (src == dst) continue;
    const uint64_t lo = src < dst ? src : dst, hi = src < dst ? dst : src;
    /* + 1 keeps the key nonzero (0 marks an empty slot) */
    if (!kset_add(&s, ((lo << 32) | hi) + 1)) continue;
    out_src[got] = (int32_t)lo;
    out_dst[got] = (int32_t)hi;
    got++;
  }
  free(s.k);
  return (int64_t)i;
}
