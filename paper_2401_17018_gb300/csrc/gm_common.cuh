// gm_common.cuh -- shared device-side types and helpers of libgamma.
//
// Adjacency key (one uint32 per directed adjacency entry):
//   key = (label << (idb + 1)) | (id << 1) | flag
// where idb = bits of the vertex id.  Every adjacency list is sorted by key,
// i.e. by neighbour label first, then id, so the neighbours of v that carry
// label l (N^l(v), Sec. II-A) form one contiguous segment found by two binary
// searches, and two lists can be intersected segment by segment.  flag = 1
// marks an edge touched by the staged batch; its update index and sign are in
// etag[] at the same slot: etag = (update index << 1) | (1 if deletion).
// The flag is the least significant bit so it never changes the sort order.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gamma.h"

#define GM_MAXQ 16
#define GM_HUB_MIN 16           // default list length that makes a vertex a hub (hash-indexed) at load
#define GM_SCAN_MAX 16          // lists up to this length are read whole for a membership test
#define GM_COL_PAD 8            // words after the adjacency pool, so 16-byte reads of a short list stay inside
#define GM_EMPTY 0x80000000u    // empty hash slot (keys use at most 31 bits when hashing is on)
#define GM_FULL 0xffffffffu
#define GM_MAX_DEVICES 128       // device ordinals the library keeps per-device state for

// ---------------------------------------------------------------------------
// device status block (one per context, reset at the start of every call)
// ---------------------------------------------------------------------------
struct GmStatus {
  int32_t err;            // first error code set (0 = none)
  int32_t abort;          // set when the work budget is exceeded
  int64_t bad_index;      // smallest offending update / edge index
  uint32_t ntouched;      // vertices whose list the batch touches (groups)
  uint32_t pool_top;      // adjacency slots allocated
  uint64_t reloc_total;   // slots the batch needs for relocated lists
  uint64_t nseeds;        // seeds passing label + filter tests
  uint64_t nitems;        // DFS work items written (may exceed capacity)
  uint64_t next_item;     // DFS scheduling cursor
  uint64_t expansions;    // 32-wide expansion steps done
  uint64_t rows;          // match rows produced (may exceed capacity)
  uint64_t live;          // change of directed entries at commit
  uint64_t alg_bytes;     // DFS algorithmic bytes (instrumented mode)
  uint64_t garbage;       // slots freed by relocation
  uint32_t max_label;     // load: largest vertex label
  uint32_t hub_top;       // hub hash slots allocated
  uint32_t tasks_donated; // tasks the last DFS launch split off
  uint32_t n2_valid;      // staged directed entries (the sorted batch's entries before its unused tail)
};

// DFS scheduling counters, one per 128-byte line (reset before every DFS launch)
#define GM_SCHED_TICKET 0   // tickets taken by warps waiting for donated work
#define GM_SCHED_RESERVE 32 // donated-task slots reserved (slot t goes to ticket t)
#define GM_SCHED_BUSY 64    // warps holding work, including reserved but unclaimed slots
#define GM_SCHED_WORDS 128

// ---------------------------------------------------------------------------
// device view of the dynamic CSR (passed by value)
// ---------------------------------------------------------------------------
struct GraphDev {
  const int32_t *label;  // [n]
  uint2 *adj;            // [n] {offset into col, length}
  uint32_t *cap;         // [n] slots reserved at offset
  uint32_t *col;         // [pool] adjacency keys
  uint32_t *etag;        // [pool] batch tag of flagged entries
  uint8_t *elab;         // [pool] edge label of each entry (null: an unlabelled graph, every edge label 0)
  uint8_t *nlf;          // [n * nlfw] per-label neighbour counts of the union graph, saturated at 255
  int32_t *vgroup;       // [n] while a batch is staged: the vertex's group in the sorted batch, else -1
  // hub index: vertices whose list had >= the hub threshold entries at load keep the
  // start of every label segment and an open-addressing hash set of their keys
  const int32_t *hub_id; // [n] hub number or -1
  uint32_t *hub_lofs;    // [nhub * (nlab + 1)] label-segment starts within the list
  uint2 *hub_tab;        // [n] per vertex {first slot in hub_keys, log2 capacity} (capacity 0: no table)
  uint32_t *hub_keys;    // hash slots (GM_EMPTY or an adjacency key)
  uint32_t hub_keys_cap;
  int32_t nhub;
  int32_t n;
  int32_t idb;           // id bits
  int32_t nlab;          // labels 0..nlab-1
  int32_t nlfw;          // bytes per nlf row (multiple of 4)
  uint32_t idmask;
  uint32_t pool_cap;
};

// ---------------------------------------------------------------------------
// matching plan: one per (query, query edge, orientation)  (Alg. 1 input pi)
// ---------------------------------------------------------------------------
struct Plan {
  int32_t qslot;                  // index of the query in the current apply call
  int32_t q;                      // query vertices
  int32_t qid;                    // registered query id
  int32_t pad;
  int32_t lab[GM_MAXQ];           // label of pi[l]
  uint16_t bwd[GM_MAXQ];          // positions k < l with (pi[k], pi[l]) in E(Q)
  uint16_t samelab[GM_MAXQ];      // positions k < l with L(pi[k]) = L(pi[l])
  int8_t qv[GM_MAXQ];             // pi[l] (query vertex id)
  uint8_t nreq[GM_MAXQ];          // neighbour-label requirements of pi[l]
  uint8_t req_lab[GM_MAXQ][GM_MAXQ - 1];
  uint8_t req_cnt[GM_MAXQ][GM_MAXQ - 1];
  uint8_t el[GM_MAXQ][GM_MAXQ];   // el[l][k], k < l: label of the query edge (pi[l], pi[k]) (Sec. II-A)
};

// DFS work item: a seed (update, plan) and a slice of its level-2 candidates
struct WorkItem {
  uint32_t upd;
  uint16_t plan;
  uint8_t drv;   // position (0 or 1) whose neighbour segment drives level 2
  uint8_t pad;
  uint32_t lo;   // first col slot of the slice
  uint32_t len;  // slots in the slice
};

// Work split off by a busy DFS warp for an idle one: the slots [lo, lo+len)
// of the driver segment of one partial match at stored level `depth` (its
// vertices at positions 2..depth+2 in m[]; positions 0, 1 are the update's
// endpoints), or, with depth -1, a slice of a seed's level-2 segment.
#define GM_TASK_M 12
struct Task {
  uint32_t upd;
  uint16_t plan;
  int8_t depth;
  uint8_t drv;
  uint32_t lo;
  uint32_t len;
  uint32_t m[GM_TASK_M];
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
__host__ __device__ inline uint32_t gm_key(int32_t lab, uint32_t id, int idb) {
  return ((uint32_t)lab << (idb + 1)) | (id << 1);
}

// first index in a[0, len) whose value is >= key
__device__ __forceinline__ uint32_t gm_lower_bound(const uint32_t *__restrict__ a, uint32_t len,
                                                   uint32_t key) {
  uint32_t lo = 0, hi = len;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__host__ __device__ __forceinline__ uint32_t gm_hash(uint32_t k) {
  k ^= k >> 16; k *= 0x85ebca6bu;
  k ^= k >> 13; k *= 0xc2b2ae35u;
  k ^= k >> 16;
  return k;
}

__device__ __forceinline__ void gm_set_err(GmStatus *st, int code) {
  atomicCAS(&st->err, 0, code);
}

__device__ __forceinline__ void gm_bad_index(GmStatus *st, int64_t k) {
  atomicMin((long long *)&st->bad_index, (long long)k);
}

#define GM_CUDA(call)                                                   \
  do {                                                                  \
    cudaError_t e__ = (call);                                           \
    if (e__ != cudaSuccess) return gm_cuda_fail(e__, #call, __FILE__, __LINE__); \
  } while (0)

int gm_cuda_fail(cudaError_t e, const char *what, const char *file, int line);

// kernels launched by the library in this process (read into gamma_stats)
extern unsigned long long gm_launch_count;
#define GM_LAUNCHED() __atomic_add_fetch(&gm_launch_count, 1ull, __ATOMIC_RELAXED)

// primitives (gm_prims.cu)
int gm_scan_excl_u32(const uint32_t *in, uint32_t *out, int64_t n, cudaStream_t s);
int gm_scan_excl_u64(const uint64_t *in, uint64_t *out, int64_t n, cudaStream_t s);
// LSD radix sort of (key, value) pairs on bits [b0, b1); keys/vals are sorted in place
// using tk/tv as the alternate buffers (each >= n elements); vals may be NULL.
int gm_radix_sort(uint64_t *keys, uint32_t *vals, uint64_t *tk, uint32_t *tv, int64_t n,
                  int b0, int b1, cudaStream_t s);
