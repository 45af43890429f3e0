// gm_prims.cu -- device-wide exclusive scan and LSD radix sort used by the
// graph loader and the batch stager.  Temporaries come from the stream-ordered
// allocator (cudaMallocAsync), so a sequence of calls needs no host sync.
#include <stdio.h>

#include "gm_common.cuh"

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Block-local exclusive scan of one tile; block total to part[blockIdx.x].
template <typename T>
__global__ void k_scan_tile(const T *__restrict__ in, T *__restrict__ out, int64_t n,
                            T *__restrict__ part) {
  __shared__ T warp_tot[SCAN_THREADS / 32];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  T v[SCAN_ITEMS];
  T run = 0;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; j++) {
    int64_t i = base + j;
    T x = (i < n) ? in[i] : T(0);
    v[j] = run;
    run += x;
  }
  // warp-inclusive scan of per-thread totals
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T inc = run;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T y = __shfl_up_sync(GM_FULL, inc, d);
    if (lane >= d) inc += y;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T w = (lane < SCAN_THREADS / 32) ? warp_tot[lane] : T(0);
    T wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      T y = __shfl_up_sync(GM_FULL, wi, d);
      if (lane >= d) wi += y;
    }
    if (lane < SCAN_THREADS / 32) warp_tot[lane] = wi - w;  // exclusive
    if (lane == SCAN_THREADS / 32 - 1 && part) part[blockIdx.x] = wi;
  }
  __syncthreads();
  T off = warp_tot[warp] + inc - run;
#pragma unroll
  for (int j = 0; j < SCAN_ITEMS; j++) {
    int64_t i = base + j;
    if (i < n) out[i] = v[j] + off;
  }
}

template <typename T>
__global__ void k_scan_add(T *__restrict__ out, int64_t n, const T *__restrict__ part) {
  T add = part[blockIdx.x];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  for (int j = threadIdx.x; j < SCAN_TILE; j += blockDim.x) {
    int64_t i = base + j;
    if (i < n) out[i] += add;
  }
}

template <typename T>
int scan_excl(const T *in, T *out, int64_t n, cudaStream_t s) {
  if (n <= 0) return GAMMA_OK;
  int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb == 1) {
    k_scan_tile<T><<<1, SCAN_THREADS, 0, s>>>(in, out, n, (T *)nullptr);
    GM_LAUNCHED();
    GM_CUDA(cudaGetLastError());
    return GAMMA_OK;
  }
  T *part = nullptr;
  GM_CUDA(cudaMallocAsync((void **)&part, sizeof(T) * nb, s));
  k_scan_tile<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n, part);
  GM_LAUNCHED();
  GM_CUDA(cudaGetLastError());
  int rc = scan_excl<T>(part, part, nb, s);
  if (rc) { cudaFreeAsync(part, s); return rc; }
  k_scan_add<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(out, n, part);
  GM_LAUNCHED();
  GM_CUDA(cudaGetLastError());
  GM_CUDA(cudaFreeAsync(part, s));
  return GAMMA_OK;
}

// ---------------------------------------------------------------------------
// LSD radix sort, 8-bit digits.  A tile of RS_TILE keys per block; per pass:
// digit histogram per tile, exclusive scan of the digit-major count matrix,
// stable scatter (per-warp ranks with __match_any_sync, warps in order).
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_PER_WARP = 256;
constexpr int RS_TILE = RS_WARPS * RS_PER_WARP;

__global__ void k_rs_hist(const uint64_t *__restrict__ keys, int64_t n, int shift,
                          uint32_t *__restrict__ counts, int nblocks) {
  __shared__ uint32_t h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int j = threadIdx.x; j < RS_TILE; j += blockDim.x) {
    int64_t i = base + j;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) counts[(int64_t)d * nblocks + blockIdx.x] = h[d];
}

template <bool HAS_VAL>
__global__ void k_rs_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                             uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n,
                             int shift, const uint32_t *__restrict__ offs, int nblocks) {
  __shared__ uint32_t wcnt[RS_WARPS][256];
  __shared__ uint32_t boff[256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < RS_WARPS * 256; i += blockDim.x) (&wcnt[0][0])[i] = 0;
  for (int d = threadIdx.x; d < 256; d += blockDim.x) boff[d] = offs[(int64_t)d * nblocks + blockIdx.x];
  __syncthreads();
  const int64_t wbase = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * RS_PER_WARP;
  for (int r = 0; r < RS_PER_WARP / 32; r++) {
    int64_t i = wbase + r * 32 + lane;
    bool valid = i < n;
    uint32_t d = valid ? (uint32_t)((kin[i] >> shift) & 255u) : 256u + lane;
    unsigned peers = __match_any_sync(GM_FULL, d);
    if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {
    int d = threadIdx.x;  // RS_THREADS == 256 digits
    uint32_t run = 0;
    for (int w = 0; w < RS_WARPS; w++) {
      uint32_t t = wcnt[w][d];
      wcnt[w][d] = run;
      run += t;
    }
  }
  __syncthreads();
  for (int r = 0; r < RS_PER_WARP / 32; r++) {
    int64_t i = wbase + r * 32 + lane;
    bool valid = i < n;
    uint64_t k = valid ? kin[i] : 0;
    uint32_t v = (HAS_VAL && valid) ? vin[i] : 0;
    uint32_t d = valid ? (uint32_t)((k >> shift) & 255u) : 256u + lane;
    unsigned peers = __match_any_sync(GM_FULL, d);
    unsigned rank = __popc(peers & ((1u << lane) - 1u));
    if (valid) {
      uint32_t pos = boff[d] + wcnt[warp][d] + rank;
      kout[pos] = k;
      if (HAS_VAL) vout[pos] = v;
    }
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] += __popc(peers);
    __syncwarp();
  }
}

}  // namespace

int gm_scan_excl_u32(const uint32_t *in, uint32_t *out, int64_t n, cudaStream_t s) {
  return scan_excl<uint32_t>(in, out, n, s);
}

int gm_scan_excl_u64(const uint64_t *in, uint64_t *out, int64_t n, cudaStream_t s) {
  return scan_excl<uint64_t>(in, out, n, s);
}

int gm_radix_sort(uint64_t *keys, uint32_t *vals, uint64_t *tk, uint32_t *tv, int64_t n, int b0,
                  int b1, cudaStream_t s) {
  if (n <= 1) return GAMMA_OK;
  if (n >= (int64_t)1 << 32) return GAMMA_EINVAL;
  int nb = (int)((n + RS_TILE - 1) / RS_TILE);
  uint32_t *counts = nullptr;
  GM_CUDA(cudaMallocAsync((void **)&counts, sizeof(uint32_t) * 256 * (size_t)nb, s));
  uint64_t *ka = keys, *kb = tk;
  uint32_t *va = vals, *vb = tv;
  int passes = 0;
  for (int shift = b0; shift < b1; shift += 8, passes++) {
    k_rs_hist<<<nb, RS_THREADS, 0, s>>>(ka, n, shift, counts, nb);
    GM_LAUNCHED();
    GM_CUDA(cudaGetLastError());
    int rc = gm_scan_excl_u32(counts, counts, (int64_t)256 * nb, s);
    if (rc) return rc;
    if (vals)
      k_rs_scatter<true><<<nb, RS_THREADS, 0, s>>>(ka, va, kb, vb, n, shift, counts, nb);
    else
      k_rs_scatter<false><<<nb, RS_THREADS, 0, s>>>(ka, nullptr, kb, nullptr, n, shift, counts, nb);
    GM_LAUNCHED();
    GM_CUDA(cudaGetLastError());
    uint64_t *tk2 = ka; ka = kb; kb = tk2;
    uint32_t *tv2 = va; va = vb; vb = tv2;
  }
  if (passes & 1) {
    GM_CUDA(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
    if (vals) GM_CUDA(cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
  }
  GM_CUDA(cudaFreeAsync(counts, s));
  return GAMMA_OK;
}
