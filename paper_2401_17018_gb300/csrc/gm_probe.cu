// gm_probe.cu -- gamma_probe_bandwidth: the read bandwidth of this GPU's
// memory hierarchy for a working set of a given size, measured by a
// read-only streaming kernel.  No counterpart in the paper: it supplies the
// denominator of the roofline for kernels whose working set stays in L2
// (the adjacency lists of the smaller graphs and the hubs' hash sets), which
// a DRAM copy bandwidth does not bound.
//
// The kernel: a grid of SMs x resident blocks; every thread reads 16-byte
// vectors at a grid stride over the buffer with loads that bypass L1
// (ld.global.cg), so a buffer smaller than L2 is served by L2 once warm, and
// a larger one by DRAM.  The XOR of the loaded words is kept and written
// only when it equals an impossible sentinel, so the loads are not removed.
#include <vector>

#include "gm_common.cuh"

namespace {

__global__ void __launch_bounds__(512) k_probe_read(const uint4 *__restrict__ buf, size_t nvec, int reps,
                                                    uint32_t *sink) {
  uint32_t acc = 0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; r++) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvec; i += stride) {
      const uint4 v = __ldcg(buf + i);
      acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
  }
  if (acc == 0x9e3779b9u) sink[0] = acc;
}

__global__ void k_probe_fill(uint4 *buf, size_t nvec) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvec; i += stride)
    buf[i] = make_uint4((uint32_t)i, (uint32_t)(i >> 32), 0x5bd1e995u, (uint32_t)i * 2654435761u);
}

}  // namespace

extern "C" int gamma_probe_bandwidth(int device, int64_t bytes, int32_t reps, int32_t trials, double *out_gbs) {
  if (!out_gbs || bytes < (1 << 20) || reps < 1 || trials < 1) return GAMMA_EINVAL;
  *out_gbs = 0.0;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return GAMMA_ECUDA;
  }
  GM_CUDA(cudaSetDevice(device));
  int sms = 0, per_sm = 0;
  GM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  const int threads = 512;
  GM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_read, threads, 0));
  if (per_sm < 1) return GAMMA_ECUDA;
  const size_t nvec = (size_t)bytes / sizeof(uint4);
  uint4 *buf = nullptr;
  uint32_t *sink = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = GAMMA_OK;
  float best = 0.f;
  if (cudaMalloc((void **)&buf, nvec * sizeof(uint4)) != cudaSuccess || cudaMalloc((void **)&sink, 4) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = GAMMA_ENOMEM;
  } else {
    k_probe_fill<<<sms * 4, 256, 0, s>>>(buf, nvec);
    GM_LAUNCHED();
    k_probe_read<<<sms * per_sm, threads, 0, s>>>(buf, nvec, 1, sink);  // warm: the buffer's lines into L2
    GM_LAUNCHED();
    for (int t = 0; t < trials && rc == GAMMA_OK; t++) {
      cudaEventRecord(e0, s);
      k_probe_read<<<sms * per_sm, threads, 0, s>>>(buf, nvec, reps, sink);
      GM_LAUNCHED();
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) { rc = GAMMA_ECUDA; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms > 0.f) {
        const float gbs = (float)((double)nvec * sizeof(uint4) * reps / (ms * 1e-3) / 1e9);
        if (gbs > best) best = gbs;
      }
    }
    if (cudaGetLastError() != cudaSuccess) rc = GAMMA_ECUDA;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (buf) cudaFree(buf);
  if (sink) cudaFree(sink);
  *out_gbs = best;
  return rc;
}
