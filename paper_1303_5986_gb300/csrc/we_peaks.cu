// we_peaks.cu -- measured throughput of the arithmetic pipes the SSA kernels use, the
// denominators of their rooflines: FP64 fused multiply-adds, 32-bit integer multiply-adds and
// 32-bit integer ALU operations (xor + add, the bulk of a Philox round and of the table
// path's index arithmetic), each counted in lane operations per second over the whole GPU.
//
// Every thread runs kChains independent dependency chains (enough to hide the pipe latency),
// the grid keeps every SM full, and the time is the CUDA-event duration of one launch after a
// warm-up launch.  The chains' results feed a store that never happens unless a caller passes
// an impossible seed, so the compiler keeps every operation.
#include <cuda_runtime.h>

#include "../../include/we_ssa.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_peak_fp64(int iters, double seed, double *sink) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + c + threadIdx.x;
  const double m = 1.0000000001, b = 1e-12;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = __fma_rn(a[c], m, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == -1.0) sink[0] = s;
}

__global__ void __launch_bounds__(kThreads) k_peak_imad(int iters, uint32_t seed, uint32_t *sink) {
  uint32_t a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + c * 7919u + threadIdx.x;
  const uint32_t m = 0x9E3779B1u, b = 0x7F4A7C15u;
  for (int i = 0; i < iters; ++i) {
    const uint32_t mi = m ^ (uint32_t)(i << 1);       // a new odd multiplier each step: no closed form
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = a[c] * mi + b;
  }
  uint32_t s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s ^= a[c];
  if (s == 0xFFFFFFFFu && seed == 1u) sink[0] = s;
}

// xor then add: two integer ALU operations per step of each chain
__global__ void __launch_bounds__(kThreads) k_peak_ialu(int iters, uint32_t seed, uint32_t *sink) {
  uint32_t a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + c * 104729u + threadIdx.x;
  const uint32_t k0 = 0xBB67AE85u, k1 = 0x3C6EF372u;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = (a[c] ^ k0) + (k1 + (uint32_t)i);
  }
  uint32_t s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s ^= a[c];
  if (s == 0xFFFFFFFFu && seed == 1u) sink[0] = s;
}

__global__ void k_empty() {}

}  // namespace

// The launch-latency floor of a WE iteration: one CUDA graph of `kernels` empty launches in a
// chain (each one block per SM of 128 threads, the shape of the iteration's kernels without
// their work), replayed n_replays times back to back; the CUDA-event time per replay.
extern "C" we_status we_measure_graph_floor(int32_t kernels, int32_t n_replays, void *stream,
                                            double *ms_per_replay) {
  if (kernels < 1 || kernels > 64 || n_replays < 1 || !ms_per_replay) return WE_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return WE_ECUDA;
  }
  cudaStream_t cap = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t x = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  we_status rc = WE_OK;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    rc = WE_ECUDA;
  } else {
    for (int k = 0; k < kernels; ++k) k_empty<<<sms, 128, 0, cap>>>();
    if (cudaStreamEndCapture(cap, &g) != cudaSuccess || cudaGraphInstantiate(&x, g, 0) != cudaSuccess)
      rc = WE_ECUDA;
  }
  if (rc == WE_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = WE_ECUDA;
  if (rc == WE_OK) {
    float ms = 0.f;
    for (int rep = 0; rep < 2 && rc == WE_OK; ++rep) {   // warm-up, then the timed replays
      cudaEventRecord(e0, st);
      for (int i = 0; i < n_replays; ++i) cudaGraphLaunch(x, st);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        rc = WE_ECUDA;
    }
    if (rc == WE_OK) *ms_per_replay = (double)ms / n_replays;
  }
  if (x) cudaGraphExecDestroy(x);
  if (g) cudaGraphDestroy(g);
  if (cap) cudaStreamDestroy(cap);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc != WE_OK) cudaGetLastError();
  return rc;
}

extern "C" we_status we_measure_alu_peaks(void *stream, double *fp64_fma_per_s, double *imad_per_s,
                                          double *ialu_per_s) {
  if (!fp64_fma_per_s || !imad_per_s || !ialu_per_s) return WE_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return WE_ECUDA;
  }
  void *sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  we_status rc = WE_OK;
  if (cudaMalloc(&sink, 64) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = WE_ECUDA;
  }
  const int blocks = sms * 8;                         // 8 blocks of 256 threads per SM
  const double lanes = (double)blocks * kThreads * kChains;
  auto timed = [&](int which, int iters, double *out, double ops_per_step) {
    if (rc != WE_OK) return;
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {               // warm-up, then the timed launch
      cudaEventRecord(e0, st);
      if (which == 0) k_peak_fp64<<<blocks, kThreads, 0, st>>>(iters, 0.5, static_cast<double *>(sink));
      else if (which == 1) k_peak_imad<<<blocks, kThreads, 0, st>>>(iters, 3u, static_cast<uint32_t *>(sink));
      else k_peak_ialu<<<blocks, kThreads, 0, st>>>(iters, 3u, static_cast<uint32_t *>(sink));
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = WE_ECUDA;
        return;
      }
    }
    *out = lanes * iters * ops_per_step / (ms * 1e-3);
  };
  timed(0, 4096, fp64_fma_per_s, 1.0);
  timed(1, 65536, imad_per_s, 1.0);
  timed(2, 65536, ialu_per_s, 2.0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (rc != WE_OK) cudaGetLastError();
  return rc;
}
