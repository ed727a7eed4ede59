// we_static.cu -- split/merge of one run's walkers for callers that cannot allocate device
// memory.  Some callers run inside a host framework whose caching allocator already owns all
// of the GPU's memory, or inside a loop where a cudaMalloc (which may synchronise the device
// and may fail under memory pressure) is not allowed once set-up is over.  This entry point
// gives them the bin-by-bin split/merge with its working memory taken from one fixed array in
// device global memory that is part of the library image, so nothing is allocated per call.
//
// The array holds working space for at most kStaticMaxWalkers walkers and kStaticMaxBins bins;
// every GPU that loads the library keeps it for the life of the process.  All calls share it:
// calls whose GPU work overlaps (concurrent streams, or the same call enqueued twice without
// ordering) race on it and give wrong results.  Each call clears what must start at zero.
#include <mutex>

#include "../../include/we_ssa.h"
#include "we_internal.cuh"

namespace we {
cudaError_t launch_resample_chain(const PropagateParams &prm, cudaStream_t st);
}
using namespace we;

namespace {

constexpr int kStaticMaxWalkers = WE_STATIC_MAX_WALKERS;
constexpr int kStaticMaxBins = WE_STATIC_MAX_BINS;

// Byte layout of the array (each piece 256-byte aligned).
constexpr size_t kOffScalars = 0;                                     // iter, count, n_tasks, status, run_id
constexpr size_t kOffBinCount = 256;
constexpr size_t kOffCursor = kOffBinCount + 4ull * kStaticMaxBins;
constexpr size_t kOffTasks = kOffCursor + 4ull * kStaticMaxBins;
constexpr size_t kOffBins = kOffTasks + 16ull * kStaticMaxBins;       // checked copy of the caller's bins
constexpr size_t kOffSlot = kOffBins + 4ull * kStaticMaxWalkers;
constexpr size_t kOffAlive = kOffSlot + 4ull * kStaticMaxWalkers;
constexpr size_t kOffSortedW = kOffAlive + 4ull * kStaticMaxWalkers;
constexpr size_t kStaticBytes = kOffSortedW + 8ull * kStaticMaxWalkers;

__device__ __align__(256) unsigned char g_scratch[kStaticBytes];

std::mutex g_mu;
void *g_scratch_ptr[256] = {};

// Device address of the array on the current device, looked up once per device.
cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Reset the per-call state: scalars, and bin counts that the grouping accumulates into.
__global__ void k_static_setup(unsigned char *scr, int n, int iter, uint32_t run_id, int n_bins) {
  int32_t *sc = reinterpret_cast<int32_t *>(scr + kOffScalars);
  int32_t *bc = reinterpret_cast<int32_t *>(scr + kOffBinCount);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc[0] = iter;
    sc[1] = n;
    sc[2] = 0;
    sc[3] = 0;
    reinterpret_cast<uint32_t *>(sc)[4] = run_id;
  }
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n_bins; b += gridDim.x * blockDim.x) bc[b] = 0;
}

// Copy the caller's bins into the array, counting walkers per bin; an out-of-range bin is
// replaced by bin 0 (so no access leaves the array) and flags WE_EINVAL.
__global__ void k_static_count(unsigned char *scr, const int32_t *bins, int n, int n_bins) {
  int32_t *sc = reinterpret_cast<int32_t *>(scr + kOffScalars);
  int32_t *bc = reinterpret_cast<int32_t *>(scr + kOffBinCount);
  int32_t *cb = reinterpret_cast<int32_t *>(scr + kOffBins);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int b = bins[i];
    if (b < 0 || b >= n_bins) {
      atomicCAS(&sc[3], 0, WE_EINVAL);
      b = 0;
    }
    cb[i] = b;
    atomicAdd(&bc[b], 1);
  }
}

// New walker count, or the negative status of a failed call.
__global__ void k_static_finish(const unsigned char *scr, int m_targ, int capacity, int32_t *out_count) {
  const int32_t *sc = reinterpret_cast<const int32_t *>(scr + kOffScalars);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const long long c = (long long)sc[2] * m_targ;
    out_count[0] = sc[3] ? sc[3] : (c > capacity ? WE_EOVERFLOW : (int32_t)c);
  }
}

}  // namespace

extern "C" we_status we_resample_static(int32_t n, const int32_t *bins, const double *weights,
                                        int32_t n_bins, int32_t m_targ, int32_t iter,
                                        uint64_t seed, uint32_t run_id, int32_t capacity,
                                        double *out_weights, int32_t *out_parent,
                                        int32_t *out_count, void *stream) {
  if (n < 1 || n > kStaticMaxWalkers) return WE_EINVAL;
  if (n_bins < 1 || n_bins > kStaticMaxBins) return WE_EINVAL;
  if (m_targ < 1 || iter < 0 || capacity < n || capacity > kStaticMaxWalkers) return WE_EINVAL;
  if (!bins || !weights || !out_weights || !out_parent || !out_count) return WE_EINVAL;
  void *p = nullptr;
  if (scratch_address(&p) != cudaSuccess) { cudaGetLastError(); return WE_ECUDA; }
  unsigned char *scr = static_cast<unsigned char *>(p);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  PropagateParams prm{};
  prm.resample = 1;
  prm.bins.n_bins = n_bins;
  EnsView &E = prm.ens;
  E.R = 1;
  E.cap = capacity;
  E.S = 1;
  E.m_targ = m_targ;
  E.div_magic = nullptr;                                 // the floating-point split/merge path
  E.record_iters = 0;                       // nothing is recorded
  E.first_iter = iter;
  E.seed = seed;
  const int par = iter & 1;
  int32_t *sc = reinterpret_cast<int32_t *>(scr + kOffScalars);
  E.iter = &sc[0];
  E.count = &sc[1];
  E.n_tasks = &sc[2];
  E.status = &sc[3];
  E.run_id = reinterpret_cast<const uint32_t *>(&sc[4]);
  E.w[par] = const_cast<double *>(weights);
  E.w[par ^ 1] = out_weights;
  E.parent[par ^ 1] = out_parent;
  E.bin = reinterpret_cast<int32_t *>(scr + kOffBins);
  E.bin_count = reinterpret_cast<int32_t *>(scr + kOffBinCount);
  E.cursor = reinterpret_cast<int32_t *>(scr + kOffCursor);
  E.tasks = reinterpret_cast<int4 *>(scr + kOffTasks);
  E.sorted_slot = reinterpret_cast<int32_t *>(scr + kOffSlot);
  E.alive = reinterpret_cast<int32_t *>(scr + kOffAlive);
  E.sorted_w = reinterpret_cast<double *>(scr + kOffSortedW);

  const int grid = (n + 255) / 256 < 152 ? (n + 255) / 256 : 152;
  k_static_setup<<<grid, 256, 0, st>>>(scr, n, iter, run_id, n_bins);
  k_static_count<<<grid, 256, 0, st>>>(scr, bins, n, n_bins);
  cudaError_t e = launch_resample_chain(prm, st);
  if (e == cudaSuccess) {
    k_static_finish<<<1, 32, 0, st>>>(scr, m_targ, E.cap, out_count);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) { cudaGetLastError(); return WE_ECUDA; }
  return WE_OK;
}
