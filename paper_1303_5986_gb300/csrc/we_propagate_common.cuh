// we_propagate_common.cuh -- device helpers shared by the SSA kernels of we_propagate.cu and
// the pipelined table kernel (we_pipe.cuh, compiled in we_pipe3.cu and we_pipe4.cu): the
// canonical-tree descent, the state-indexed table row, the shared-memory prologue, the
// epilogue that stores a walker and records the interval's observables, and the host-side
// launch helpers.
#pragma once
#include <algorithm>

#include "we_ssa_common.cuh"

namespace we {

// A double as an unevaluated float pair (hi = nearest float, lo = nearest float to the rest).
__device__ __forceinline__ float2 split_ff(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(__dsub_rn(x, (double)h)));
}

template <int P, int LOG2P>
__device__ __forceinline__ int descend(const double *nd, unsigned long long m) {
  double target = __dmul_rn(u01_index(m), nd[1]);
  int k = 1;
  for (int lvl = 0; lvl < LOG2P; ++lvl) {
    const double L = nd[2 * k], R = nd[2 * k + 1];
    const bool right = (bits(R) != 0) && !(bits(target) < bits(L));
    if (right) { target = __dsub_rn(target, L); k = 2 * k + 1; }
    else { k = 2 * k; }
  }
  return k - P;
}

// Row x of the state-indexed table (P 64-bit words): the float-float (2^62 / tau) / a0 that
// turns -log u1 into clock units, then the breakpoints b_1 .. b_{P-1}, b_i being the least
// uniform index m whose descent picks a reaction >= i.  The descent is monotone in m (the
// target fl(u2 a0) grows with u2, each comparison is a threshold, each subtraction is monotone),
// so the reaction for m is the number of b_i <= m: the hot loop selects with integer compares
// and reaches exactly the reaction the floating-point descent would.  base holds the counts of
// the species other than `species`.
__device__ __forceinline__ unsigned long long pack_ff(float2 f) {
  return ((unsigned long long)__float_as_uint(f.y) << 32) | (unsigned long long)__float_as_uint(f.x);
}
__device__ __forceinline__ float2 unpack_ff(unsigned long long v) {
  return make_float2(__uint_as_float((uint32_t)v), __uint_as_float((uint32_t)(v >> 32)));
}

// (2^62 / tau) / a0 as a float-float, or zero when nothing can fire.
__device__ __forceinline__ float2 wait_scale(double a0, double clock_scale) {
  return bits(a0) > 0 ? split_ff(__ddiv_rn(clock_scale, a0)) : make_float2(0.0f, 0.0f);
}

template <int P, int LOG2P>
struct TableRow {
  float2 w;
  unsigned long long bp[P > 1 ? P - 1 : 1];
  bool direct;

  // rw: a row of P words, 16-byte aligned when P is even (read two words at a time)
  __device__ __forceinline__ void read(const unsigned long long *rw) {
    unsigned long long v[P];
    if (P % 2 == 0) {
#pragma unroll
      for (int i = 0; i < P; i += 2) {
        const ulonglong2 q = reinterpret_cast<const ulonglong2 *>(rw)[i / 2];
        v[i] = q.x;
        v[i + 1 < P ? i + 1 : i] = q.y;
      }
    } else {
#pragma unroll
      for (int i = 0; i < P; ++i) v[i] = rw[i];
    }
    w = unpack_ff(v[0]);
#pragma unroll
    for (int i = 1; i < P; ++i) bp[i - 1] = v[i];
    direct = false;
  }
  // counts xme (stride B) are current, including the table species
  __device__ __forceinline__ void evaluate(double *fb, const RxnMeta *meta, const double *keff,
                                           const double *Kn, const int32_t *xme, int B, double clock_scale) {
#pragma unroll
    for (int j = 0; j < P; ++j) fb[P + j] = propensity(meta[j], keff[j], Kn[j], xme, B);
#pragma unroll
    for (int k = P - 1; k >= 1; --k) fb[k] = __dadd_rn(fb[2 * k], fb[2 * k + 1]);
    w = wait_scale(fb[1], clock_scale);
    direct = true;
  }
  __device__ __forceinline__ bool idle() const { return __float_as_uint(w.x) == 0u; }
  __device__ __forceinline__ int select_table(unsigned long long m2) const {
    int j = 0;                                            // reaction = breakpoints at or below m2
#pragma unroll
    for (int i = 0; i + 1 < P; ++i) j += (long long)m2 >= (long long)bp[i] ? 1 : 0;
    return j;
  }
  __device__ __forceinline__ int select(unsigned long long m2, const double *fb) const {
    if (direct) return descend<P, LOG2P>(fb, m2);
    int j = 0;                                            // reaction = breakpoints at or below m2
#pragma unroll
    for (int i = 0; i + 1 < P; ++i) j += (long long)m2 >= (long long)bp[i] ? 1 : 0;
    return j;
  }
};

// Shared prologue: network records, rate constants, net changes and log tables to shared
// memory.  Returns the per-thread count slots (S x blockDim, species-major).
struct Smem {
  RxnMeta *meta;
  double *keff, *Kn;
  int32_t *dsp, *dval;
  LogTables *logt;
  int32_t *xs;
};

template <int P>
__device__ __forceinline__ Smem load_smem(const PropagateParams &prm, unsigned char *raw) {
  const NetView &N = prm.net;
  const int B = blockDim.x, tid = threadIdx.x;
  Smem m;
  m.logt = reinterpret_cast<LogTables *>(raw);
  m.meta = reinterpret_cast<RxnMeta *>(m.logt + 1);
  m.keff = reinterpret_cast<double *>(m.meta + P);
  m.Kn = m.keff + N.n_param_sets * P;
  m.dsp = reinterpret_cast<int32_t *>(m.Kn + N.n_param_sets * P);
  m.dval = m.dsp + N.n_delta;
  m.xs = m.dval + N.n_delta;
  const double *lt = reinterpret_cast<const double *>(prm.logt);
  double *ls = reinterpret_cast<double *>(m.logt);
  for (int i = tid; i < (int)(sizeof(LogTables) / 8); i += B) ls[i] = lt[i];
  for (int i = tid; i < P * 16; i += B)
    reinterpret_cast<int32_t *>(m.meta)[i] = reinterpret_cast<const int32_t *>(N.meta)[i];
  for (int i = tid; i < N.n_param_sets * P; i += B) { m.keff[i] = N.keff[i]; m.Kn[i] = N.hill_Kn[i]; }
  for (int i = tid; i < N.n_delta; i += B) { m.dsp[i] = N.d_sp[i]; m.dval[i] = N.d_val[i]; }
  __syncthreads();
  return m;
}

// Epilogue: store the counts, bin the walker, record the interval's observables.
__device__ __forceinline__ void finish_walker(const PropagateParams &prm, int r, int g, int par, int iter,
                                              int32_t *xme, int B, double t, long long nev,
                                              int nrec, int status, int near) {
  const EnsView &E = prm.ens;
  const int ld = E.R * E.cap;
  // the walker's weight is loaded first, so that the load overlaps the stores and the binning
  const int slot = iter - E.first_iter;
  const bool rec = slot >= 0 && slot < E.record_iters;
  const double wt = rec ? E.w[par][g] : 0.0;
  int32_t *X = E.x[par];
  // target checked at the interval's end only: a walker found in it goes to the recycle state
  if (E.end_check && in_target(E, r, xme, B)) {
    for (int s = 0; s < E.S; ++s) xme[s * B] = E.recycle[r * E.S + s];
    nrec = 1;
  }
  for (int s = 0; s < E.S; ++s) X[(size_t)s * ld + g] = xme[s * B];
  E.nrec[g] = nrec;
  E.tlast[g] = t;
  if (E.fpt) record_first_passage(E, r, g, xme, B, nrec, t);
  if (status) atomicCAS(&E.status[r], 0, status);
  if (!prm.bins.learned) {
    const int b = bin_of(prm.bins, xme, B);
    E.bin[g] = b;
    if (prm.resample) atomicAdd(&E.bin_count[r * prm.bins.n_bins + b], 1);
  }
  if (rec) {
    const int o = slot * E.R + r;
    if (nrec) atomicAdd(&E.obs_flux[o], __dmul_rn((double)nrec, wt));
    if (nev) atomicAdd(&E.obs_events[o], (unsigned long long)nev);
    if (near) atomicAdd(&E.obs_near[o], 1);
    if (E.hist_len > 0) {
      const int v = xme[E.hist_species * B];
      const int idx = v < E.hist_len - 1 ? v : E.hist_len - 1;
      atomicAdd(&E.obs_hist[(size_t)o * E.hist_len + idx], wt);
    }
    if (!prm.resample) atomicAdd(&E.obs_totw[o], wt);
  }
}

// Warp-specialised kernels: rounds of draws handed from draw warps to the event warp(s).
constexpr int kRoundDraws = 16;
constexpr int kWindowMargin = 96;    // table rows staged beyond a block's range of counts

// Off-table rows: the canonical tree evaluated on the fly (counts beyond the table), kept out
// of line so that the event chain stays short.
template <int P, int LOG2P>
__device__ __forceinline__ float2 evaluate_row(double *fb, const RxnMeta *meta, const double *keff,
                                            const double *Kn, const int32_t *xme, int B, double clock_scale) {
#pragma unroll
  for (int j = 0; j < P; ++j) fb[P + j] = propensity(meta[j], keff[j], Kn[j], xme, B);
#pragma unroll
  for (int k = P - 1; k >= 1; --k) fb[k] = __dadd_rn(fb[2 * k], fb[2 * k + 1]);
  return wait_scale(fb[1], clock_scale);
}
template <int P, int LOG2P>
__device__ __forceinline__ int descend_row(const double *fb, unsigned long long m2) {
  return descend<P, LOG2P>(fb, m2);
}

size_t propagate_pipe_smem(const NetView &N, int table_rows);

template <typename K>
static cudaError_t launch_k(K kern, const PropagateParams &prm, int grid, int block, size_t smem,
                            cudaStream_t st) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, block, smem, st>>>(prm);
  return cudaGetLastError();
}

// Rows of the table a block of the warp-specialised kernel may stage: as many as fit while
// every block of the launch stays resident at once (up to the kernel's register limit of
// blocks per SM), and no more than the table has.
static int device_attr(cudaDeviceAttr a, int fallback) {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, a, dev) != cudaSuccess) {
    cudaGetLastError();
    return fallback;
  }
  return v;
}
static int num_sms() { return std::max(1, device_attr(cudaDevAttrMultiProcessorCount, 1)); }

template <typename K>
static int pipe_table_rows(K kern, const PropagateParams &prm, int grid, int max_per_sm) {
  if (prm.tab.species < 0 || prm.tab.len <= 0 || prm.tab.species2 >= 0) return 0;   // 1-D window only
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) { cudaGetLastError(); return 0; }
  const int by_regs = std::min(max_per_sm, std::max(1, 65536 / std::max(1, fa.numRegs * 128)));
  const int sms = num_sms();
  const int per_sm = std::min(by_regs, std::max(1, (grid + sms - 1) / sms));
  // an SM's shared memory, shared by per_sm blocks, each of which also holds the reserved
  // bytes per block and the kernel's static shared variables; a block's own limit on top
  const size_t sm_bytes = (size_t)device_attr(cudaDevAttrMaxSharedMemoryPerMultiprocessor, 228 * 1024);
  const size_t reserved = (size_t)device_attr(cudaDevAttrReservedSharedMemoryPerBlock, 1024);
  const size_t block_max = (size_t)device_attr(cudaDevAttrMaxSharedMemoryPerBlockOptin, 227 * 1024);
  const size_t per_block = sm_bytes / per_sm;
  if (per_block <= reserved + fa.sharedSizeBytes || block_max <= fa.sharedSizeBytes) return 0;
  const size_t budget = std::min(per_block - reserved, block_max) - fa.sharedSizeBytes;
  const size_t base = propagate_pipe_smem(prm.net, 0);
  if (base >= budget) return 0;
  const size_t rows = (budget - base) / ((size_t)prm.net.P * sizeof(unsigned long long));
  return (int)std::min<size_t>(rows, (size_t)prm.tab.len);
}

// Blocks of a persistent launch: enough for every capacity slot, at most the resident ones
// (the kernels loop over groups of 32 walkers).
template <typename K>
static int persistent_grid(K kern, int groups, int max_per_sm = 16) {
  cudaFuncAttributes fa;
  int per_sm = 4;
  if (cudaFuncGetAttributes(&fa, kern) == cudaSuccess && fa.numRegs > 0)
    per_sm = std::max(1, std::min(max_per_sm, 65536 / (fa.numRegs * 128)));
  else
    cudaGetLastError();
  return std::max(1, std::min(groups, per_sm * num_sms()));
}

// The pipelined kernel built for blocks_per_sm blocks per SM is launched with at most that many
// per SM (its table window takes the shared memory they leave).
template <typename K>
static cudaError_t launch_pipe(K kern, const PropagateParams &prm_in, int groups, cudaStream_t st,
                               int blocks_per_sm) {
  PropagateParams prm = prm_in;
  const int grid = persistent_grid(kern, groups, blocks_per_sm);
  prm.tab.smem_rows = pipe_table_rows(kern, prm, grid, blocks_per_sm);
  // the window is sized to fill the SM's shared memory: ask for the largest carveout
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  return launch_k(kern, prm, grid, 128, propagate_pipe_smem(prm.net, prm.tab.smem_rows), st);
}

template <typename K>
static cudaError_t launch_ws(K kern, const PropagateParams &prm, int groups, size_t smem, cudaStream_t st) {
  return launch_k(kern, prm, persistent_grid(kern, groups), 128, smem, st);
}

}  // namespace we
