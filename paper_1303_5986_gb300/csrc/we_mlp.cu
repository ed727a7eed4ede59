// we_mlp.cu -- a small MLP progress coordinate for WE binning (species counts -> log1p ->
// 64 -> 64 -> 1 with SiLU), trained by hand-written forward/backward kernels and used only to
// place bins.  WE is unbiased under any binning (Sec. II.B; adaptive or learned bins are the
// open problem of Sec. IV.B), so the learned coordinate changes efficiency, never the answer.
//
//   training (FP32 master weights), two kernels per Adam step:
//     k_mlp_train_tiles  a block per tile of samples: forward pass, BCE-with-logits loss and
//                        backward pass in shared memory; per-block gradient rows
//     k_mlp_reduce       one thread per parameter: the rows summed in block order
//                        (deterministic), then an Adam step (or just the gradient, for checks)
//   inference (BF16 weights, FP32 arithmetic), fused with bin assignment:
//     k_learned_bins one thread per walker after the SSA kernel: z, its bin, bin counts
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/we_ssa.h"
#include "we_mlp.cuh"
#include "we_ssa_common.cuh"

namespace we {

// Parameter layout (flat, FP32): W1[H][n_in], b1[H], W2[H][H], b2[H], w3[H], b3.
struct MlpShape {
  int n_in, H;
  __host__ __device__ int o_w1() const { return 0; }
  __host__ __device__ int o_b1() const { return H * n_in; }
  __host__ __device__ int o_w2() const { return H * n_in + H; }
  __host__ __device__ int o_b2() const { return H * n_in + H + H * H; }
  __host__ __device__ int o_w3() const { return H * n_in + 2 * H + H * H; }
  __host__ __device__ int o_b3() const { return H * n_in + 3 * H + H * H; }
  __host__ __device__ int n_params() const { return H * n_in + 3 * H + H * H + 1; }
};

__device__ __forceinline__ float sigmoid_f(float a) { return __fdiv_rn(1.0f, __fadd_rn(1.0f, expf(-a))); }
__device__ __forceinline__ float dsilu_f(float a) {              // d/da (a sigmoid(a))
  const float s = sigmoid_f(a);
  return __fmul_rn(s, __fadd_rn(1.0f, __fmul_rn(a, __fsub_rn(1.0f, s))));
}

// Training step, kernel 1 of 2.  A block takes tiles of SB samples (tile t = samples
// start + t*SB ... of the batch, wrapping around the data); for each tile it runs the forward
// pass, the BCE-with-logits loss and the backward pass in shared memory, and adds the tile's
// parameter gradients (and loss) to its own row of `part` in tile order.  Weights sit in shared
// memory (W2 also transposed, so both passes read it without bank conflicts); W1 too when it fits.
// Per-sample quantities: dz = (sigmoid(z) - y)/B is the gradient of the batch-mean loss.
__host__ __device__ inline size_t train_smem_floats(const MlpShape &sh, int SB, bool w1_smem) {
  const size_t H = sh.H, ni = sh.n_in;
  return (w1_smem ? H * ni : 0) + 2 * H * H + 4 * H + 1       // W1, W2, W2^T, b1, b2, w3, b3
         + (size_t)SB * ni + 6 * (size_t)SB * H + 3 * (size_t)SB;  // phi, a1 h1 a2 h2 da2 da1, z dz l
}

template <bool W1S>
__global__ void __launch_bounds__(256) k_mlp_train_tiles(MlpShape sh, const float *p, const int32_t *states,
                                                         const float *labels, int n, int start, int B, int SB,
                                                         float *part) {
  extern __shared__ __align__(16) float sm[];
  const int H = sh.H, ni = sh.n_in, np = sh.n_params();
  const int tid = threadIdx.x, nt = blockDim.x;
  float *w1 = sm;
  float *w2 = w1 + (W1S ? H * ni : 0);
  float *w2t = w2 + H * H;
  float *b1 = w2t + H * H, *b2 = b1 + H, *w3 = b2 + H, *b3 = w3 + H;
  float *phi = b3 + 1;
  float *a1 = phi + SB * ni, *h1 = a1 + SB * H, *a2 = h1 + SB * H, *h2 = a2 + SB * H;
  float *da2 = h2 + SB * H, *da1 = da2 + SB * H;
  float *zs = da1 + SB * H, *dz = zs + SB, *ls = dz + SB;
  const float *gw1 = W1S ? w1 : p + sh.o_w1();
  if (W1S)
    for (int i = tid; i < H * ni; i += nt) w1[i] = p[sh.o_w1() + i];
  for (int i = tid; i < H * H; i += nt) {
    const float v = p[sh.o_w2() + i];
    w2[i] = v;
    w2t[(i % H) * H + i / H] = v;
  }
  for (int i = tid; i < H; i += nt) { b1[i] = p[sh.o_b1() + i]; b2[i] = p[sh.o_b2() + i]; w3[i] = p[sh.o_w3() + i]; }
  if (tid == 0) b3[0] = p[sh.o_b3()];
  float *row = part + (size_t)blockIdx.x * (np + 1);
  const int n_tiles = (B + SB - 1) / SB;
  bool first = true;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int nb = min(SB, B - tile * SB);
    __syncthreads();
    for (int q = tid; q < nb * ni; q += nt) {
      const int j = q / ni, i = q - j * ni;
      const int s = (int)(((long long)start + (long long)tile * SB + j) % n);
      phi[j * ni + i] = log1pf((float)states[(size_t)s * ni + i]);
    }
    __syncthreads();
    for (int q = tid; q < nb * H; q += nt) {                  // layer 1
      const int j = q / H, o = q - j * H;
      float a = b1[o];
      for (int i = 0; i < ni; ++i) a = __fmaf_rn(gw1[o * ni + i], phi[j * ni + i], a);
      a1[q] = a;
      h1[q] = silu_f(a);
    }
    __syncthreads();
    for (int q = tid; q < nb * H; q += nt) {                  // layer 2
      const int j = q / H, o = q - j * H;
      float a = b2[o];
      for (int i = 0; i < H; ++i) a = __fmaf_rn(w2t[i * H + o], h1[j * H + i], a);
      a2[q] = a;
      h2[q] = silu_f(a);
    }
    __syncthreads();
    for (int j = tid; j < nb; j += nt) {                      // output, loss, dz
      float z = b3[0];
      for (int o = 0; o < H; ++o) z = __fmaf_rn(w3[o], h2[j * H + o], z);
      const int s = (int)(((long long)start + (long long)tile * SB + j) % n);
      const float y = labels[s];
      zs[j] = z;
      ls[j] = __fdiv_rn(__fadd_rn(__fsub_rn(fmaxf(z, 0.0f), __fmul_rn(z, y)), log1pf(expf(-fabsf(z)))), (float)B);
      dz[j] = __fdiv_rn(__fsub_rn(sigmoid_f(z), y), (float)B);
    }
    __syncthreads();
    for (int q = tid; q < nb * H; q += nt) {                  // da2
      const int j = q / H, o = q - j * H;
      da2[q] = __fmul_rn(__fmul_rn(dz[j], w3[o]), dsilu_f(a2[q]));
    }
    __syncthreads();
    for (int q = tid; q < nb * H; q += nt) {                  // da1
      const int j = q / H, i = q - j * H;
      float g = 0.0f;
      for (int o = 0; o < H; ++o) g = __fmaf_rn(da2[j * H + o], w2[o * H + i], g);
      da1[q] = __fmul_rn(g, dsilu_f(a1[q]));
    }
    __syncthreads();
    // parameter gradients of the tile, summed over its samples in order, added to the row
    for (int k = tid; k <= np; k += nt) {
      float g = 0.0f;
      if (k < sh.o_b1()) {
        const int o = k / ni, i = k - o * ni;
        for (int j = 0; j < nb; ++j) g = __fmaf_rn(da1[j * H + o], phi[j * ni + i], g);
      } else if (k < sh.o_w2()) {
        const int o = k - sh.o_b1();
        for (int j = 0; j < nb; ++j) g = __fadd_rn(g, da1[j * H + o]);
      } else if (k < sh.o_b2()) {
        const int q = k - sh.o_w2(), o = q / H, i = q - o * H;
        for (int j = 0; j < nb; ++j) g = __fmaf_rn(da2[j * H + o], h1[j * H + i], g);
      } else if (k < sh.o_w3()) {
        const int o = k - sh.o_b2();
        for (int j = 0; j < nb; ++j) g = __fadd_rn(g, da2[j * H + o]);
      } else if (k < sh.o_b3()) {
        const int o = k - sh.o_w3();
        for (int j = 0; j < nb; ++j) g = __fmaf_rn(dz[j], h2[j * H + o], g);
      } else if (k < np) {
        for (int j = 0; j < nb; ++j) g = __fadd_rn(g, dz[j]);
      } else {
        for (int j = 0; j < nb; ++j) g = __fadd_rn(g, ls[j]);
      }
      row[k] = first ? g : __fadd_rn(row[k], g);
    }
    first = false;
  }
  if (first)                                                   // a block without tiles
    for (int k = tid; k <= np; k += nt) row[k] = 0.0f;
}

// Training step, kernel 2 of 2: one thread per parameter sums the blocks' rows in block order
// (deterministic), then writes the gradient (grad != null) or applies Adam (step t >= 1).  The
// extra index np is the loss.
__global__ void k_mlp_reduce(MlpShape sh, float *p, float *m, float *v, int rows, const float *part,
                             float *grad, float *loss, float lr, float b1, float b2, float eps, int t) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int np = sh.n_params();
  if (k > np) return;
  float g = 0.0f;
  for (int r = 0; r < rows; ++r) g = __fadd_rn(g, part[(size_t)r * (np + 1) + k]);
  if (k == np) { if (loss) *loss = g; return; }
  if (grad) { grad[k] = g; return; }
  const float mk = __fmaf_rn(b1, m[k], __fmul_rn(1.0f - b1, g));
  const float vk = __fmaf_rn(b2, v[k], __fmul_rn(__fmul_rn(1.0f - b2, g), g));
  m[k] = mk;
  v[k] = vk;
  const float mh = __fdiv_rn(mk, 1.0f - powf(b1, (float)t));
  const float vh = __fdiv_rn(vk, 1.0f - powf(b2, (float)t));
  p[k] = __fsub_rn(p[k], __fdiv_rn(__fmul_rn(lr, mh), __fadd_rn(sqrtf(vh), eps)));
}

// Round a float to the nearest BF16 value (ties to even), returned as a float.
__device__ __forceinline__ float bf16_round_dev(float f) {
  uint32_t u = __float_as_uint(f);
  if ((u & 0x7f800000u) == 0x7f800000u) return f;
  u += 0x7fffu + ((u >> 16) & 1u);
  return __uint_as_float(u & 0xffff0000u);
}

// z of samples from the FP32 master weights, or from their BF16 roundings (BF16 = true), in the
// operation order of mlp_coordinate, so that the BF16 form equals the binning kernel's z.
template <bool BF16>
__global__ void k_mlp_forward(MlpShape sh, const float *p, const int32_t *states, int n, float *z) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  const int H = sh.H, ni = sh.n_in;
  auto wt = [](float w) { return BF16 ? bf16_round_dev(w) : w; };
  float h1[64];
#pragma unroll
  for (int o = 0; o < 64; ++o) h1[o] = 0.0f;
  for (int i = 0; i < ni; ++i) {
    const float phi = log1pf((float)states[(size_t)b * ni + i]);
#pragma unroll
    for (int o = 0; o < 64; ++o)
      if (o < H) h1[o] = __fmaf_rn(wt(p[sh.o_w1() + o * ni + i]), phi, h1[o]);
  }
#pragma unroll
  for (int o = 0; o < 64; ++o)
    if (o < H) h1[o] = silu_f(__fadd_rn(h1[o], p[sh.o_b1() + o]));
  float zz = p[sh.o_b3()];
  for (int o = 0; o < H; ++o) {
    float a = p[sh.o_b2() + o];
#pragma unroll
    for (int i = 0; i < 64; ++i)
      if (i < H) a = __fmaf_rn(wt(p[sh.o_w2() + o * H + i]), h1[i], a);
    zz = __fmaf_rn(wt(p[sh.o_w3() + o]), silu_f(a), zz);
  }
  z[b] = zz;
}

// z of every live walker after the SSA kernel, its bin and the bin counts (learned bin maps).
__global__ void k_learned_bins(PropagateParams prm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const EnsView &E = prm.ens;
  const BinView &bv = prm.bins;
  const MlpView &m = bv.mlp;
  const int H = m.hidden, ni = m.n_in;
  uint16_t *w1 = reinterpret_cast<uint16_t *>(smem_raw);
  uint16_t *w2 = w1 + H * ni;
  uint16_t *w3 = w2 + H * H;
  float *bb = reinterpret_cast<float *>(reinterpret_cast<uintptr_t>(w3 + H + 1) & ~(uintptr_t)3);
  for (int i = threadIdx.x; i < H * ni; i += blockDim.x) w1[i] = m.w1[i];
  for (int i = threadIdx.x; i < H * H; i += blockDim.x) w2[i] = m.w2[i];
  for (int i = threadIdx.x; i < H; i += blockDim.x) { w3[i] = m.w3[i]; bb[i] = m.b1[i]; bb[H + i] = m.b2[i]; }
  if (threadIdx.x == 0) bb[2 * H] = m.b3[0];
  __syncthreads();
  MlpView ms = m;
  ms.w1 = w1; ms.w2 = w2; ms.w3 = w3; ms.b1 = bb; ms.b2 = bb + H; ms.b3 = bb + 2 * H;
  const int iter = *E.iter;
  const int par = iter & 1;
  const int ld = E.R * E.cap;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ld; g += gridDim.x * blockDim.x) {
    const int r = g / E.cap, w = g - r * E.cap;
    if (w >= E.count[r]) continue;
    const float z = mlp_coordinate(ms, E.x[par] + g, ld);
    const int b = z_bin(bv, z);
    E.bin[g] = b;
    if (bv.zout) bv.zout[g] = z;
    if (prm.resample) atomicAdd(&E.bin_count[r * bv.n_bins + b], 1);
  }
}

size_t learned_bins_smem(int n_in, int H) { return 2 * ((size_t)H * n_in + H * H + H + 2) + 4 * (2 * H + 1) + 16; }

cudaError_t launch_learned_bins(const PropagateParams &prm, cudaStream_t st) {
  const size_t smem = learned_bins_smem(prm.bins.mlp.n_in, prm.bins.mlp.hidden);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_learned_bins, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int ld = prm.ens.R * prm.ens.cap;
  int grid = (ld + 127) / 128;
  if (grid > 152 * 4) grid = 152 * 4;
  k_learned_bins<<<grid, 128, smem, st>>>(prm);
  return cudaGetLastError();
}

}  // namespace we

using namespace we;

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
struct we_mlp {
  MlpShape sh{};
  float *p = nullptr, *m = nullptr, *v = nullptr;   // device: params, Adam moments
  int step = 0;
};

static uint16_t f32_to_bf16_rne(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)((u >> 16) | ((u & 0xffffu) ? 0x40u : 0u));
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  return (uint16_t)(u >> 16);
}

extern "C" we_status we_mlp_create(int32_t n_in, int32_t hidden, const float *params, we_mlp **out) {
  if (!out) return WE_EINVAL;
  *out = nullptr;
  if (n_in < 1 || n_in > 4096 || hidden < 1 || hidden > 64 || !params) return WE_EINVAL;
  we_mlp *M = new (std::nothrow) we_mlp();
  if (!M) return WE_ENOMEM;
  M->sh.n_in = n_in;
  M->sh.H = hidden;
  const size_t np = (size_t)M->sh.n_params();
  if (cudaMalloc(&M->p, 4 * np) || cudaMalloc(&M->m, 4 * np) || cudaMalloc(&M->v, 4 * np)) {
    cudaGetLastError();
    cudaFree(M->p); cudaFree(M->m); cudaFree(M->v);
    delete M;
    return WE_ENOMEM;
  }
  cudaError_t e = cudaMemcpy(M->p, params, 4 * np, cudaMemcpyHostToDevice);
  e = e ? e : cudaMemset(M->m, 0, 4 * np);
  e = e ? e : cudaMemset(M->v, 0, 4 * np);
  if (e) { cudaGetLastError(); cudaFree(M->p); cudaFree(M->m); cudaFree(M->v); delete M; return WE_ECUDA; }
  *out = M;
  return WE_OK;
}

extern "C" void we_mlp_destroy(we_mlp *M) {
  if (!M) return;
  cudaFree(M->p); cudaFree(M->m); cudaFree(M->v);
  delete M;
}

extern "C" int32_t we_mlp_n_params(const we_mlp *M) { return M ? M->sh.n_params() : 0; }

extern "C" we_status we_mlp_get_params(const we_mlp *M, float *dst, size_t dst_floats) {
  if (!M || !dst || dst_floats < (size_t)M->sh.n_params()) return WE_EINVAL;
  if (cudaMemcpy(dst, M->p, 4 * (size_t)M->sh.n_params(), cudaMemcpyDeviceToHost)) { cudaGetLastError(); return WE_ECUDA; }
  return WE_OK;
}

// Launch shape of the training kernels: samples per tile, W1 placement, shared memory, grid.
struct TrainPlan {
  int SB = 32;
  bool w1_smem = true;
  size_t smem = 0;
  int grid = 0;
};

static TrainPlan plan_training(const MlpShape &sh, int B) {
  const size_t limit = 200 * 1024;
  TrainPlan tp;
  for (int SB = 32; SB >= 8; SB >>= 1) {
    for (int w1 = 1; w1 >= 0; --w1) {
      const size_t bytes = 4 * train_smem_floats(sh, SB, w1 != 0);
      if (bytes <= limit) { tp.SB = SB; tp.w1_smem = w1 != 0; tp.smem = bytes; goto done; }
    }
  }
  tp.SB = 8; tp.w1_smem = false; tp.smem = 4 * train_smem_floats(sh, 8, false);
done:
  const int tiles = (B + tp.SB - 1) / tp.SB;
  tp.grid = tiles < 2 * 152 ? tiles : 2 * 152;
  return tp;
}

static cudaError_t launch_train_tiles(const TrainPlan &tp, const MlpShape &sh, const float *p,
                                      const int32_t *states, const float *labels, int n, int start, int B,
                                      float *part, cudaStream_t st) {
  cudaError_t e;
  if (tp.w1_smem) {
    e = cudaFuncSetAttribute(k_mlp_train_tiles<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tp.smem);
    if (e) return e;
    k_mlp_train_tiles<true><<<tp.grid, 256, tp.smem, st>>>(sh, p, states, labels, n, start, B, tp.SB, part);
  } else {
    e = cudaFuncSetAttribute(k_mlp_train_tiles<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tp.smem);
    if (e) return e;
    k_mlp_train_tiles<false><<<tp.grid, 256, tp.smem, st>>>(sh, p, states, labels, n, start, B, tp.SB, part);
  }
  return cudaGetLastError();
}

extern "C" we_status we_mlp_gradient(const we_mlp *M, const int32_t *states, const float *labels,
                                     int32_t n, float *grad, float *loss, void *stream) {
  if (!M || !states || !labels || n < 1 || !grad || !loss) return WE_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const TrainPlan tp = plan_training(M->sh, n);
  const int np = M->sh.n_params();
  float *part = nullptr;
  if (cudaMalloc(&part, 4 * ((size_t)tp.grid * (np + 1) + 1))) { cudaGetLastError(); return WE_ENOMEM; }
  float *dloss = part + (size_t)tp.grid * (np + 1);
  cudaError_t e = launch_train_tiles(tp, M->sh, M->p, states, labels, n, 0, n, part, st);
  if (!e) {
    k_mlp_reduce<<<(np + 1 + 127) / 128, 128, 0, st>>>(M->sh, M->p, M->m, M->v, tp.grid, part, grad, dloss,
                                                      0.f, 0.f, 0.f, 0.f, 0);
    e = cudaGetLastError();
  }
  e = e ? e : cudaMemcpyAsync(loss, dloss, 4, cudaMemcpyDeviceToHost, st);
  e = e ? e : cudaStreamSynchronize(st);
  cudaFree(part);
  if (e) { cudaGetLastError(); return WE_ECUDA; }
  return WE_OK;
}

extern "C" we_status we_mlp_forward(const we_mlp *M, const int32_t *states, int32_t n, int32_t bf16,
                                    float *z, void *stream) {
  if (!M || n < 0 || (n > 0 && (!states || !z))) return WE_EINVAL;
  if (n == 0) return WE_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (bf16) k_mlp_forward<true><<<(n + 127) / 128, 128, 0, st>>>(M->sh, M->p, states, n, z);
  else k_mlp_forward<false><<<(n + 127) / 128, 128, 0, st>>>(M->sh, M->p, states, n, z);
  cudaError_t e = cudaGetLastError();
  e = e ? e : cudaStreamSynchronize(st);
  if (e) { cudaGetLastError(); return WE_ECUDA; }
  return WE_OK;
}

extern "C" we_status we_mlp_train(we_mlp *M, const int32_t *states, const float *labels, int32_t n,
                                  int32_t steps, int32_t batch, float lr, float *loss_per_step,
                                  void *stream) {
  if (!M || !states || !labels || n < 1 || steps < 0 || batch < 1 || !(lr > 0.0f)) return WE_EINVAL;
  if (batch > n) batch = n;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const TrainPlan tp = plan_training(M->sh, batch);
  const int np = M->sh.n_params();
  float *part = nullptr;
  if (cudaMalloc(&part, 4 * ((size_t)tp.grid * (np + 1) + (size_t)(steps > 0 ? steps : 1)))) {
    cudaGetLastError();
    return WE_ENOMEM;
  }
  float *dloss = part + (size_t)tp.grid * (np + 1);
  cudaError_t e = cudaSuccess;
  for (int it = 0; it < steps && !e; ++it) {
    const int start = (int)(((long long)it * batch) % n);
    e = launch_train_tiles(tp, M->sh, M->p, states, labels, n, start, batch, part, st);
    if (e) break;
    M->step += 1;
    k_mlp_reduce<<<(np + 1 + 127) / 128, 128, 0, st>>>(M->sh, M->p, M->m, M->v, tp.grid, part, nullptr,
                                                      dloss + it, lr, 0.9f, 0.999f, 1e-8f, M->step);
    e = cudaGetLastError();
  }
  if (loss_per_step && steps > 0 && !e)
    e = cudaMemcpyAsync(loss_per_step, dloss, 4 * (size_t)steps, cudaMemcpyDeviceToHost, st);
  e = e ? e : cudaStreamSynchronize(st);
  cudaFree(part);
  if (e) { cudaGetLastError(); return WE_ECUDA; }
  return WE_OK;
}

// Learned bin map: a BF16 snapshot of the MLP's current weights plus bin edges on z.
we_status make_learned_snapshot(const we_mlp *M, int32_t n_bins, const float *edges, we_learned_bins *L) {
  if (!M || n_bins < 1 || n_bins > 65536 || !edges) return WE_EINVAL;
  for (int k = 0; k < n_bins; ++k)
    if (!(edges[k + 1] > edges[k])) return WE_EINVAL;
  const MlpShape sh = M->sh;
  std::vector<float> p(sh.n_params());
  if (cudaMemcpy(p.data(), M->p, 4 * p.size(), cudaMemcpyDeviceToHost)) { cudaGetLastError(); return WE_ECUDA; }
  L->n_in = sh.n_in; L->H = sh.H; L->n_bins = n_bins;
  L->w1.resize((size_t)sh.H * sh.n_in); L->w2.resize((size_t)sh.H * sh.H); L->w3.resize(sh.H);
  for (size_t i = 0; i < L->w1.size(); ++i) L->w1[i] = f32_to_bf16_rne(p[sh.o_w1() + i]);
  for (size_t i = 0; i < L->w2.size(); ++i) L->w2[i] = f32_to_bf16_rne(p[sh.o_w2() + i]);
  for (int i = 0; i < sh.H; ++i) L->w3[i] = f32_to_bf16_rne(p[sh.o_w3() + i]);
  L->b1.assign(p.begin() + sh.o_b1(), p.begin() + sh.o_b1() + sh.H);
  L->b2.assign(p.begin() + sh.o_b2(), p.begin() + sh.o_b2() + sh.H);
  L->b3.assign(1, p[sh.o_b3()]);
  L->zedges.assign(edges, edges + n_bins + 1);
  return WE_OK;
}
