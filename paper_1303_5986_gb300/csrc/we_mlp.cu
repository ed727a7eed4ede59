// we_mlp.cu -- a small MLP progress coordinate for WE binning (species counts -> log1p ->
// 64 -> 64 -> 1 with SiLU), trained by hand-written forward/backward kernels and used only to
// place bins.  WE is unbiased under any binning (Sec. II.B; adaptive or learned bins are the
// open problem of Sec. IV.B), so the learned coordinate changes efficiency, never the answer.
//
//   training (FP32 master weights):
//     k_mlp_sample   one thread per sample: forward pass, BCE-with-logits loss, and the
//                    backward pass down to per-sample activation gradients
//     k_mlp_params   one thread per parameter: batch sum of its gradient in sample order
//                    (deterministic), then an Adam step (or just the gradient, for checks)
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

// Per-sample scratch of a training batch (B x H each, sample-major) and phi (B x n_in).
struct MlpBatch {
  float *phi, *a1, *h1, *a2, *h2, *da1, *da2, *dz;
  float *loss;                    // one accumulator
};

// Forward pass and activation gradients of samples idx[b] (b < B).  dz = (sigmoid(z) - y)/B
// is the gradient of the batch-mean BCE-with-logits loss with respect to z.
__global__ void k_mlp_sample(MlpShape sh, const float *p, const int32_t *states, const float *labels,
                             int n, int start, int B, MlpBatch mb) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int H = sh.H, ni = sh.n_in;
  const int s = (start + b) % n;
  float *phi = mb.phi + (size_t)b * ni;
  for (int i = 0; i < ni; ++i) phi[i] = log1pf((float)states[(size_t)s * ni + i]);
  float *a1 = mb.a1 + (size_t)b * H, *h1 = mb.h1 + (size_t)b * H;
  float *a2 = mb.a2 + (size_t)b * H, *h2 = mb.h2 + (size_t)b * H;
  for (int o = 0; o < H; ++o) {
    float a = p[sh.o_b1() + o];
    for (int i = 0; i < ni; ++i) a = __fmaf_rn(p[sh.o_w1() + o * ni + i], phi[i], a);
    a1[o] = a;
    h1[o] = silu_f(a);
  }
  float z = p[sh.o_b3()];
  for (int o = 0; o < H; ++o) {
    float a = p[sh.o_b2() + o];
    for (int i = 0; i < H; ++i) a = __fmaf_rn(p[sh.o_w2() + o * H + i], h1[i], a);
    a2[o] = a;
    h2[o] = silu_f(a);
    z = __fmaf_rn(p[sh.o_w3() + o], h2[o], z);
  }
  const float y = labels[s];
  // BCE with logits: max(z,0) - z y + log(1 + exp(-|z|))
  const float l = __fadd_rn(__fsub_rn(fmaxf(z, 0.0f), __fmul_rn(z, y)), log1pf(expf(-fabsf(z))));
  atomicAdd(mb.loss, __fdiv_rn(l, (float)B));
  const float dz = __fdiv_rn(__fsub_rn(sigmoid_f(z), y), (float)B);
  mb.dz[b] = dz;
  float *da2 = mb.da2 + (size_t)b * H, *da1 = mb.da1 + (size_t)b * H;
  for (int o = 0; o < H; ++o) da2[o] = __fmul_rn(__fmul_rn(dz, p[sh.o_w3() + o]), dsilu_f(a2[o]));
  for (int i = 0; i < H; ++i) {
    float g = 0.0f;
    for (int o = 0; o < H; ++o) g = __fmaf_rn(da2[o], p[sh.o_w2() + o * H + i], g);
    da1[i] = __fmul_rn(g, dsilu_f(a1[i]));
  }
}

// One thread per parameter: its gradient summed over the batch in sample order, then either
// written out (grad != null) or applied with Adam (lr, beta1, beta2, eps; step t >= 1).
__global__ void k_mlp_params(MlpShape sh, float *p, float *m, float *v, int B, MlpBatch mb,
                             float *grad, float lr, float b1, float b2, float eps, int t) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int np = sh.n_params();
  if (k >= np) return;
  const int H = sh.H, ni = sh.n_in;
  float g = 0.0f;
  if (k < sh.o_b1()) {                                   // W1[o][i]
    const int o = k / ni, i = k - o * ni;
    for (int b = 0; b < B; ++b) g = __fmaf_rn(mb.da1[(size_t)b * H + o], mb.phi[(size_t)b * ni + i], g);
  } else if (k < sh.o_w2()) {                            // b1[o]
    const int o = k - sh.o_b1();
    for (int b = 0; b < B; ++b) g = __fadd_rn(g, mb.da1[(size_t)b * H + o]);
  } else if (k < sh.o_b2()) {                            // W2[o][i]
    const int q = k - sh.o_w2(), o = q / H, i = q - o * H;
    for (int b = 0; b < B; ++b) g = __fmaf_rn(mb.da2[(size_t)b * H + o], mb.h1[(size_t)b * H + i], g);
  } else if (k < sh.o_w3()) {                            // b2[o]
    const int o = k - sh.o_b2();
    for (int b = 0; b < B; ++b) g = __fadd_rn(g, mb.da2[(size_t)b * H + o]);
  } else if (k < sh.o_b3()) {                            // w3[o]
    const int o = k - sh.o_w3();
    for (int b = 0; b < B; ++b) g = __fmaf_rn(mb.dz[b], mb.h2[(size_t)b * H + o], g);
  } else {                                               // b3
    for (int b = 0; b < B; ++b) g = __fadd_rn(g, mb.dz[b]);
  }
  if (grad) { grad[k] = g; return; }
  const float mk = __fmaf_rn(b1, m[k], __fmul_rn(1.0f - b1, g));
  const float vk = __fmaf_rn(b2, v[k], __fmul_rn(__fmul_rn(1.0f - b2, g), g));
  m[k] = mk;
  v[k] = vk;
  const float mh = __fdiv_rn(mk, 1.0f - powf(b1, (float)t));
  const float vh = __fdiv_rn(vk, 1.0f - powf(b2, (float)t));
  p[k] = __fsub_rn(p[k], __fdiv_rn(__fmul_rn(lr, mh), __fadd_rn(sqrtf(vh), eps)));
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

// Batch workspace of B samples.
struct BatchMem {
  MlpBatch mb{};
  float *base = nullptr;
  we_status alloc(const MlpShape &sh, int B) {
    const size_t per = (size_t)B * (sh.n_in + 7 * sh.H + 1) + 4;
    if (cudaMalloc(&base, 4 * per)) { cudaGetLastError(); return WE_ENOMEM; }
    float *q = base;
    mb.phi = q; q += (size_t)B * sh.n_in;
    mb.a1 = q; q += (size_t)B * sh.H;
    mb.h1 = q; q += (size_t)B * sh.H;
    mb.a2 = q; q += (size_t)B * sh.H;
    mb.h2 = q; q += (size_t)B * sh.H;
    mb.da1 = q; q += (size_t)B * sh.H;
    mb.da2 = q; q += (size_t)B * sh.H;
    mb.dz = q; q += (size_t)B;
    mb.loss = q;
    return WE_OK;
  }
  ~BatchMem() { if (base) cudaFree(base); }
};

extern "C" we_status we_mlp_gradient(const we_mlp *M, const int32_t *states, const float *labels,
                                     int32_t n, float *grad, float *loss, void *stream) {
  if (!M || !states || !labels || n < 1 || !grad || !loss) return WE_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  BatchMem bm;
  we_status s = bm.alloc(M->sh, n);
  if (s) return s;
  cudaError_t e = cudaMemsetAsync(bm.mb.loss, 0, 4, st);
  k_mlp_sample<<<(n + 127) / 128, 128, 0, st>>>(M->sh, M->p, states, labels, n, 0, n, bm.mb);
  k_mlp_params<<<(M->sh.n_params() + 127) / 128, 128, 0, st>>>(M->sh, M->p, M->m, M->v, n, bm.mb, grad,
                                                               0.f, 0.f, 0.f, 0.f, 0);
  e = e ? e : cudaGetLastError();
  e = e ? e : cudaMemcpyAsync(loss, bm.mb.loss, 4, cudaMemcpyDeviceToHost, st);
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
  BatchMem bm;
  we_status s = bm.alloc(M->sh, batch);
  if (s) return s;
  std::vector<float> losses;
  float *dloss = nullptr;
  if (loss_per_step && steps > 0) {
    if (cudaMalloc(&dloss, 4 * (size_t)steps)) { cudaGetLastError(); return WE_ENOMEM; }
  }
  cudaError_t e = cudaSuccess;
  for (int it = 0; it < steps && !e; ++it) {
    const int start = (int)(((long long)it * batch) % n);
    e = cudaMemsetAsync(bm.mb.loss, 0, 4, st);
    k_mlp_sample<<<(batch + 127) / 128, 128, 0, st>>>(M->sh, M->p, states, labels, n, start, batch, bm.mb);
    M->step += 1;
    k_mlp_params<<<(M->sh.n_params() + 127) / 128, 128, 0, st>>>(M->sh, M->p, M->m, M->v, batch, bm.mb,
                                                                 nullptr, lr, 0.9f, 0.999f, 1e-8f, M->step);
    e = e ? e : cudaGetLastError();
    if (dloss && !e) e = cudaMemcpyAsync(dloss + it, bm.mb.loss, 4, cudaMemcpyDeviceToDevice, st);
  }
  if (dloss && !e) e = cudaMemcpyAsync(loss_per_step, dloss, 4 * (size_t)steps, cudaMemcpyDeviceToHost, st);
  e = e ? e : cudaStreamSynchronize(st);
  if (dloss) cudaFree(dloss);
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
