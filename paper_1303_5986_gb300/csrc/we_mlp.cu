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
//     k_learned_bins a block per tile of 128 walkers after the SSA kernel: the first layer on
//                    the CUDA cores (one walker per thread), the 64 x 64 layer on the tensor
//                    cores (tcgen05, accumulator in tensor memory), then z, its bin, bin counts
//     k_mlp_forward_tc the same tile computation for given states (the standalone BF16 forward)
//   The tensor cores take BF16 operands: each activation of the first layer is split into three
//   BF16 parts (h = h0 + h1 + h2 to about 2^-26 relative) and each part is multiplied by the
//   BF16 weights into the same FP32 accumulator, so the layer keeps FP32-level accuracy.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/we_ssa.h"
#include "we_mlp.cuh"
#include "we_ssa_common.cuh"
#include "we_tc.cuh"

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

// z of samples from the FP32 master weights, FP32 arithmetic on the CUDA cores (the reference
// form of the trained network; the BF16 inference form is k_mlp_forward_tc).
__global__ void k_mlp_forward(MlpShape sh, const float *p, const int32_t *states, int n, float *z) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  const int H = sh.H, ni = sh.n_in;
  auto wt = [](float w) { return w; };
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

// ------------------------------------------------------------------------------------------
// Tensor-core inference.  Dynamic shared memory of a 128-thread block:
//   [0, 48 KB)     three A tiles (parts 0, 1, 2 of the activations): 128 samples x 64, BF16,
//                  core-matrix layout, 16 KB each; reused chunk by chunk for the inputs of the
//                  first layer when that layer runs on the tensor cores
//   [48, 56 KB)    B tile: W2 (64 x 64, zero beyond H), BF16, core-matrix layout
//   [56 KB, +16)   mbarrier, tensor-memory address
//   [57 KB, ...)   first layer on the CUDA cores (few inputs): W1 (H x n_in) as BF16;
//                  on the tensor cores (n_in >= kTcLayer1MinInputs): W1 as ceil(n_in / 64)
//                  B tiles of 64 x 64 (8 KB each, inputs 64c .. 64c+63, zero-padded);
//                  then w3 (H) as BF16 and b1, b2 (H each), b3 as FP32
// Tensor memory: 128 columns; the second layer's accumulator at column 0, the first layer's at
// column 64.
// ------------------------------------------------------------------------------------------
constexpr int kTcTile = 128;
constexpr size_t kTcWeightsOff = 57 * 1024;
constexpr int kTcParts = 3;
constexpr long kTcWaitLimit = 1l << 24;
constexpr int kTcLayer1MinInputs = 32;     // below this the CUDA-core first layer is cheaper

__host__ __device__ inline bool tc_layer1(int n_in) { return n_in >= kTcLayer1MinInputs; }
__host__ __device__ inline int tc_chunks(int n_in) { return (n_in + 63) / 64; }

size_t tc_mlp_smem(int n_in, int H) {
  const size_t w1 = tc_layer1(n_in) ? (size_t)tc_chunks(n_in) * 8192 : 2 * (size_t)H * n_in;
  return kTcWeightsOff + w1 + 2 * (size_t)H + 8 + 4 * (2 * (size_t)H + 1) + 16;
}

struct TcMlp {
  unsigned char *a, *b;          // A tiles (kTcParts x 16 KB), B tile
  unsigned char *b1;             // first-layer B tiles (tensor-core first layer), else null
  int n_chunks;
  uint64_t *mbar;
  uint32_t *slot;
  uint32_t phase;                // mbarrier phases completed so far
  MlpView m;                     // weights and biases in shared memory
};

// Carve the shared memory, stage the BF16 weights (w1, w2, w3 given as BF16 bits) and biases,
// fill the B tiles, allocate 128 tensor-memory columns (warp 0) and initialise the mbarrier.
__device__ TcMlp tc_mlp_setup(unsigned char *sm, int n_in, int H, const uint16_t *w1, const uint16_t *w2,
                              const uint16_t *w3, const float *b1, const float *b2, const float *b3) {
  TcMlp T;
  T.a = sm;
  T.b = sm + 49152;
  T.mbar = reinterpret_cast<uint64_t *>(sm + 57344);
  T.slot = reinterpret_cast<uint32_t *>(sm + 57352);
  T.phase = 0;
  const bool tc1 = tc_layer1(n_in);
  T.n_chunks = tc1 ? tc_chunks(n_in) : 0;
  uint16_t *sw1 = reinterpret_cast<uint16_t *>(sm + kTcWeightsOff);
  T.b1 = tc1 ? sm + kTcWeightsOff : nullptr;
  uint16_t *sw3 = tc1 ? reinterpret_cast<uint16_t *>(sm + kTcWeightsOff + (size_t)T.n_chunks * 8192)
                      : sw1 + (size_t)H * n_in;
  float *sb = reinterpret_cast<float *>(reinterpret_cast<uintptr_t>(sw3 + H + 3) & ~(uintptr_t)7);
  if (tc1) {
    for (int e = threadIdx.x; e < T.n_chunks * 64 * 64; e += blockDim.x) {
      const int c = e >> 12, n = (e >> 6) & 63, k = e & 63, i = c * 64 + k;
      *reinterpret_cast<uint16_t *>(T.b1 + (size_t)c * 8192 + tc_tile_offset(n, k)) =
          (n < H && i < n_in) ? w1[(size_t)n * n_in + i] : (uint16_t)0;
    }
  } else {
    for (int i = threadIdx.x; i < H * n_in; i += blockDim.x) sw1[i] = w1[i];
  }
  for (int i = threadIdx.x; i < H; i += blockDim.x) { sw3[i] = w3[i]; sb[i] = b1[i]; sb[H + i] = b2[i]; }
  if (threadIdx.x == 0) sb[2 * H] = b3[0];
  for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
    const int n = e >> 6, k = e & 63;
    *reinterpret_cast<uint16_t *>(T.b + tc_tile_offset(n, k)) = (n < H && k < H) ? w2[n * H + k] : (uint16_t)0;
  }
  if (threadIdx.x == 0) tc_mbar_init(T.mbar, 1);
  if (threadIdx.x < 32) tc_alloc(T.slot, 128);
  tc_fence_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  T.m.n_in = n_in;
  T.m.hidden = H;
  T.m.w1 = tc1 ? nullptr : sw1;
  T.m.w2 = nullptr;
  T.m.w3 = sw3;
  T.m.b1 = sb;
  T.m.b2 = sb + H;
  T.m.b3 = sb + 2 * H;
  return T;
}

// Free the tensor memory.  After a timed-out wait (ok = false) one more bounded wait lets the
// MMAs still in flight finish before their accumulator is released.
__device__ __forceinline__ void tc_mlp_teardown(TcMlp &T, bool ok) {
  if (!ok) {
    const bool late = tc_mbar_wait(T.mbar, T.phase & 1u, kTcWaitLimit);
    __syncthreads_or(late ? 1 : 0);
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) tc_dealloc(*T.slot, 128);
}

// The next mbarrier phase, every thread waiting at most kTcWaitLimit polls; false (for every
// thread) if it did not complete.  On success the phase counter advances.
__device__ __forceinline__ bool tc_wait_phase(TcMlp &T) {
  const bool done = __syncthreads_and(tc_mbar_wait(T.mbar, T.phase & 1u, kTcWaitLimit) ? 1 : 0) != 0;
  tc_fence_after();
  if (done) T.phase += 1;
  return done;
}

// Split 8 FP32 values into kTcParts BF16 parts (part q+1 = BF16 of what parts 0..q leave over;
// their sum equals the value to ~2^-26 relative) and store them as row t, columns col..col+7 of
// the three A tiles.
__device__ __forceinline__ void tc_store_parts(unsigned char *a, int t, int col, const float (&v)[8]) {
  uint32_t pw[kTcParts][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float ra = v[2 * j], rb = v[2 * j + 1];
#pragma unroll
    for (int q = 0; q < kTcParts; ++q) {
      const float pa = bf16_round_dev(ra), pb = bf16_round_dev(rb);
      pw[q][j] = (__float_as_uint(pa) >> 16) | (__float_as_uint(pb) & 0xffff0000u);
      ra = __fsub_rn(ra, pa);                                       // exact
      rb = __fsub_rn(rb, pb);
    }
  }
#pragma unroll
  for (int q = 0; q < kTcParts; ++q)
    *reinterpret_cast<uint4 *>(a + q * 16384 + tc_tile_offset(t, col)) = make_uint4(pw[q][0], pw[q][1], pw[q][2], pw[q][3]);
}

// thread 0: D (tensor memory at taddr) (+)= sum over the three A parts of part . B^T, K = 64
__device__ __forceinline__ void tc_issue_parts(const TcMlp &T, uint32_t taddr, const unsigned char *btile, bool acc) {
  tc_fence_after();
  constexpr uint32_t idesc = tc_idesc_bf16(kTcTile, 64);
  const uint32_t aa = tc_smem_addr(T.a), bb = tc_smem_addr(btile);
#pragma unroll
  for (int part = 0; part < kTcParts; ++part)
#pragma unroll
    for (int kc = 0; kc < 4; ++kc)
      tc_mma_bf16(taddr, tc_desc(aa + 16384 * part + 256 * kc, 128, 1024), tc_desc(bb + 256 * kc, 128, 1024),
                  idesc, acc || part > 0 || kc > 0);
  tc_commit(T.mbar);
}

// One tile: thread t holds sample t (valid or not).  First layer: on the tensor cores for
// n_in >= kTcLayer1MinInputs (phi = log1p x of 64 inputs at a time split into three BF16 parts
// in the A tiles, times the W1 chunk, accumulated in tensor memory column 64 on; then
// h1 = silu(acc + b1)), else on the CUDA cores.  Second layer: the activations split into three
// BF16 parts in the A tiles, thread 0 issues part_p . W2^T for p = 0, 1, 2 (K = 16 per
// instruction) into one 128 x 64 FP32 accumulator at column 0; every thread reads its
// accumulator row and finishes z = b3 + sum_o w3_o silu(acc_o + b2_o).  Returns false (for
// every thread) if the tensor core did not complete in time; z is then NaN and the caller
// issues no further tile.
__device__ bool tc_mlp_tile(TcMlp &T, const int32_t *xs, int stride, bool valid, float &z) {
  const int t = threadIdx.x;
  const int H = T.m.hidden;
  const uint32_t taddr = *T.slot;
  z = __int_as_float(0x7fc00000);
  float h1[64];
  if (T.n_chunks > 0) {
    const int n_in = T.m.n_in;
    for (int c = 0; c < T.n_chunks; ++c) {
#pragma unroll 1
      for (int kg = 0; kg < 8; ++kg) {
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = c * 64 + kg * 8 + q;
          v[q] = (valid && i < n_in) ? log1pf((float)xs[(size_t)i * stride]) : 0.0f;
        }
        tc_store_parts(T.a, t, kg * 8, v);
      }
      tc_fence_smem();
      __syncthreads();
      if (t == 0) tc_issue_parts(T, taddr + 64, T.b1 + (size_t)c * 8192, c > 0);
      if (!tc_wait_phase(T)) return false;
    }
    float acc[64];
    tc_ld_row64(taddr + 64, acc);
#pragma unroll
    for (int o = 0; o < 64; ++o) h1[o] = (o < H) ? silu_f(__fadd_rn(acc[o], T.m.b1[o])) : 0.0f;
  } else {
    mlp_layer1(T.m, xs, stride, valid, h1);
  }
#pragma unroll
  for (int kg = 0; kg < 8; ++kg) {
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = h1[kg * 8 + q];
    tc_store_parts(T.a, t, kg * 8, v);
  }
  tc_fence_smem();
  __syncthreads();
  if (t == 0) tc_issue_parts(T, taddr, T.b, false);
  if (!tc_wait_phase(T)) return false;
  float acc[64];
  tc_ld_row64(taddr, acc);
  float zz = T.m.b3[0];
#pragma unroll
  for (int o = 0; o < 64; ++o)
    if (o < H) zz = __fmaf_rn(bf16_to_f32(T.m.w3[o]), silu_f(__fadd_rn(acc[o], T.m.b2[o])), zz);
  z = zz;
  tc_fence_before();
  __syncthreads();                                    // A tiles and the accumulators free again
  return true;
}

// z of every live walker after the SSA kernel, its bin and the bin counts (learned bin maps):
// tiles of 128 live walkers in run order, a persistent grid.
__global__ void __launch_bounds__(128) k_learned_bins(PropagateParams prm) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const EnsView &E = prm.ens;
  const BinView &bv = prm.bins;
  const MlpView &m = bv.mlp;
  TcMlp T = tc_mlp_setup(smem_raw, m.n_in, m.hidden, m.w1, m.w2, m.w3, m.b1, m.b2, m.b3);
  const int par = (*E.iter) & 1;
  const int ld = E.R * E.cap;
  const int total = E.run_off[E.R];
  bool ok = true;
  for (int base = blockIdx.x * kTcTile; base < total && ok; base += gridDim.x * kTcTile) {
    const int f = base + (int)threadIdx.x;
    const bool valid = f < total;
    const int r = !valid ? 0 : (E.R == 1 ? 0 : find_run(E.run_off, E.R, f));
    const int g = r * E.cap + (valid ? f - E.run_off[r] : 0);
    float z;
    ok = tc_mlp_tile(T, E.x[par] + g, ld, valid, z);
    if (!valid) continue;
    if (!ok) atomicCAS(&E.status[r], 0, WE_ETIMEOUT);   // this block issues no further tile
    const int b = ok ? z_bin(bv, z) : 0;
    E.bin[g] = b;
    if (bv.zout) bv.zout[g] = z;
    if (prm.resample) atomicAdd(&E.bin_count[r * bv.n_bins + b], 1);
  }
  tc_mlp_teardown(T, ok);
}

// The standalone BF16 forward pass of given states (walker-major, n x n_in) from the FP32 master
// weights rounded to BF16 here: the same tile computation, so z equals the binning kernel's.
__global__ void __launch_bounds__(128) k_mlp_forward_tc(MlpShape sh, const float *p, const int32_t *states, int n,
                                                        uint16_t *wbf, float *z, int32_t *status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int H = sh.H, ni = sh.n_in;
  TcMlp T = tc_mlp_setup(smem_raw, ni, H, wbf, wbf + (size_t)H * ni, wbf + (size_t)H * ni + H * H,
                         p + sh.o_b1(), p + sh.o_b2(), p + sh.o_b3());
  bool ok = true;
  for (int base = blockIdx.x * kTcTile; base < n && ok; base += gridDim.x * kTcTile) {
    const int b = base + (int)threadIdx.x;
    const bool valid = b < n;
    float zz;
    ok = tc_mlp_tile(T, states + (size_t)(valid ? b : 0) * ni, 1, valid, zz);
    if (valid) z[b] = zz;
  }
  if (!ok && threadIdx.x == 0) atomicCAS(status, 0, WE_ETIMEOUT);
  tc_mlp_teardown(T, ok);
}

// BF16 bits of the weights W1, W2, w3 (round to nearest even), packed in that order.
__global__ void k_mlp_weights_bf16(MlpShape sh, const float *p, uint16_t *out) {
  const int H = sh.H, ni = sh.n_in;
  const int n1 = H * ni, n2 = H * H;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n1 + n2 + H; i += gridDim.x * blockDim.x) {
    const float w = i < n1 ? p[sh.o_w1() + i] : (i < n1 + n2 ? p[sh.o_w2() + i - n1] : p[sh.o_w3() + i - n1 - n2]);
    out[i] = (uint16_t)(__float_as_uint(bf16_round_dev(w)) >> 16);
  }
}

size_t learned_bins_smem(int n_in, int H) { return tc_mlp_smem(n_in, H); }

cudaError_t launch_learned_bins(const PropagateParams &prm, cudaStream_t st) {
  const size_t smem = learned_bins_smem(prm.bins.mlp.n_in, prm.bins.mlp.hidden);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_learned_bins, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int ld = prm.ens.R * prm.ens.cap;
  int grid = (ld + kTcTile - 1) / kTcTile;
  if (grid > 152 * 2) grid = 152 * 2;
  k_learned_bins<<<grid, kTcTile, smem, st>>>(prm);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Order statistics of z (bin edges of a learned coordinate): radix select on order-preserving
// 32-bit keys of the floats, one 8-bit digit per pass from the top.  State: {prefix, mask, k}.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t float_key(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_float(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__global__ void k_radix_hist(const float *z, int n, const uint32_t *state, int shift, uint32_t *hist) {
  __shared__ uint32_t h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const uint32_t prefix = state[0], mask = state[1];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t k = float_key(z[i]);
    if ((k & mask) == prefix) atomicAdd(&h[(k >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

// One thread: the digit holding the k-th key among those matching the prefix; clears hist.
__global__ void k_radix_pick(uint32_t *state, int shift, uint32_t *hist) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint32_t k = state[2], cum = 0;
  int d = 255;
  for (int i = 0; i < 256; ++i) {
    if (cum + hist[i] > k) { d = i; break; }
    cum += hist[i];
  }
  state[0] |= (uint32_t)d << shift;
  state[1] |= 255u << shift;
  state[2] = k - cum;
  for (int i = 0; i < 256; ++i) hist[i] = 0;
}

// edges[i] = lo + (hi - lo) i / n_bins in double, rounded to float (hi = lo + 1 when hi <= lo)
__global__ void k_coordinate_edges(const uint32_t *st_lo, const uint32_t *st_hi, int n_bins, float *edges) {
  const double lo = (double)key_float(st_lo[0]);
  double hi = (double)key_float(st_hi[0]);
  if (!(hi > lo)) hi = lo + 1.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n_bins; i += gridDim.x * blockDim.x)
    edges[i] = (float)(lo + (hi - lo) * (double)i / (double)n_bins);
}

}  // namespace we

using namespace we;

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
struct we_mlp {
  MlpShape sh{};
  float *p = nullptr, *m = nullptr, *v = nullptr;   // device: params, Adam moments
  uint16_t *wbf = nullptr;                          // device: BF16 weights for the forward pass
  int32_t *status = nullptr;                        // device: WE_ETIMEOUT of the last BF16 forward pass
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
  const size_t nw = (size_t)hidden * n_in + (size_t)hidden * hidden + hidden;
  if (device_alloc((void **)&M->p, 4 * np) || device_alloc((void **)&M->m, 4 * np) ||
      device_alloc((void **)&M->v, 4 * np) || device_alloc((void **)&M->wbf, 2 * nw + 16)) {
    cudaGetLastError();
    cudaFree(M->p); cudaFree(M->m); cudaFree(M->v); cudaFree(M->wbf);
    delete M;
    return WE_ENOMEM;
  }
  M->status = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(M->wbf) + ((2 * nw + 3) & ~(size_t)3));
  cudaError_t e = cudaMemcpy(M->p, params, 4 * np, cudaMemcpyHostToDevice);
  e = e ? e : cudaMemset(M->m, 0, 4 * np);
  e = e ? e : cudaMemset(M->v, 0, 4 * np);
  if (e) {
    cudaGetLastError();
    cudaFree(M->p); cudaFree(M->m); cudaFree(M->v); cudaFree(M->wbf);
    delete M;
    return WE_ECUDA;
  }
  *out = M;
  return WE_OK;
}

// splitmix64 (Steele, Lea & Flood, OOPSLA 2014): the library's own initial weights
static uint64_t splitmix64(uint64_t &s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

extern "C" we_status we_mlp_create_init(int32_t n_in, int32_t hidden, uint64_t seed, we_mlp **out) {
  if (!out) return WE_EINVAL;
  *out = nullptr;
  if (n_in < 1 || n_in > 4096 || hidden < 1 || hidden > 64) return WE_EINVAL;
  MlpShape sh{};
  sh.n_in = n_in;
  sh.H = hidden;
  std::vector<float> p((size_t)sh.n_params(), 0.0f);
  uint64_t s = seed;
  auto fill = [&](int off, int count, int fan_in) {
    const double a = 1.0 / std::sqrt((double)fan_in);
    for (int i = 0; i < count; ++i) {
      const double u = (double)(splitmix64(s) >> 11) * 0x1p-53;        // [0, 1)
      p[(size_t)off + i] = (float)((2.0 * u - 1.0) * a);
    }
  };
  fill(sh.o_w1(), hidden * n_in, n_in);
  fill(sh.o_w2(), hidden * hidden, hidden);
  fill(sh.o_w3(), hidden, hidden);
  return we_mlp_create(n_in, hidden, p.data(), out);
}

extern "C" we_status we_mlp_coordinate_edges(const we_mlp *M, const int32_t *states, int32_t n, int32_t n_bins,
                                             double lo_q, float *edges, void *stream) {
  if (!M || !states || n < 1 || n_bins < 1 || n_bins > 65536 || !edges || !(lo_q >= 0.0) || !(lo_q <= 1.0))
    return WE_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float *z = nullptr;
  uint32_t *aux = nullptr;                     // state lo (3), state hi (3), hist (256)
  float *dedges = nullptr;
  if (device_alloc((void **)&z, 4 * (size_t)n) || device_alloc((void **)&aux, 4 * (6 + 256)) ||
      device_alloc((void **)&dedges, 4 * ((size_t)n_bins + 1))) {
    cudaGetLastError();
    cudaFree(z); cudaFree(aux); cudaFree(dedges);
    return WE_ENOMEM;
  }
  we_status rc = we_mlp_forward(M, states, n, 1, z, stream);
  const uint32_t k_lo = (uint32_t)std::floor(lo_q * (double)(n - 1));
  const uint32_t init[6] = {0u, 0u, k_lo, 0u, 0u, (uint32_t)(n - 1)};
  cudaError_t e = rc ? cudaSuccess : cudaMemcpyAsync(aux, init, sizeof(init), cudaMemcpyHostToDevice, st);
  e = e ? e : cudaMemsetAsync(aux + 6, 0, 4 * 256, st);
  int grid = (n + 255) / 256;
  if (grid > 152 * 4) grid = 152 * 4;
  for (int which = 0; which < 2 && !rc && !e; ++which) {
    uint32_t *state = aux + 3 * which;
    for (int shift = 24; shift >= 0 && !e; shift -= 8) {
      k_radix_hist<<<grid, 256, 0, st>>>(z, n, state, shift, aux + 6);
      k_radix_pick<<<1, 32, 0, st>>>(state, shift, aux + 6);
      e = cudaGetLastError();
    }
  }
  if (!rc && !e) {
    k_coordinate_edges<<<(n_bins + 256) / 256, 256, 0, st>>>(aux, aux + 3, n_bins, dedges);
    e = cudaGetLastError();
  }
  e = e ? e : cudaMemcpyAsync(edges, dedges, 4 * ((size_t)n_bins + 1), cudaMemcpyDefault, st);
  e = e ? e : cudaStreamSynchronize(st);
  cudaFree(z); cudaFree(aux); cudaFree(dedges);
  if (rc) return rc;
  if (e) { cudaGetLastError(); return WE_ECUDA; }
  return WE_OK;
}

extern "C" void we_mlp_destroy(we_mlp *M) {
  if (!M) return;
  cudaFree(M->p); cudaFree(M->m); cudaFree(M->v); cudaFree(M->wbf);
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
  if (device_alloc((void **)&part, 4 * ((size_t)tp.grid * (np + 1) + 1))) { cudaGetLastError(); return WE_ENOMEM; }
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
  cudaError_t e = cudaSuccess;
  int32_t st_h = 0;
  if (bf16) {
    const size_t smem = tc_mlp_smem(M->sh.n_in, M->sh.H);
    if (smem > 227 * 1024) return WE_ENOTSUPPORTED;
    k_mlp_weights_bf16<<<64, 256, 0, st>>>(M->sh, M->p, M->wbf);
    e = cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int grid = (n + kTcTile - 1) / kTcTile;
    if (grid > 152 * 2) grid = 152 * 2;
    e = e ? e : cudaMemsetAsync(M->status, 0, 4, st);
    if (!e) k_mlp_forward_tc<<<grid, kTcTile, smem, st>>>(M->sh, M->p, states, n, M->wbf, z, M->status);
    e = e ? e : cudaGetLastError();
    e = e ? e : cudaMemcpyAsync(&st_h, M->status, 4, cudaMemcpyDeviceToHost, st);
  } else {
    k_mlp_forward<<<(n + 127) / 128, 128, 0, st>>>(M->sh, M->p, states, n, z);
  }
  e = e ? e : cudaGetLastError();
  e = e ? e : cudaStreamSynchronize(st);
  if (e) { cudaGetLastError(); return WE_ECUDA; }
  return st_h ? st_h : WE_OK;
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
  if (device_alloc((void **)&part, 4 * ((size_t)tp.grid * (np + 1) + (size_t)(steps > 0 ? steps : 1)))) {
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
