// we_reweight.cu -- steady-state reweighting of Bhatt et al. (Sec. II.B.2, Eq. "ss").
//
// In steady state each bin's inflow equals its outflow, sum_j (k_ij w_j - k_ji w_i) = 0, with
// f_ij = k_ij w_j the flux into bin i from bin j.  The rates come from the transfers measured
// over every interval so far: F_ij = weight that started an interval in bin j and ended it in
// bin i, W_j = sum_i F_ij, k_ij = F_ij / W_j.  Every reweight_period-th iteration, after the
// split/merge, the balance equations over the bins with W_j > 0 (the last replaced by
// sum_i w_i = 1) are solved, and the walkers of each bin that holds any are rescaled so that
// the bins carry the solved weights (their total unchanged).
//
//   k_rw_flux   (after the SSA, before the split/merge): one warp per bin of the previous
//               split/merge, whose M_targ walkers are consecutive slots; lane 0 sums their
//               weights by end bin in ascending slot order and adds each sum to F once.
//   k_rw_solve  (after the split/merge; one block per run): Gaussian elimination with partial
//               pivoting and column-oriented back substitution, every product and difference
//               rounded on its own (no fused multiply-add), so the factors are the same bits
//               as a sequential elimination in the same order.
//   k_rw_apply  multiplies each walker's weight by its bin's factor.
#include "we_internal.cuh"

namespace we {

__global__ void k_rw_flux(EnsView E, RwView rw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nb = rw.nb;
  double *acc = reinterpret_cast<double *>(smem_raw);
  int32_t *mark = reinterpret_cast<int32_t *>(acc + nb);
  const int r = blockIdx.y, t = blockIdx.x, lane = threadIdx.x;
  const int iter = *E.iter;
  if (iter <= E.first_iter) return;                 // the initial walkers' start bins are unknown
  if (t >= E.n_tasks[r]) return;
  for (int e = lane; e < nb; e += 32) mark[e] = 0;
  __syncwarp();
  if (lane != 0) return;
  const int4 tk = E.tasks[(size_t)r * nb + t];      // (bin, in offset, count, out offset)
  const int b = tk.x, o = tk.w;
  const int n = min(E.m_targ, E.count[r] - o);
  const int par = iter & 1;
  const double *w = E.w[par] + (size_t)r * E.cap + o;
  const int32_t *bin = E.bin + (size_t)r * E.cap + o;
  for (int k = 0; k < n; ++k) {
    const int e = bin[k];
    if (!mark[e]) { mark[e] = 1; acc[e] = 0.0; }
    acc[e] = __dadd_rn(acc[e], w[k]);
  }
  double *Fr = rw.F + (size_t)r * nb * nb;
  for (int k = 0; k < n; ++k) {
    const int e = bin[k];
    if (mark[e]) {
      Fr[(size_t)e * nb + b] = __dadd_rn(Fr[(size_t)e * nb + b], acc[e]);
      mark[e] = 0;
    }
  }
}

// The iteration that just finished (k_finalize has advanced E.iter) and whether it reweights.
__device__ __forceinline__ bool rw_due(const EnsView &E, const RwView &rw, int &li) {
  li = *E.iter - 1 - E.first_iter;
  return li >= 0 && (li + 1) % rw.period == 0;
}

__global__ void __launch_bounds__(256) k_rw_solve(EnsView E, RwView rw) {
  const int r = blockIdx.x, tid = threadIdx.x, B = blockDim.x;
  const int nb = rw.nb;
  int li = 0;
  const bool due = rw_due(E, rw, li);
  const bool rec = li >= 0 && li < E.record_iters;
  if (!due) {
    if (tid == 0 && rec) rw.obs[(size_t)li * E.R + r] = 0;
    return;
  }
  const double *F = rw.F + (size_t)r * nb * nb;
  double *W = rw.W + (size_t)r * nb, *cb = rw.cb + (size_t)r * nb, *fac = rw.fac + (size_t)r * nb;
  double *rhs = rw.rhs + (size_t)r * nb, *x = rw.x + (size_t)r * nb;
  double *M = rw.M + (size_t)r * nb * nb;
  int32_t *A = rw.act + (size_t)r * nb;
  __shared__ int s_n, s_ok, s_p;
  __shared__ double s_v[256];
  __shared__ int s_i[256];
  for (int b = tid; b < nb; b += B) {
    double s = 0.0;
    for (int e = 0; e < nb; ++e) s = __dadd_rn(s, F[(size_t)e * nb + b]);
    W[b] = s;
    fac[b] = 0.0;
    cb[b] = 0.0;
  }
  __syncthreads();
  // current bin weights: the walkers of each bin of the split/merge just done, in slot order
  const int par = (*E.iter) & 1;
  for (int t = tid; t < E.n_tasks[r]; t += B) {
    const int4 tk = E.tasks[(size_t)r * nb + t];
    const int n = min(E.m_targ, E.count[r] - tk.w);
    const double *w = E.w[par] + (size_t)r * E.cap + tk.w;
    double s = 0.0;
    for (int k = 0; k < n; ++k) s = __dadd_rn(s, w[k]);
    cb[tk.x] = s;
  }
  if (tid == 0) {
    int n = 0;
    for (int b = 0; b < nb; ++b)
      if (W[b] > 0.0) A[n++] = b;
    s_n = n;
    s_ok = n >= 2;
  }
  __syncthreads();
  const int n = s_n;
  if (s_ok) {
    for (int idx = tid; idx < n * n; idx += B) {
      const int i = idx / n, j = idx - i * n;
      M[idx] = i == j ? 0.0 : __ddiv_rn(F[(size_t)A[i] * nb + A[j]], W[A[j]]);
    }
    __syncthreads();
    for (int j = tid; j < n; j += B) {
      double out = 0.0;
      for (int i = 0; i < n; ++i)
        if (i != j) out = __dadd_rn(out, M[(size_t)i * n + j]);
      M[(size_t)j * n + j] = -out;
    }
    __syncthreads();
    for (int j = tid; j < n; j += B) M[(size_t)(n - 1) * n + j] = 1.0;
    for (int i = tid; i < n; i += B) rhs[i] = i == n - 1 ? 1.0 : 0.0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
      // pivot: the first row (from k) of largest magnitude in column k
      double bv = -1.0;
      int bi = n;
      for (int rr = k + tid; rr < n; rr += B) {
        const double v = fabs(M[(size_t)rr * n + k]);
        if (v > bv) { bv = v; bi = rr; }
      }
      s_v[tid] = bv;
      s_i[tid] = bi;
      __syncthreads();
      for (int h = B / 2; h > 0; h >>= 1) {
        if (tid < h) {
          const double ov = s_v[tid + h];
          const int oi = s_i[tid + h];
          if (ov > s_v[tid] || (ov == s_v[tid] && oi < s_i[tid])) { s_v[tid] = ov; s_i[tid] = oi; }
        }
        __syncthreads();
      }
      const int p = s_i[0];
      if (M[(size_t)p * n + k] == 0.0) {
        if (tid == 0) s_ok = 0;
        break;                                       // uniform: every thread read the same p
      }
      if (p != k) {
        for (int c = tid; c < n; c += B) {
          const double a = M[(size_t)k * n + c];
          M[(size_t)k * n + c] = M[(size_t)p * n + c];
          M[(size_t)p * n + c] = a;
        }
        if (tid == 0) { const double a = rhs[k]; rhs[k] = rhs[p]; rhs[p] = a; }
      }
      __syncthreads();
      const int wdt = n - k;                         // columns k+1 .. n-1 and the right-hand side
      for (int idx = tid; idx < (n - k - 1) * wdt; idx += B) {
        const int rr = k + 1 + idx / wdt, c = k + 1 + idx % wdt;
        const double l = __ddiv_rn(M[(size_t)rr * n + k], M[(size_t)k * n + k]);
        if (c < n) M[(size_t)rr * n + c] = __dsub_rn(M[(size_t)rr * n + c], __dmul_rn(l, M[(size_t)k * n + c]));
        else rhs[rr] = __dsub_rn(rhs[rr], __dmul_rn(l, rhs[k]));
      }
      __syncthreads();
    }
    __syncthreads();
  }
  if (s_ok) {
    for (int k = n - 1; k >= 0; --k) {
      if (tid == 0) x[k] = __ddiv_rn(rhs[k], M[(size_t)k * n + k]);
      __syncthreads();
      const double xk = x[k];
      for (int rr = tid; rr < k; rr += B) rhs[rr] = __dsub_rn(rhs[rr], __dmul_rn(M[(size_t)rr * n + k], xk));
      __syncthreads();
    }
  }
  if (tid == 0) {
    int outcome = -1;
    if (s_ok) {
      double C = 0.0, T = 0.0;
      int held = 0;
      bool good = true;
      for (int i = 0; i < n && good; ++i) {
        if (!(cb[A[i]] > 0.0)) continue;
        if (!(x[i] > 0.0) || isinf(x[i])) { good = false; break; }
        C = __dadd_rn(C, cb[A[i]]);
        T = __dadd_rn(T, x[i]);
        ++held;
      }
      if (good && held > 0 && T > 0.0 && !isinf(T)) {
        const double q = __ddiv_rn(C, T);
        for (int i = 0; i < n; ++i)
          if (cb[A[i]] > 0.0) fac[A[i]] = __ddiv_rn(__dmul_rn(x[i], q), cb[A[i]]);
        outcome = 1;
      }
    }
    if (rec) rw.obs[(size_t)li * E.R + r] = outcome;
  }
}

__global__ void k_rw_apply(EnsView E, RwView rw) {
  int li = 0;
  if (!rw_due(E, rw, li)) return;
  const int par = (*E.iter) & 1;
  const int ld = E.R * E.cap;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ld; g += gridDim.x * blockDim.x) {
    const int r = g / E.cap, w = g - r * E.cap;
    if (w >= E.count[r]) continue;
    const int b = E.tasks[(size_t)r * rw.nb + w / E.m_targ].x;
    const double f = rw.fac[(size_t)r * rw.nb + b];
    if (f != 0.0) E.w[par][g] = __dmul_rn(E.w[par][g], f);
  }
}

cudaError_t launch_rw_flux(const PropagateParams &prm, cudaStream_t st) {
  const EnsView &E = prm.ens;
  const RwView &rw = prm.rw;
  const int tasks = rw.nb < E.cap ? rw.nb : E.cap;
  const size_t smem = 12 * (size_t)rw.nb;
  k_rw_flux<<<dim3(tasks, E.R), 32, smem, st>>>(E, rw);
  return cudaGetLastError();
}

cudaError_t launch_rw_solve_apply(const PropagateParams &prm, cudaStream_t st) {
  const EnsView &E = prm.ens;
  k_rw_solve<<<E.R, 256, 0, st>>>(E, prm.rw);
  const int ld = E.R * E.cap;
  int grid = (ld + 255) / 256;
  if (grid > 152 * 8) grid = 152 * 8;
  k_rw_apply<<<grid, 256, 0, st>>>(E, prm.rw);
  return cudaGetLastError();
}

}  // namespace we
