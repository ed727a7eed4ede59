// we_reweight.cu -- steady-state reweighting of Bhatt et al. (Sec. II.B.2, Eq. "ss").
//
// In steady state each bin's inflow equals its outflow, sum_j (k_ij w_j - k_ji w_i) = 0, with
// f_ij = k_ij w_j the flux into bin i from bin j.  The rates come from the transfers measured
// over every interval so far: F_ij = weight that started an interval in bin j and ended it in
// bin i, W_j = sum_i F_ij, k_ij = F_ij / W_j.  Every reweight_period-th iteration, after the
// split/merge, the balance equations are solved on the largest strongly connected set of bins
// with W_j > 0 (transfers leaving the set left out), and the walkers of each of its bins that
// holds any are rescaled so that those bins carry the solved weights (their total unchanged).
//
//   k_rw_flux   (after the SSA, before the split/merge): one warp per bin of the previous
//               split/merge, whose M_targ walkers are consecutive slots; lane 0 sums their
//               weights by end bin in ascending slot order and adds each sum to F once.
//   k_rw_solve  (after the split/merge; one block per run): the largest strongly connected
//               set of bins (one warp, Kosaraju), then the elimination of Grassmann, Taksar
//               and Heyman on it -- only sums and products of non-negative numbers, so every
//               bin weight keeps its relative accuracy however small -- with the sums taken
//               in a fixed order by one thread and the rank-one updates in parallel, each
//               product and sum rounded on its own (no fused multiply-add): the factors are
//               the same bits as the sequential elimination.
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
  if (iter <= E.first_iter && !rw.start_known) return;   // the initial walkers' start bins are unknown
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

// The iteration that just finished (k_finalize has advanced E.iter), as an index into the
// recorded iterations, and whether it reweights: after iterations period-1, 2 period-1, ... of
// the run counted from 0, whatever iteration this ensemble started at.
__device__ __forceinline__ bool rw_due(const EnsView &E, const RwView &rw, int &li) {
  const int it = *E.iter - 1;
  li = it - E.first_iter;
  return li >= 0 && (it + 1) % rw.period == 0;
}

// The largest strongly connected component of the observed-transfer graph over the active bins
// act[0..n) (edge j -> i when i != j and F[i][j] > 0), written ascending over act; returns its
// size (largest by bin count, ties to the component with the lowest bin).  Kosaraju's two
// iterative depth-first passes, run by one warp: every lane follows the same search, the next
// neighbour is found 32 candidates at a time by ballot, and lane 0 writes the scratch (6 n
// ints) that the lanes read after a warp barrier.
// The next i >= from (i != j) with mark[i] == unmarked and an observed transfer j -> i (i -> j
// when transposed), 32 candidates per ballot; n if there is none.  Called by a whole warp.
__device__ __forceinline__ int rw_next_neighbour(int n, const int32_t *act, const double *F, int nb, int j,
                                                 int from, const int32_t *mark, int unmarked, bool transposed) {
  const int lane = threadIdx.x & 31;
  for (int base = from; base < n; base += 32) {
    const int i = base + lane;
    bool ok = false;
    if (i < n && i != j && mark[i] == unmarked) {
      const double f = transposed ? F[(size_t)act[j] * nb + act[i]] : F[(size_t)act[i] * nb + act[j]];
      ok = f > 0.0;
    }
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    if (m) return base + __ffs(m) - 1;
  }
  return n;
}

__device__ __forceinline__ int rw_largest_scc(int n, int32_t *act, const double *F, int nb, int32_t *scr) {
  const int lane = threadIdx.x & 31;
  int32_t *seen = scr, *order = scr + n, *stk = scr + 2 * n, *nxt = scr + 3 * n;
  int32_t *csize = scr + 4 * n, *cfirst = scr + 5 * n;
  for (int k = lane; k < n; k += 32) seen[k] = 0;
  __syncwarp();
  int no = 0;
  for (int s0 = 0; s0 < n; ++s0) {
    if (seen[s0]) continue;
    int top = 0;
    if (lane == 0) { stk[0] = s0; nxt[0] = 0; seen[s0] = 1; }
    __syncwarp();
    while (top >= 0) {
      const int j = stk[top];
      const int i = rw_next_neighbour(n, act, F, nb, j, nxt[top], seen, 0, false);
      if (i < n) {
        if (lane == 0) { nxt[top] = i + 1; seen[i] = 1; stk[top + 1] = i; nxt[top + 1] = 0; }
        ++top;
      } else {
        if (lane == 0) order[no] = j;
        ++no;
        --top;
      }
      __syncwarp();
    }
  }
  int32_t *comp = seen;                              // reused: component labels, -1 = none yet
  for (int k = lane; k < n; k += 32) comp[k] = -1;
  __syncwarp();
  int nc = 0;
  for (int q = n - 1; q >= 0; --q) {
    const int s1 = order[q];
    if (comp[s1] >= 0) continue;
    int top = 0;
    if (lane == 0) { stk[0] = s1; nxt[0] = 0; comp[s1] = nc; }
    __syncwarp();
    while (top >= 0) {
      const int j = stk[top];
      const int i = rw_next_neighbour(n, act, F, nb, j, nxt[top], comp, -1, true);
      if (i < n) {
        if (lane == 0) { nxt[top] = i + 1; comp[i] = nc; stk[top + 1] = i; nxt[top + 1] = 0; }
        ++top;
      } else {
        --top;
      }
      __syncwarp();
    }
    ++nc;
  }
  for (int c = lane; c < nc; c += 32) { csize[c] = 0; cfirst[c] = n; }
  __syncwarp();
  if (lane == 0)
    for (int k = 0; k < n; ++k) {
      const int c = comp[k];
      if (csize[c] == 0) cfirst[c] = k;
      ++csize[c];
    }
  __syncwarp();
  int best = -1, best_size = 0, best_min = 0;
  for (int c = 0; c < nc; ++c)
    if (csize[c] > best_size || (csize[c] == best_size && cfirst[c] < best_min)) {
      best = c; best_size = csize[c]; best_min = cfirst[c];
    }
  if (lane == 0) {
    int m = 0;
    for (int k = 0; k < n; ++k)
      if (comp[k] == best) act[m++] = act[k];
  }
  __syncwarp();
  return best_size;
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
  double *x = rw.x + (size_t)r * nb;
  double *M = rw.M + (size_t)r * nb * nb;
  int32_t *A = rw.act + (size_t)r * nb;
  int32_t *scr = rw.iscr + (size_t)r * 6 * nb;
  __shared__ int s_n, s_ok;
  __shared__ double s_out;
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
  __syncthreads();
  if (tid < 32) {                                    // warp 0: the active list, then the set search
    int na = 0;
    for (int b0 = 0; b0 < nb; b0 += 32) {
      const int b = b0 + tid;
      const bool act_b = b < nb && W[b] > 0.0;
      const unsigned m = __ballot_sync(0xffffffffu, act_b);
      if (act_b) A[na + __popc(m & ((1u << tid) - 1u))] = b;
      na += __popc(m);
    }
    __syncwarp();
    const int n = na >= 2 ? rw_largest_scc(na, A, F, nb, scr) : 0;
    if (tid == 0) { s_n = n; s_ok = n >= 2; }
  }
  __syncthreads();
  const int n = s_n;
  if (s_ok) {
    // R[a][b] = rate from the a-th to the b-th bin of the set, k_ba = F[b][a] / W[a]
    for (int idx = tid; idx < n * n; idx += B) {
      const int a = idx / n, b = idx - a * n;
      M[idx] = a == b ? 0.0 : __ddiv_rn(F[(size_t)A[b] * nb + A[a]], W[A[a]]);
    }
    __syncthreads();
    // GTH elimination, last state first (non-negative arithmetic only)
    for (int k = n - 1; k >= 1; --k) {
      if (tid == 0) {
        double out = 0.0;
        for (int j = 0; j < k; ++j) out = __dadd_rn(out, M[(size_t)k * n + j]);
        s_out = out;
        if (!(out > 0.0)) s_ok = 0;
      }
      __syncthreads();
      if (!s_ok) break;                              // uniform: every thread read the same flag
      const double out = s_out;
      for (int i = tid; i < k; i += B) M[(size_t)i * n + k] = __ddiv_rn(M[(size_t)i * n + k], out);
      __syncthreads();
      for (int idx = tid; idx < k * k; idx += B) {
        const int i = idx / k, j = idx - i * k;
        if (i != j)
          M[(size_t)i * n + j] = __dadd_rn(M[(size_t)i * n + j], __dmul_rn(M[(size_t)i * n + k], M[(size_t)k * n + j]));
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    int outcome = -1;
    if (s_ok) {
      x[0] = 1.0;
      for (int k = 1; k < n; ++k) {
        double v = 0.0;
        for (int i = 0; i < k; ++i) v = __dadd_rn(v, __dmul_rn(x[i], M[(size_t)i * n + k]));
        x[k] = v;
      }
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
