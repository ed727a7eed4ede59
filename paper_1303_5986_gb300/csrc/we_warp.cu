// we_warp.cu -- one warp per walker, for networks too large for a register tree (up to 8192
// reactions): Gillespie's direct method (Sec. II.A) for one interval tau, with recycling
// (Sec. II.B.2), bin assignment and observables, as in the thread kernels.
//
// The walker's counts and its whole canonical propensity tree (P leaves, node k = node 2k +
// node 2k+1, rounded; 16P bytes) live in shared memory.  Per event:
//   * the warp makes 32 draws at a time (one Philox block and one float-float logarithm per
//     lane) and hands them out one per event by shuffle;
//   * every lane walks the same descent (uniform control flow, broadcast loads);
//   * after the reaction fires, the lanes re-evaluate the reactions the dependency graph lists
//     for it, one per lane, and recompute the dirty tree nodes level by level -- duplicates
//     compute the same rounded sum, so no ordering is needed -- giving the same node values
//     as a full rebuild (each node is a function of its two children only).
#include "we_ssa_common.cuh"

namespace we {

__device__ __forceinline__ void finish_walker_warp(const PropagateParams &prm, int r, int g, int par,
                                                   const int32_t *xs, double t, long long nev,
                                                   int nrec, int status, int lane) {
  const EnsView &E = prm.ens;
  const int ld = E.R * E.cap;
  for (int s = lane; s < E.S; s += 32) E.x[par][(size_t)s * ld + g] = xs[s];
  if (lane != 0) return;
  E.nrec[g] = nrec;
  E.tlast[g] = t;
  if (status) atomicCAS(&E.status[r], 0, status);
  if (!prm.bins.learned) {
    const int b = bin_of(prm.bins, xs, 1);
    E.bin[g] = b;
    if (prm.resample) atomicAdd(&E.bin_count[r * prm.bins.n_bins + b], 1);
  }
  const int slot = *E.iter - E.first_iter;
  if (slot >= 0 && slot < E.record_iters) {
    const double wt = E.w[par][g];
    const int o = slot * E.R + r;
    if (nrec) atomicAdd(&E.obs_flux[o], __dmul_rn((double)nrec, wt));
    if (nev) atomicAdd(&E.obs_events[o], (unsigned long long)nev);
    if (E.hist_len > 0) {
      const int v = xs[E.hist_species];
      const int idx = v < E.hist_len - 1 ? v : E.hist_len - 1;
      atomicAdd(&E.obs_hist[(size_t)o * E.hist_len + idx], wt);
    }
    if (!prm.resample) atomicAdd(&E.obs_totw[o], wt);
  }
}

// Block = one warp = one walker.  Shared memory: tree (2P doubles), counts (S ints), log tables.
__global__ void __launch_bounds__(32) k_propagate_warp(PropagateParams prm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const NetView &N = prm.net;
  const EnsView &E = prm.ens;
  const int lane = threadIdx.x;
  const int P = N.P, L = N.log2P;
  double *nd = reinterpret_cast<double *>(smem_raw);                    // 2P
  LogTables *lt = reinterpret_cast<LogTables *>(nd + 2 * P);
  int32_t *xs = reinterpret_cast<int32_t *>(lt + 1);                      // S
  {
    const double *src = reinterpret_cast<const double *>(prm.logt);
    double *dst = reinterpret_cast<double *>(lt);
    for (int i = lane; i < (int)(sizeof(LogTables) / 8); i += 32) dst[i] = src[i];
  }
  const int iter = *E.iter;
  const int total = E.run_off[E.R];
  const int f = blockIdx.x;
  if (f >= total) return;
  const int r = E.R == 1 ? 0 : find_run(E.run_off, E.R, f);
  const int w = f - E.run_off[r];
  const int g = r * E.cap + w;
  const int par = iter & 1;
  const int ld = E.R * E.cap;
  for (int s = lane; s < E.S; s += 32) xs[s] = E.x[par][(size_t)s * ld + g];
  const int ps = E.param_set[r];
  const double *keff = N.keff + (size_t)ps * P;
  const double *Kn = N.hill_Kn + (size_t)ps * P;
  const uint32_t k0 = (uint32_t)E.seed;
  const uint32_t k1 = (uint32_t)(E.seed >> 32) + E.run_id[r];
  __syncwarp();

  // full rebuild of leaves and internal nodes
  auto rebuild = [&]() {
    for (int j = lane; j < P; j += 32) nd[P + j] = propensity(N.meta[j], keff[j], Kn[j], xs, 1);
    __syncwarp();
    for (int lvl = L - 1; lvl >= 0; --lvl) {
      for (int k = (1 << lvl) + lane; k < (2 << lvl); k += 32) nd[k] = __dadd_rn(nd[2 * k], nd[2 * k + 1]);
      __syncwarp();
    }
  };
  rebuild();
  __syncwarp();

  const long long tau_bits = bits(E.tau);
  double t = 0.0;
  long long nev = 0;
  int nrec = 0, status = 0;
  const LogTables &T = *lt;
  // draws: lane i holds draw (batch*32 + i)
  uint32_t batch = 0;
  unsigned long long my_m = 0;
  float2 my_e = make_float2(0.f, 0.f);
  ssa_draw((uint32_t)lane, (uint32_t)iter, (uint32_t)w, k0, k1, T, my_m, my_e);
  int used = 0;
  for (;;) {
    const double a0 = nd[1];
    if (bits(a0) == 0) break;
    if (used == 32) {
      ++batch;
      ssa_draw(batch * 32u + (uint32_t)lane, (uint32_t)iter, (uint32_t)w, k0, k1, T, my_m, my_e);
      used = 0;
    }
    const unsigned long long m2 = __shfl_sync(0xffffffffu, my_m, used);
    float2 e;
    e.x = __shfl_sync(0xffffffffu, my_e.x, used);
    e.y = __shfl_sync(0xffffffffu, my_e.y, used);
    ++used;
    const double tn = advance_clock(t, e, rcp_pos(a0));
    if (bits(tn) > tau_bits) break;
    if (nev >= E.max_steps) { status = kStatusStepCap; break; }
    double target = __dmul_rn(u01_index(m2), a0);
    int k = 1;
    for (int lvl = 0; lvl < L; ++lvl) {
      const double Lv = nd[2 * k], Rv = nd[2 * k + 1];
      const bool right = (bits(Rv) != 0) && !(bits(target) < bits(Lv));
      if (right) { target = __dsub_rn(target, Lv); k = 2 * k + 1; }
      else { k = 2 * k; }
    }
    const int j = k - P;
    const int db = N.meta[j].d_begin, de = N.meta[j].d_end;
    // overflow check, then apply the net changes (one lane per changed species)
    bool over = false;
    for (int q = db + lane; q < de; q += 32) over |= xs[N.d_sp[q]] + N.d_val[q] > kMaxCount;
    if (__any_sync(0xffffffffu, over)) { status = kStatusOverflow; break; }
    for (int q = db + lane; q < de; q += 32) xs[N.d_sp[q]] += N.d_val[q];
    __syncwarp();
    ++nev;
    t = tn;
    bool recycled = false;
    if (E.feedback) {
      bool in = true;
      for (int c = 0; c < E.n_clauses; ++c) {
        const int v = xs[E.tgt_species[c]];
        const int thr = E.tgt_thr[r * E.n_clauses + c];
        in = in && (E.tgt_op[c] == 0 ? v >= thr : v <= thr);
      }
      if (in) {
        ++nrec;
        recycled = true;
        __syncwarp();
        for (int s = lane; s < E.S; s += 32) xs[s] = E.recycle[r * E.S + s];
        __syncwarp();
      }
    }
    if (recycled) { rebuild(); __syncwarp(); continue; }
    // dependent reactions: new leaves, then their ancestors level by level
    const int qb = N.dep_ptr[j], qe = N.dep_ptr[j + 1];
    for (int q0 = qb; q0 < qe; q0 += 32) {
      const int q = q0 + lane;
      int node = 0;
      if (q < qe) {
        const int i = N.dep_idx[q];
        nd[P + i] = propensity(N.meta[i], keff[i], Kn[i], xs, 1);
        node = (P + i) >> 1;
      }
      __syncwarp();
      for (int lvl = 0; lvl < L; ++lvl) {
        if (q < qe) nd[node] = __dadd_rn(nd[2 * node], nd[2 * node + 1]);
        __syncwarp();
        node >>= 1;
      }
    }
  }
  __syncwarp();
  finish_walker_warp(prm, r, g, par, xs, t, nev, nrec, status, lane);
}

size_t propagate_warp_smem(const NetView &N, int block) {
  (void)block;
  return 16 * (size_t)N.P + sizeof(LogTables) + 4 * (size_t)N.S + 16;
}

cudaError_t launch_propagate_warp(const PropagateParams &prm, int block, cudaStream_t st) {
  (void)block;
  const size_t smem = propagate_warp_smem(prm.net, 32);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_propagate_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int grid = prm.ens.R * prm.ens.cap;
  k_propagate_warp<<<grid, 32, smem, st>>>(prm);
  return cudaGetLastError();
}

}  // namespace we
