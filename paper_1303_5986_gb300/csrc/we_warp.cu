// we_warp.cu -- one warp per walker, for networks too large for a register tree (up to 16,384
// reactions): Gillespie's direct method (Sec. II.A) for one interval tau, with recycling
// (Sec. II.B.2), bin assignment and observables, as in the thread kernels.
//
// The walker's counts and its canonical propensity tree (Pw = max(P, 4) leaves, node k = node
// 2k + node 2k+1, rounded) live in shared memory.  The leaves and the internal nodes of every
// level but the lowest are stored (12 Pw bytes); a lowest-level node, the sum of two adjacent
// leaves, is recomputed where it is read.  That is the same rounded sum the stored node would
// hold, so values and descent are those of the full tree, and four walkers of a 4096-leaf
// network fit on one SM instead of three.  Per event:
//   * the warp makes 32 draws at a time (one Philox block and one float-float logarithm per
//     lane) and hands them out one per event by shuffle;
//   * every lane walks the same descent, two levels per shared-memory round trip;
//   * the fired reaction's event record (its net changes and its dependents' species,
//     multiplicities and rate constants, at a fixed stride) is fetched in one round trip,
//     requested before the clock arithmetic so that the two overlap; the descent runs before
//     the clock too, as it has no side effects;
//   * the lanes re-evaluate the dependent reactions (up to three per lane) and then recompute
//     the dirty ancestors once, level by level: while a level has more than 32 nodes each lane
//     updates its dependents' ancestors (duplicates compute the same rounded sum), above that
//     every node of the level is recomputed, one per lane.  Each node is a function of its two
//     children only, so the tree equals a full rebuild.
#include "we_ssa_common.cuh"

namespace we {

__device__ __forceinline__ void finish_walker_warp(const PropagateParams &prm, int r, int g, int par, int iter,
                                                   int32_t *xs, double t, long long nev,
                                                   int nrec, int status, int near, int lane) {
  const EnsView &E = prm.ens;
  const int ld = E.R * E.cap;
  // the walker's weight is loaded first, so that the load overlaps the stores and the binning
  const int slot = iter - E.first_iter;
  const bool rec = lane == 0 && slot >= 0 && slot < E.record_iters;
  const double wt = rec ? E.w[par][g] : 0.0;
  // target checked at the interval's end only: a walker found in it goes to the recycle state
  if (E.end_check && in_target(E, r, xs, 1)) {            // every lane reads the same counts
    __syncwarp();
    for (int s = lane; s < E.S; s += 32) xs[s] = E.recycle[r * E.S + s];
    __syncwarp();
    nrec = 1;
  }
  for (int s = lane; s < E.S; s += 32) E.x[par][(size_t)s * ld + g] = xs[s];
  if (lane != 0) return;
  E.nrec[g] = nrec;
  E.tlast[g] = t;
  if (E.fpt) record_first_passage(E, r, g, xs, 1, nrec, t);
  if (status) atomicCAS(&E.status[r], 0, status);
  if (!prm.bins.learned) {
    const int b = bin_of(prm.bins, xs, 1);
    E.bin[g] = b;
    if (prm.resample) atomicAdd(&E.bin_count[r * prm.bins.n_bins + b], 1);
  }
  if (rec) {
    const int o = slot * E.R + r;
    if (nrec) atomicAdd(&E.obs_flux[o], __dmul_rn((double)nrec, wt));
    if (nev) atomicAdd(&E.obs_events[o], (unsigned long long)nev);
    if (near) atomicAdd(&E.obs_near[o], 1);
    if (E.hist_len > 0) {
      const int v = xs[E.hist_species];
      const int idx = v < E.hist_len - 1 ? v : E.hist_len - 1;
      atomicAdd(&E.obs_hist[(size_t)o * E.hist_len + idx], wt);
    }
    if (!prm.resample) atomicAdd(&E.obs_totw[o], wt);
  }
}

// One dependent reaction from an event record (layout at NetView::wrec); w.x < 0: no entry.
struct DepRec {
  int4 w;
  double keff, Kn;
};

__device__ __forceinline__ DepRec load_dep(const int4 *dr, int q, int n) {
  DepRec d{make_int4(-1, 0, 0, 0), 0.0, 0.0};
  if (q < n) {
    d.w = __ldg(dr + 2 * q);
    const double2 k = __ldg(reinterpret_cast<const double2 *>(dr + 2 * q + 1));
    d.keff = k.x;
    d.Kn = k.y;
  }
  return d;
}

__device__ __forceinline__ int dep_index(const DepRec &d) { return d.w.x & 0xFFFFF; }

// The same operations, in the same order, as propensity() for the entry's reaction.
__device__ __forceinline__ double propensity_rec(const DepRec &d, const int32_t *xs) {
  const int pk = d.w.x >> 20;
  if ((pk >> 2) & 1) {
    const int hn = (pk >> 3) & 3;
    const long long y = xs[d.w.y];
    long long yn = y;
    if (hn >= 2) yn *= y;
    if (hn >= 3) yn *= y;
    return __ddiv_rn(d.keff, __dadd_rn(d.Kn, __ll2double_rn(yn)));
  }
  const int nr = pk & 3;
  long long h = 1;
  if (nr > 0) h *= binom_small(xs[d.w.y], (pk >> 5) & 3);
  if (nr > 1) h *= binom_small(xs[d.w.z], (pk >> 7) & 3);
  if (nr > 2) h *= binom_small(xs[d.w.w], (pk >> 9) & 3);
  return __dmul_rn(d.keff, __ll2double_rn(h));
}

__device__ __forceinline__ double2 lds2(const double *p) { return *reinterpret_cast<const double2 *>(p); }

// Node k of the lowest stored level (k in [Pw/4, Pw/2)) from its four leaves lf[4k - Pw ...].
__device__ __forceinline__ void update_from_leaves(double *nd, const double *lf, int Pw, int k) {
  const double2 l = lds2(lf + 4 * k - Pw), r = lds2(lf + 4 * k - Pw + 2);
  nd[k] = __dadd_rn(__dadd_rn(l.x, l.y), __dadd_rn(r.x, r.y));
}

__device__ __forceinline__ void update_from_children(double *nd, int k) {
  const double2 c = lds2(nd + 2 * k);
  nd[k] = __dadd_rn(c.x, c.y);
}

// One descent step at a node whose children have values (lv, rv).
__device__ __forceinline__ void descend_step(double &target, int &k, double lv, double rv) {
  const bool right = (bits(rv) != 0) && !(bits(target) < bits(lv));
  if (right) target = __dsub_rn(target, lv);
  k = 2 * k + (right ? 1 : 0);
}

// Block = one warp = one walker.  Shared memory: internal nodes (Pw/2 doubles, index 0 unused),
// leaves (Pw doubles), log tables, counts (S ints).
__global__ void __launch_bounds__(32) k_propagate_warp(PropagateParams prm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const NetView &N = prm.net;
  const EnsView &E = prm.ens;
  const int lane = threadIdx.x;
  const int P = N.P;
  const int Lw = N.log2P < 2 ? 2 : N.log2P, Pw = 1 << Lw;
  double *nd = reinterpret_cast<double *>(smem_raw);                    // Pw/2
  double *lf = nd + Pw / 2;                                              // Pw
  LogTables *lt = reinterpret_cast<LogTables *>(lf + Pw);
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
  int r_start = 0;
  const int r = E.R == 1 ? 0 : find_run_start(E.run_off, E.R, f, r_start);
  const int w = f - r_start;
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

  // full rebuild: leaves, the lowest stored level from four leaves each, then the levels above
  auto rebuild = [&]() {
    for (int j = lane; j < Pw; j += 32) lf[j] = j < P ? propensity(N.meta[j], keff[j], Kn[j], xs, 1) : 0.0;
    __syncwarp();
    for (int k = Pw / 4 + lane; k < Pw / 2; k += 32) update_from_leaves(nd, lf, Pw, k);
    __syncwarp();
    for (int lvl = Lw - 3; lvl >= 0; --lvl) {
      for (int k = (1 << lvl) + lane; k < (2 << lvl); k += 32) update_from_children(nd, k);
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
  // absorbing target: a walker that starts the interval inside it fires nothing
  const bool absorbed = E.feedback == 2 && in_target(E, r, xs, 1);
  double t_stop = 0.0;
  for (; !absorbed;) {
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
    // descent (no side effects, so it may run before the clock decides whether the event
    // fires): stored levels two at a time, then the computed lowest level and the leaves
    double target = __dmul_rn(u01_index(m2), a0);
    int k = 1, lvl = 0;
    for (; lvl + 2 <= Lw - 2; lvl += 2) {
      const double2 c = lds2(nd + 2 * k), g0 = lds2(nd + 4 * k), g1 = lds2(nd + 4 * k + 2);
      const bool right = (bits(c.y) != 0) && !(bits(target) < bits(c.x));
      if (right) target = __dsub_rn(target, c.x);
      k = 2 * k + (right ? 1 : 0);
      const double2 gc = right ? g1 : g0;
      descend_step(target, k, gc.x, gc.y);
    }
    if (lvl < Lw - 2) {
      const double2 c = lds2(nd + 2 * k);
      descend_step(target, k, c.x, c.y);
    }
    {
      const double2 l = lds2(lf + 4 * k - Pw), rr = lds2(lf + 4 * k - Pw + 2);
      const double lv = __dadd_rn(l.x, l.y), rv = __dadd_rn(rr.x, rr.y);
      const bool right = (bits(rv) != 0) && !(bits(target) < bits(lv));
      if (right) target = __dsub_rn(target, lv);
      k = 2 * k + (right ? 1 : 0);
      const double2 pr = right ? rr : l;
      descend_step(target, k, pr.x, pr.y);
    }
    const int j = k - Pw;
    // the fired reaction's record -- net changes and the dependents' parameters, one round
    // trip -- is requested before the clock arithmetic, which then overlaps the loads
    const int4 *rec = N.wrec + (size_t)j * N.wrec_stride;
    const int4 hdr = __ldg(rec);                       // n_changes, n_dependents, d_begin, dep_begin
    int2 chg = make_int2(-1, 0);
    if (lane < N.wrec_chg) chg = __ldg(reinterpret_cast<const int2 *>(rec + 1) + lane);
    const int4 *dr = rec + 1 + (N.wrec_chg + 1) / 2;
    DepRec da = load_dep(dr, lane, N.wrec_dep);
    DepRec db = load_dep(dr, lane + 32, N.wrec_dep);
    DepRec dc = load_dep(dr, lane + 64, N.wrec_dep);
    const double tn = advance_clock(t, e, rcp_pos(a0));
    if (bits(tn) > tau_bits) { t_stop = tn; break; }
    if (nev >= E.max_steps) { status = kStatusStepCap; break; }
    if (ps != 0) {                                      // the record holds parameter set 0
      if (da.w.x >= 0) { da.keff = keff[dep_index(da)]; da.Kn = Kn[dep_index(da)]; }
      if (db.w.x >= 0) { db.keff = keff[dep_index(db)]; db.Kn = Kn[dep_index(db)]; }
      if (dc.w.x >= 0) { dc.keff = keff[dep_index(dc)]; dc.Kn = Kn[dep_index(dc)]; }
    }
    const int cb = hdr.z + N.wrec_chg, ce = hdr.z + hdr.x;      // changes past the record
    const int qb = hdr.w + N.wrec_dep, qe = hdr.w + hdr.y;      // dependents past the record
    // overflow check, then apply the net changes (one lane per changed species)
    bool over = chg.x >= 0 && xs[chg.x] + chg.y > kMaxCount;
    for (int q = cb + lane; q < ce; q += 32) over |= xs[N.d_sp[q]] + N.d_val[q] > kMaxCount;
    if (__any_sync(0xffffffffu, over)) { status = kStatusOverflow; break; }
    if (chg.x >= 0) xs[chg.x] += chg.y;
    for (int q = cb + lane; q < ce; q += 32) xs[N.d_sp[q]] += N.d_val[q];
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
        if (E.feedback == 2) break;                     // absorbed at its first passage
        recycled = true;
        __syncwarp();
        for (int s = lane; s < E.S; s += 32) xs[s] = E.recycle[r * E.S + s];
        __syncwarp();
      }
    }
    if (recycled) { rebuild(); __syncwarp(); continue; }
    // dependent reactions: new leaves, then the dirty ancestors once, level by level
    {
      double pa = 0.0, pb = 0.0, pc = 0.0;
      if (da.w.x >= 0) pa = propensity_rec(da, xs);
      if (db.w.x >= 0) pb = propensity_rec(db, xs);
      if (dc.w.x >= 0) pc = propensity_rec(dc, xs);
      if (da.w.x >= 0) lf[dep_index(da)] = pa;
      if (db.w.x >= 0) lf[dep_index(db)] = pb;
      if (dc.w.x >= 0) lf[dep_index(dc)] = pc;
    }
    for (int q = qb + lane; q < qe; q += 32) {
      const int i = N.dep_idx[q];
      lf[i] = propensity(N.meta[i], keff[i], Kn[i], xs, 1);
    }
    __syncwarp();
    for (int sh = 2; sh <= Lw; ++sh) {
      const int cnt = Pw >> sh;            // nodes on this level: [cnt, 2 cnt)
      if (cnt > 32) {
        if (sh == 2) {
          if (da.w.x >= 0) update_from_leaves(nd, lf, Pw, (Pw + dep_index(da)) >> 2);
          if (db.w.x >= 0) update_from_leaves(nd, lf, Pw, (Pw + dep_index(db)) >> 2);
          if (dc.w.x >= 0) update_from_leaves(nd, lf, Pw, (Pw + dep_index(dc)) >> 2);
          for (int q = qb + lane; q < qe; q += 32) update_from_leaves(nd, lf, Pw, (Pw + N.dep_idx[q]) >> 2);
        } else {
          if (da.w.x >= 0) update_from_children(nd, (Pw + dep_index(da)) >> sh);
          if (db.w.x >= 0) update_from_children(nd, (Pw + dep_index(db)) >> sh);
          if (dc.w.x >= 0) update_from_children(nd, (Pw + dep_index(dc)) >> sh);
          for (int q = qb + lane; q < qe; q += 32) update_from_children(nd, (Pw + N.dep_idx[q]) >> sh);
        }
      } else if (lane < cnt) {
        if (sh == 2) update_from_leaves(nd, lf, Pw, cnt + lane);
        else update_from_children(nd, cnt + lane);
      }
      __syncwarp();
    }
  }
  __syncwarp();
  finish_walker_warp(prm, r, g, par, iter, xs, t, nev, nrec, status, near_tau_fp64(E.tau, t, t_stop), lane);
}

size_t propagate_warp_smem(const NetView &N, int block) {
  (void)block;
  const size_t Pw = N.P < 4 ? 4 : (size_t)N.P;
  return 12 * Pw + sizeof(LogTables) + 4 * (size_t)N.S + 16;
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
