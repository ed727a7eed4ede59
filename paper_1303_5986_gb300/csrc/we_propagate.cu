// we_propagate.cu -- the SSA kernels: one interval tau of Gillespie's direct method per walker
// (Sec. II.A; the "propagate dynamics" step of the WE algorithm, Sec. II.B), with in-interval
// recycling (Sec. II.B.2), bin assignment and the interval's observables in the epilogue.
//
//   k_propagate_direct<P>  one thread per walker; every propensity and the canonical tree are
//                          recomputed after each event, in registers (small networks)
//   k_propagate_table<P>   one thread per walker for networks whose propensities all read one
//                          species: the whole tree and 1/a0 are looked up by that species' count
//                          in a table built once per ensemble by the same device arithmetic, so
//                          an event costs a handful of FP64 operations instead of tens
//
// Both kernels draw the next event's random numbers and waiting-time logarithm while the
// current event is processed (the draw does not depend on the state), keeping the ~700-cycle
// FP64 chain of the logarithm off the event-to-event critical path.
#include "we_ssa_common.cuh"

namespace we {

// A double as an unevaluated float pair (hi = nearest float, lo = nearest float to the rest).
__device__ __forceinline__ float2 split_ff(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(__dsub_rn(x, (double)h)));
}

// Tables of neg_log_u01, from CUDA's own double log and division.
__global__ void k_init_log_tables(LogTables *T) {
  const int i = threadIdx.x;
  if (i < 128) {
    const double c = 1.0 + (double)(2 * i + 1) / 256.0;
    T->inv_c[i] = split_ff(__ddiv_rn(1.0, c));
    T->b[i] = split_ff(-log(c * 0.5));
  }
  if (i < 64) T->n_ln2[i] = split_ff(log(ldexp(1.0, i)));
}

// The reaction the canonical descent picks for the 52-bit uniform index m, u2 = (2m+1)/2^53.
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

// Row x of the state-indexed table: [1/a0, a0, b_1 .. b_{P-1}, unused], where b_i is the least
// uniform index m whose descent picks a reaction >= i.  The descent is monotone in m (the
// target fl(u2 a0) grows with u2, each comparison is a threshold, each subtraction is monotone),
// so the reaction for m is the number of b_i <= m: the hot loop selects with integer compares
// and reaches exactly the reaction the floating-point descent would.  base holds the counts of
// the species other than `species`.
template <int P, int LOG2P>
__global__ void k_build_table(NetView N, const int32_t *base, int species, int len, double *rows) {
  const int ps = blockIdx.y;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < len; x += gridDim.x * blockDim.x) {
    int32_t xs[kThreadMaxSpecies];
    for (int s = 0; s < N.S; ++s) xs[s] = base[s];
    xs[species] = x;
    double nd[2 * P];
#pragma unroll
    for (int j = 0; j < P; ++j)
      nd[P + j] = propensity(N.meta[j], N.keff[ps * P + j], N.hill_Kn[ps * P + j], xs, 1);
#pragma unroll
    for (int k = P - 1; k >= 1; --k) nd[k] = __dadd_rn(nd[2 * k], nd[2 * k + 1]);
    double *row = rows + ((size_t)ps * len + x) * (2 * P);
    row[0] = bits(nd[1]) > 0 ? __ddiv_rn(1.0, nd[1]) : 0.0;
    row[1] = nd[1];
    for (int i = 1; i < P; ++i) {
      unsigned long long lo = 0, hi = 1ull << 52;            // m = 2^52 stands for "never"
      if (bits(nd[1]) > 0) {
        while (lo < hi) {
          const unsigned long long mid = (lo + hi) >> 1;
          if (descend<P, LOG2P>(nd, mid) >= i) hi = mid; else lo = mid + 1;
        }
      }
      row[1 + i] = __longlong_as_double((long long)lo);
    }
    for (int k = P + 1; k < 2 * P; ++k) row[k] = 0.0;
  }
}

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
__device__ __forceinline__ void finish_walker(const PropagateParams &prm, int r, int g, int par,
                                              const int32_t *xme, int B, double t, long long nev,
                                              int nrec, int status) {
  const EnsView &E = prm.ens;
  const int ld = E.R * E.cap;
  int32_t *X = E.x[par];
  for (int s = 0; s < E.S; ++s) X[(size_t)s * ld + g] = xme[s * B];
  E.nrec[g] = nrec;
  E.tlast[g] = t;
  if (status) atomicCAS(&E.status[r], 0, status);
  if (!prm.bins.learned) {
    const int b = bin_of(prm.bins, xme, B);
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
      const int v = xme[E.hist_species * B];
      const int idx = v < E.hist_len - 1 ? v : E.hist_len - 1;
      atomicAdd(&E.obs_hist[(size_t)o * E.hist_len + idx], wt);
    }
    if (!prm.resample) atomicAdd(&E.obs_totw[o], wt);
  }
}

// ------------------------------------------------------------------------------------------
// Direct evaluation: the canonical propensity tree (P leaves, node k = node 2k + node 2k+1,
// rounded) lives in registers; after unrolling every index into it is a compile-time constant
// and the descent picks children with predicated selects.  Counts sit in shared memory so that
// reactions can name them by runtime index.
// ------------------------------------------------------------------------------------------
template <int P, int LOG2P>
__global__ void __launch_bounds__(128) k_propagate_direct(PropagateParams prm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Smem sm = load_smem<P>(prm, smem_raw);
  const EnsView &E = prm.ens;
  const int B = blockDim.x, tid = threadIdx.x;
  const int iter = *E.iter;
  const int total = E.run_off[E.R];
  const int f = blockIdx.x * B + tid;
  if (f >= total) return;
  const int r = E.R == 1 ? 0 : find_run(E.run_off, E.R, f);
  const int w = f - E.run_off[r];
  const int g = r * E.cap + w;
  const int par = iter & 1;
  const int ld = E.R * E.cap;
  int32_t *xme = sm.xs + tid;
  for (int s = 0; s < E.S; ++s) xme[s * B] = E.x[par][(size_t)s * ld + g];
  const int ps = E.param_set[r];
  const double *keff = sm.keff + ps * P;
  const double *Kn = sm.Kn + ps * P;
  const uint32_t k0 = (uint32_t)E.seed;
  const uint32_t k1 = (uint32_t)(E.seed >> 32) + E.run_id[r];

  double nd[2 * P];
  auto rebuild = [&]() {
#pragma unroll
    for (int j = 0; j < P; ++j) nd[P + j] = propensity(sm.meta[j], keff[j], Kn[j], xme, B);
#pragma unroll
    for (int k = P - 1; k >= 1; --k) nd[k] = __dadd_rn(nd[2 * k], nd[2 * k + 1]);
  };
  rebuild();

  const long long tau_bits = bits(E.tau);
  double t = 0.0;
  long long nev = 0;
  int nrec = 0, status = 0;
  DrawQueue dq;
  dq.init((uint32_t)iter, (uint32_t)w, k0, k1, *sm.logt);
  for (;;) {
    const double a0 = nd[1];
    if (bits(a0) == 0) break;                        // nothing can fire: idle to tau
    unsigned long long m2;
    float2 e;
    dq.pop((uint32_t)iter, (uint32_t)w, k0, k1, *sm.logt, m2, e);
    const double tn = advance_clock(t, e, rcp_pos(a0));
    if (bits(tn) > tau_bits) break;                  // the next event falls after tau
    if (nev >= E.max_steps) { status = kStatusStepCap; break; }
    double target = __dmul_rn(u01_index(m2), a0);
    int k = 1;
#pragma unroll
    for (int lvl = 0; lvl < LOG2P; ++lvl) {
      double L = 0.0, R = 0.0;
#pragma unroll
      for (int c = (1 << lvl); c < (2 << lvl); ++c)
        if (k == c) { L = nd[2 * c]; R = nd[2 * c + 1]; }
      const bool right = (bits(R) != 0) && !(bits(target) < bits(L));
      if (right) { target = __dsub_rn(target, L); k = 2 * k + 1; }
      else { k = 2 * k; }
    }
    const RxnMeta &mt = sm.meta[k - P];
    bool over = false;
    for (int q = mt.d_begin; q < mt.d_end; ++q)
      over |= (xme[sm.dsp[q] * B] + sm.dval[q]) > kMaxCount;
    if (over) { status = kStatusOverflow; break; }
    for (int q = mt.d_begin; q < mt.d_end; ++q) xme[sm.dsp[q] * B] += sm.dval[q];
    ++nev;
    t = tn;
    if (E.feedback && in_target(E, r, xme, B)) {
      ++nrec;
      for (int s = 0; s < E.S; ++s) xme[s * B] = E.recycle[r * E.S + s];
    }
    rebuild();
  }
  finish_walker(prm, r, g, par, xme, B, t, nev, nrec, status);
}

// ------------------------------------------------------------------------------------------
// State-indexed tables: all propensities read one species x, so the whole canonical tree and
// 1/a0 are functions of x alone.  Row x of the table (built by k_build_table with the direct
// kernel's arithmetic) replaces the recomputation; counts beyond the table are evaluated into
// a per-thread row.  Per event: the waiting time (one product, one sum), the target (one
// product) and up to log2 P descent subtractions.
// ------------------------------------------------------------------------------------------
template <int P, int LOG2P>
__global__ void __launch_bounds__(128) k_propagate_table(PropagateParams prm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Smem sm = load_smem<P>(prm, smem_raw);
  const EnsView &E = prm.ens;
  const TableView &TV = prm.tab;
  const int B = blockDim.x, tid = threadIdx.x;
  int32_t *s_dx = sm.xs + E.S * B;                   // net change of the table species, per reaction
  for (int j = tid; j < P; j += B) {
    int dx = 0;
    for (int q = sm.meta[j].d_begin; q < sm.meta[j].d_end; ++q)
      if (sm.dsp[q] == TV.species) dx += sm.dval[q];
    s_dx[j] = dx;
  }
  __syncthreads();
  const int iter = *E.iter;
  const int total = E.run_off[E.R];
  const int f = blockIdx.x * B + tid;
  if (f >= total) return;
  const int r = E.R == 1 ? 0 : find_run(E.run_off, E.R, f);
  const int w = f - E.run_off[r];
  const int g = r * E.cap + w;
  const int par = iter & 1;
  const int ld = E.R * E.cap;
  int32_t *xme = sm.xs + tid;
  for (int s = 0; s < E.S; ++s) xme[s * B] = E.x[par][(size_t)s * ld + g];
  const int ps = E.param_set[r];
  const double *keff = sm.keff + ps * P;
  const double *Kn = sm.Kn + ps * P;
  const double *tab = TV.rows + (size_t)ps * TV.len * (2 * P);
  const uint32_t k0 = (uint32_t)E.seed;
  const uint32_t k1 = (uint32_t)(E.seed >> 32) + E.run_id[r];
  const int sx = TV.species;

  // Row for counts beyond the table, in thread-local memory: `row` may point here or into the
  // table, so it is read with generic loads (a global-only load of a local address faults).
  double fb[2 * P];
  auto locate = [&](int x) -> const double * {
    if (x < TV.len) return tab + (size_t)x * (2 * P);
    for (int j = 0; j < P; ++j) fb[P + j] = propensity(sm.meta[j], keff[j], Kn[j], xme, B);
    for (int k = P - 1; k >= 1; --k) fb[k] = __dadd_rn(fb[2 * k], fb[2 * k + 1]);
    fb[0] = bits(fb[1]) > 0 ? __ddiv_rn(1.0, fb[1]) : 0.0;   // fb[1] = a0 as in a table row
    return fb;
  };
  int x = xme[sx * B];
  const double *row = locate(x);

  const long long tau_bits = bits(E.tau);
  double t = 0.0;
  long long nev = 0;
  int nrec = 0, status = 0;
  DrawQueue dq;
  dq.init((uint32_t)iter, (uint32_t)w, k0, k1, *sm.logt);
  for (;;) {
    const double a0 = row[1];
    if (bits(a0) == 0) break;
    unsigned long long m2;
    float2 e;
    dq.pop((uint32_t)iter, (uint32_t)w, k0, k1, *sm.logt, m2, e);
    const double tn = advance_clock(t, e, row[0]);
    if (bits(tn) > tau_bits) break;
    if (nev >= E.max_steps) { status = kStatusStepCap; break; }
    int j;
    if (row != fb) {
      j = 0;                                         // reaction = breakpoints at or below m2
#pragma unroll
      for (int i = 1; i < P; ++i) j += (long long)m2 >= bits(row[1 + i]) ? 1 : 0;
    } else {
      j = descend<P, LOG2P>(fb, m2);
    }
    const int nx = x + s_dx[j];
    if (nx > kMaxCount) { status = kStatusOverflow; break; }
    x = nx;
    xme[sx * B] = x;
    ++nev;
    t = tn;
    if (E.feedback && in_target(E, r, xme, B)) {
      ++nrec;
      for (int s = 0; s < E.S; ++s) xme[s * B] = E.recycle[r * E.S + s];
      x = xme[sx * B];
    }
    row = locate(x);
  }
  finish_walker(prm, r, g, par, xme, B, t, nev, nrec, status);
}

// ------------------------------------------------------------------------------------------
// Warp-specialised form of both kernels.  A block of four warps serves 32 walkers (one per
// lane).  Warp 0 runs the event loops; warps 1-3, on the other sub-partitions of the SM,
// generate the next round of kRoundDraws draws per walker (Philox + logarithm, most of the
// instructions of an event) into a shared-memory buffer while warp 0 consumes the current
// one.  The two buffers alternate at a __syncthreads per round; the loop ends when warp 0
// reports that all its walkers are done, so every wait is a block barrier that all warps reach.
// ------------------------------------------------------------------------------------------
constexpr int kRoundDraws = 16;

template <int P, int LOG2P, bool TABLE>
__global__ void __launch_bounds__(128) k_propagate_ws(PropagateParams prm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Smem sm = load_smem<P>(prm, smem_raw);
  const EnsView &E = prm.ens;
  const TableView &TV = prm.tab;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int W = 32;                                  // walkers per block
  int32_t *s_dx = sm.xs + E.S * W;                       // net change of the table species
  unsigned long long *qm = reinterpret_cast<unsigned long long *>(
      (reinterpret_cast<uintptr_t>(s_dx + P) + 15) & ~(uintptr_t)15);   // [2][kRoundDraws][W]
  float2 *qe = reinterpret_cast<float2 *>(qm + 2 * kRoundDraws * W);    // [2][kRoundDraws][W]
  __shared__ int s_more;
  if (TABLE)
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
      int dx = 0;
      for (int q = sm.meta[j].d_begin; q < sm.meta[j].d_end; ++q)
        if (sm.dsp[q] == TV.species) dx += sm.dval[q];
      s_dx[j] = dx;
    }

  const int iter = *E.iter;
  const int total = E.run_off[E.R];
  const int f = blockIdx.x * W + lane;
  const bool live = f < total;
  const int r = !live ? 0 : (E.R == 1 ? 0 : find_run(E.run_off, E.R, f));
  const int w = live ? f - E.run_off[r] : 0;
  const uint32_t k0 = (uint32_t)E.seed;
  const uint32_t k1 = (uint32_t)(E.seed >> 32) + E.run_id[r];
  const LogTables &LT = *sm.logt;

  // draws [base, base + kRoundDraws) of this lane's walker into buffer b (producer warps)
  auto produce = [&](int b, uint32_t base, int first, int stride) {
    if (!live) return;
#pragma unroll 2
    for (int k = first; k < kRoundDraws; k += stride) {
      unsigned long long m2;
      float2 e;
      ssa_draw(base + (uint32_t)k, (uint32_t)iter, (uint32_t)w, k0, k1, LT, m2, e);
      qm[(b * kRoundDraws + k) * W + lane] = m2;
      qe[(b * kRoundDraws + k) * W + lane] = e;
    }
  };
  produce(0, 0u, warp, 4);                               // round 0: all four warps
  __syncthreads();

  // consumer state (warp 0)
  const int g = r * E.cap + w;
  const int par = iter & 1;
  const int ld = E.R * E.cap;
  int32_t *xme = sm.xs + lane;
  const int ps = live ? E.param_set[r] : 0;
  const double *keff = sm.keff + ps * P;
  const double *Kn = sm.Kn + ps * P;
  const long long tau_bits = bits(E.tau);
  double t = 0.0;
  long long nev = 0;
  int nrec = 0, status = 0;
  bool done = !live;
  // table path: the current row in registers
  int x = 0, dxr[P];
  double inv = 0.0, a0r = 0.0;
  long long bp[P > 1 ? P - 1 : 1];
  bool fallback = false;
  double nd[TABLE ? 1 : 2 * P];
  double fb[TABLE ? 2 * P : 1];
  const double *tab = TABLE ? TV.rows + (size_t)ps * TV.len * (2 * P) : nullptr;
  // target set seen from the table species: x in [xlo, xhi] while the other clauses hold
  int xlo = 0, xhi = 0, xrec = 0;
  bool others_ok = false;
  auto load_row = [&](int xv) {
    if (xv < TV.len) {
      const double *p = tab + (size_t)xv * (2 * P);
      inv = p[0];
      a0r = p[1];
#pragma unroll
      for (int i = 1; i < P; ++i) bp[i - 1] = bits(p[1 + i]);
      fallback = false;
    } else {
      xme[TV.species * W] = xv;
      for (int j = 0; j < P; ++j) fb[P + j] = propensity(sm.meta[j], keff[j], Kn[j], xme, W);
      for (int k = P - 1; k >= 1; --k) fb[k] = __dadd_rn(fb[2 * k], fb[2 * k + 1]);
      a0r = fb[1];
      inv = bits(a0r) > 0 ? __ddiv_rn(1.0, a0r) : 0.0;
      fallback = true;
    }
  };
  // Clauses on the table species become the window [xlo, xhi]; the others read species that no
  // reaction changes, so they are evaluated once (and again after a recycle).
  auto target_window = [&]() {
    xlo = -1;
    xhi = kMaxCount + 1;
    others_ok = true;
    for (int c = 0; c < E.n_clauses; ++c) {
      const int thr = E.tgt_thr[r * E.n_clauses + c];
      if (E.tgt_species[c] == TV.species) {
        if (E.tgt_op[c] == 0) xlo = max(xlo, thr); else xhi = min(xhi, thr);
      } else {
        const int v = xme[E.tgt_species[c] * W];
        others_ok = others_ok && (E.tgt_op[c] == 0 ? v >= thr : v <= thr);
      }
    }
  };
  auto rebuild = [&]() {
#pragma unroll
    for (int j = 0; j < P; ++j) nd[P + j] = propensity(sm.meta[j], keff[j], Kn[j], xme, W);
#pragma unroll
    for (int k = P - 1; k >= 1; --k) nd[k] = __dadd_rn(nd[2 * k], nd[2 * k + 1]);
  };
  if (warp == 0 && live) {
    for (int s = 0; s < E.S; ++s) xme[s * W] = E.x[par][(size_t)s * ld + g];
    if (TABLE) {
#pragma unroll
      for (int j = 0; j < P; ++j) dxr[j] = s_dx[j];
      x = xme[TV.species * W];
      if (E.feedback) {
        target_window();
        xrec = E.recycle[r * E.S + TV.species];
      }
      load_row(x);
    } else {
      rebuild();
    }
  }

  for (int round = 0;; ++round) {
    const int b = round & 1;
    if (warp == 0) {
      for (int k = 0; k < kRoundDraws && !done; ++k) {
        const unsigned long long m2 = qm[(b * kRoundDraws + k) * W + lane];
        const float2 e = qe[(b * kRoundDraws + k) * W + lane];
        if (TABLE) {
          if (bits(a0r) == 0) { done = true; break; }      // nothing can fire: idle to tau
          const double tn = advance_clock(t, e, inv);
          int j;
          if (!fallback) {
            j = 0;                                        // reaction = breakpoints at or below m2
#pragma unroll
            for (int i = 0; i + 1 < P; ++i) j += (long long)m2 >= bp[i] ? 1 : 0;
          } else {
            j = descend<P, LOG2P>(fb, m2);
          }
          int dx = dxr[0];
#pragma unroll
          for (int i = 1; i < P; ++i) dx = (j == i) ? dxr[i] : dx;
          const int nx = x + dx;
          if (bits(tn) > tau_bits) { done = true; break; }  // the next event falls after tau
          if (nev >= E.max_steps) { status = kStatusStepCap; done = true; break; }
          if (nx > kMaxCount) { status = kStatusOverflow; done = true; break; }
          x = nx;
          ++nev;
          t = tn;
          if (E.feedback && others_ok && x >= xlo && x <= xhi) {
            ++nrec;                                       // recycle: the whole state is reset
            for (int s = 0; s < E.S; ++s) xme[s * W] = E.recycle[r * E.S + s];
            x = xrec;
            target_window();
          }
          load_row(x);
        } else {
          const double a0 = nd[1];
          if (bits(a0) == 0) { done = true; break; }
          const double tn = advance_clock(t, e, rcp_pos(a0));
          if (bits(tn) > tau_bits) { done = true; break; }
          if (nev >= E.max_steps) { status = kStatusStepCap; done = true; break; }
          double target = __dmul_rn(u01_index(m2), a0);
          int kk = 1;
#pragma unroll
          for (int lvl = 0; lvl < LOG2P; ++lvl) {
            double L = 0.0, R = 0.0;
#pragma unroll
            for (int c = (1 << lvl); c < (2 << lvl); ++c)
              if (kk == c) { L = nd[2 * c]; R = nd[2 * c + 1]; }
            const bool right = (bits(R) != 0) && !(bits(target) < bits(L));
            if (right) { target = __dsub_rn(target, L); kk = 2 * kk + 1; }
            else { kk = 2 * kk; }
          }
          const RxnMeta &mt = sm.meta[kk - P];
          bool over = false;
          for (int q = mt.d_begin; q < mt.d_end; ++q)
            over |= (xme[sm.dsp[q] * W] + sm.dval[q]) > kMaxCount;
          if (over) { status = kStatusOverflow; done = true; break; }
          for (int q = mt.d_begin; q < mt.d_end; ++q) xme[sm.dsp[q] * W] += sm.dval[q];
          ++nev;
          t = tn;
          if (E.feedback && in_target(E, r, xme, W)) {
            ++nrec;
            for (int s = 0; s < E.S; ++s) xme[s * W] = E.recycle[r * E.S + s];
          }
          rebuild();
        }
      }
      const int more = __any_sync(0xffffffffu, !done);
      if (lane == 0) s_more = more;
    } else {
      produce(b ^ 1, (uint32_t)((round + 1) * kRoundDraws), warp - 1, 3);
    }
    __syncthreads();
    if (!s_more) break;
    __syncthreads();                                      // s_more is rewritten next round
  }
  if (warp == 0 && live) {
    if (TABLE) xme[TV.species * W] = x;
    finish_walker(prm, r, g, par, xme, W, t, nev, nrec, status);
  }
}

// ------------------------------------------------------------------------------------------
// host-side launch helpers
// ------------------------------------------------------------------------------------------
size_t propagate_thread_smem(const NetView &N, int block, bool table) {
  return sizeof(LogTables) + (size_t)N.P * sizeof(RxnMeta) +
         2 * (size_t)N.n_param_sets * N.P * sizeof(double) + 2 * (size_t)N.n_delta * sizeof(int32_t) +
         (size_t)N.S * block * sizeof(int32_t) + (table ? (size_t)N.P * sizeof(int32_t) : 0);
}

size_t propagate_ws_smem(const NetView &N) {
  return sizeof(LogTables) + (size_t)N.P * sizeof(RxnMeta) +
         2 * (size_t)N.n_param_sets * N.P * sizeof(double) + 2 * (size_t)N.n_delta * sizeof(int32_t) +
         (size_t)N.S * 32 * sizeof(int32_t) + (size_t)N.P * sizeof(int32_t) + 16 +
         2 * (size_t)kRoundDraws * 32 * (sizeof(unsigned long long) + sizeof(float2));
}

cudaError_t launch_init_log_tables(LogTables *T, cudaStream_t st) {
  k_init_log_tables<<<1, 128, 0, st>>>(T);
  return cudaGetLastError();
}

template <int P, int L>
static cudaError_t build_table_p(const NetView &N, const int32_t *base, int species, int len,
                                 double *rows, cudaStream_t st) {
  dim3 grid((len + 127) / 128, N.n_param_sets);
  k_build_table<P, L><<<grid, 128, 0, st>>>(N, base, species, len, rows);
  return cudaGetLastError();
}

cudaError_t launch_build_table(const NetView &N, const int32_t *base, int species, int len,
                               double *rows, cudaStream_t st) {
  switch (N.P) {
    case 1: return build_table_p<1, 0>(N, base, species, len, rows, st);
    case 2: return build_table_p<2, 1>(N, base, species, len, rows, st);
    case 4: return build_table_p<4, 2>(N, base, species, len, rows, st);
    case 8: return build_table_p<8, 3>(N, base, species, len, rows, st);
    case 16: return build_table_p<16, 4>(N, base, species, len, rows, st);
    default: return cudaErrorInvalidValue;
  }
}

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

cudaError_t launch_propagate_ws(const PropagateParams &prm, bool table, cudaStream_t st) {
  const int total_slots = prm.ens.R * prm.ens.cap;
  const int grid = (total_slots + 31) / 32;
  const size_t smem = propagate_ws_smem(prm.net);
#define WE_CASE(PP, LL)                                                                  \
  case PP:                                                                               \
    return table ? launch_k(k_propagate_ws<PP, LL, true>, prm, grid, 128, smem, st)      \
                 : launch_k(k_propagate_ws<PP, LL, false>, prm, grid, 128, smem, st);
  switch (prm.net.P) {
    WE_CASE(1, 0)
    WE_CASE(2, 1)
    WE_CASE(4, 2)
    WE_CASE(8, 3)
    WE_CASE(16, 4)
    default: return cudaErrorInvalidValue;
  }
#undef WE_CASE
}

cudaError_t launch_propagate_thread(const PropagateParams &prm, int block, bool table, cudaStream_t st) {
  const int total_slots = prm.ens.R * prm.ens.cap;
  const int grid = (total_slots + block - 1) / block;
  const size_t smem = propagate_thread_smem(prm.net, block, table);
#define WE_CASE(PP, LL)                                                                  \
  case PP:                                                                               \
    return table ? launch_k(k_propagate_table<PP, LL>, prm, grid, block, smem, st)       \
                 : launch_k(k_propagate_direct<PP, LL>, prm, grid, block, smem, st);
  switch (prm.net.P) {
    WE_CASE(1, 0)
    WE_CASE(2, 1)
    WE_CASE(4, 2)
    WE_CASE(8, 3)
    WE_CASE(16, 4)
    default: return cudaErrorInvalidValue;
  }
#undef WE_CASE
}

}  // namespace we
