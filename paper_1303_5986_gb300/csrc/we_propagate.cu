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
#include <algorithm>

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
    const float2 ic = split_ff(__ddiv_rn(1.0, c)), nb = split_ff(-log(c * 0.5));
    T->cb[i] = make_float4(ic.x, ic.y, nb.x, nb.y);
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
__global__ void k_build_table(NetView N, const int32_t *base, int species, int species2, int len, int lenB,
                              double clock_scale, unsigned long long *rows) {
  const int ps = blockIdx.y;
  const int n_rows = len * lenB;                             // row x = count of species * lenB + count of species2
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n_rows; x += gridDim.x * blockDim.x) {
    int32_t xs[kThreadMaxSpecies];
    for (int s = 0; s < N.S; ++s) xs[s] = base[s];
    xs[species] = x / lenB;
    if (species2 >= 0) xs[species2] = x % lenB;
    double nd[2 * P];
#pragma unroll
    for (int j = 0; j < P; ++j)
      nd[P + j] = propensity(N.meta[j], N.keff[ps * P + j], N.hill_Kn[ps * P + j], xs, 1);
#pragma unroll
    for (int k = P - 1; k >= 1; --k) nd[k] = __dadd_rn(nd[2 * k], nd[2 * k + 1]);
    unsigned long long *row = rows + ((size_t)ps * n_rows + x) * P;
    row[0] = pack_ff(wait_scale(nd[1], clock_scale));
    for (int i = 1; i < P; ++i) {
      unsigned long long lo = 0, hi = 1ull << 52;            // m = 2^52 stands for "never"
      if (bits(nd[1]) > 0) {
        while (lo < hi) {
          const unsigned long long mid = (lo + hi) >> 1;
          if (descend<P, LOG2P>(nd, mid) >= i) hi = mid; else lo = mid + 1;
        }
      }
      row[i] = lo;
    }
  }
}

// A table walker's current row in registers: the wait scale and the breakpoints, or (for
// counts beyond the table, `direct`) the canonical tree evaluated on the fly into fb, an array
// of the caller's kept apart so that the row itself stays in registers.
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
__device__ __forceinline__ void finish_walker(const PropagateParams &prm, int r, int g, int par,
                                              const int32_t *xme, int B, double t, long long nev,
                                              int nrec, int status, int near) {
  const EnsView &E = prm.ens;
  const int ld = E.R * E.cap;
  int32_t *X = E.x[par];
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
  const int slot = *E.iter - E.first_iter;
  if (slot >= 0 && slot < E.record_iters) {
    const double wt = E.w[par][g];
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
  const bool absorbed = E.feedback == 2 && in_target(E, r, xme, B);
  double t_stop = 0.0;
  for (; !absorbed;) {
    const double a0 = nd[1];
    if (bits(a0) == 0) break;                        // nothing can fire: idle to tau
    unsigned long long m2;
    float2 e;
    dq.pop((uint32_t)iter, (uint32_t)w, k0, k1, *sm.logt, m2, e);
    const double tn = advance_clock(t, e, rcp_pos(a0));
    if (bits(tn) > tau_bits) { t_stop = tn; break; } // the next event falls after tau
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
      if (E.feedback == 2) break;                    // absorbed at its first passage
      for (int s = 0; s < E.S; ++s) xme[s * B] = E.recycle[r * E.S + s];
    }
    rebuild();
  }
  finish_walker(prm, r, g, par, xme, B, t, nev, nrec, status, near_tau_fp64(E.tau, t, t_stop));
}

// ------------------------------------------------------------------------------------------
// State-indexed tables: all propensities read one species x, so the whole canonical tree and
// 1/a0 are functions of x alone.  Row x of the table (built by k_build_table with the direct
// kernel's arithmetic) replaces the recomputation; counts beyond the table are evaluated on
// the fly.  Per event: the waiting time in clock units (FP32 products, integer rounding and
// sum), the reaction by integer compares, and the next row.
// ------------------------------------------------------------------------------------------
template <int P, int LOG2P>
__global__ void __launch_bounds__(128) k_propagate_table(PropagateParams prm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Smem sm = load_smem<P>(prm, smem_raw);
  const EnsView &E = prm.ens;
  const TableView &TV = prm.tab;
  const int B = blockDim.x, tid = threadIdx.x;
  int32_t *s_dx = sm.xs + E.S * B;                   // net change of the table species, per reaction
  int32_t *s_dy = s_dx + P;                           // ... and of the second one
  for (int j = tid; j < P; j += B) {
    int dx = 0, dy = 0;
    for (int q = sm.meta[j].d_begin; q < sm.meta[j].d_end; ++q) {
      if (sm.dsp[q] == TV.species) dx += sm.dval[q];
      if (sm.dsp[q] == TV.species2) dy += sm.dval[q];
    }
    s_dx[j] = dx;
    s_dy[j] = dy;
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
  const unsigned long long *tab = TV.rows + (size_t)ps * TV.len * TV.lenB * P;
  const uint32_t k0 = (uint32_t)E.seed;
  const uint32_t k1 = (uint32_t)(E.seed >> 32) + E.run_id[r];
  const int sx = TV.species, sy = TV.species2;

  TableRow<P, LOG2P> row;
  double fb[2 * P];
  auto load_row = [&](int xv, int yv) {           // xme holds the current counts
    if (xv < TV.len && yv < TV.lenB) row.read(tab + ((size_t)xv * TV.lenB + yv) * P);
    else row.evaluate(fb, sm.meta, keff, Kn, xme, B, TV.clock_scale);
  };
  int x = xme[sx * B], y = sy >= 0 ? xme[sy * B] : 0;
  load_row(x, y);

  unsigned long long clk = 0;                       // clock units of tau / 2^62
  long long nev = 0;
  int nrec = 0, status = 0;
  DrawQueue dq;
  dq.init((uint32_t)iter, (uint32_t)w, k0, k1, *sm.logt);
  const bool absorbed = E.feedback == 2 && in_target(E, r, xme, B);
  unsigned long long stop_u = 0;                    // clock of the first draw past tau (0: none)
  for (; !absorbed;) {
    if (row.idle()) break;                           // nothing can fire: idle to tau
    unsigned long long m2;
    float2 e;
    dq.pop((uint32_t)iter, (uint32_t)w, k0, k1, *sm.logt, m2, e);
    unsigned long long dt;
    if (!wait_units(e, row.w, dt)) break;            // far beyond the interval
    if (clk + dt > kClockTau) { stop_u = clk + dt; break; }          // next event after tau
    if (nev >= E.max_steps) { status = kStatusStepCap; break; }
    const int j = row.select(m2, fb);
    const int nx = x + s_dx[j], ny = sy >= 0 ? y + s_dy[j] : 0;
    if (nx > kMaxCount || ny > kMaxCount) { status = kStatusOverflow; break; }
    x = nx;
    y = ny;
    xme[sx * B] = x;
    if (sy >= 0) xme[sy * B] = y;
    ++nev;
    clk += dt;
    if (E.feedback && in_target(E, r, xme, B)) {
      ++nrec;
      if (E.feedback == 2) break;                    // absorbed at its first passage
      for (int s = 0; s < E.S; ++s) xme[s * B] = E.recycle[r * E.S + s];
      x = xme[sx * B];
      y = sy >= 0 ? xme[sy * B] : 0;
    }
    load_row(x, y);
  }
  finish_walker(prm, r, g, par, xme, B, clock_time(clk, E.tau), nev, nrec, status, near_tau_units(clk, stop_u));
}

// ------------------------------------------------------------------------------------------
// Warp-specialised kernels: a block of four warps serves 32 walkers (one per lane), and the
// draws (Philox + logarithm, most of the instructions of an event) come from other warps than
// the event chain, through shared-memory buffers that alternate at block barriers.  Every
// wait is a block barrier that all warps reach; a loop ends when every walker is done.
// ------------------------------------------------------------------------------------------
constexpr int kRoundDraws = 16;
constexpr int kWindowMargin = 96;    // table rows staged beyond a block's range of counts

// General networks.  Warp 0 runs the event loops (FP64 propensities and tree, rebuilt after
// each event); warps 1-3 generate the next round of kRoundDraws draws per walker meanwhile.
template <int P, int LOG2P>
__global__ void __launch_bounds__(128) k_propagate_ws(PropagateParams prm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Smem sm = load_smem<P>(prm, smem_raw);
  const EnsView &E = prm.ens;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int W = 32;                                  // walkers per block
  unsigned long long *qm = reinterpret_cast<unsigned long long *>(
      (reinterpret_cast<uintptr_t>(sm.xs + E.S * W) + 15) & ~(uintptr_t)15);   // [2][kRoundDraws][W]
  float2 *qe = reinterpret_cast<float2 *>(qm + 2 * kRoundDraws * W);            // [2][kRoundDraws][W]
  __shared__ int s_more;
  // Persistent blocks: each takes groups of 32 walkers (vb) until every live walker is served,
  // so the shared prologue above is paid once per resident block, not once per capacity slot.
  const int n_live_all = E.run_off[E.R];
  for (int vb = blockIdx.x; vb * 32 < n_live_all; vb += gridDim.x) {
  __syncthreads();                                       // the previous group's buffers are free

  const int iter = *E.iter;
  const int total = E.run_off[E.R];
  const int f = vb * W + lane;
  const bool live = f < total;
  const int r = !live ? 0 : (E.R == 1 ? 0 : find_run(E.run_off, E.R, f));
  const int w = live ? f - E.run_off[r] : 0;
  const uint32_t k0 = (uint32_t)E.seed;
  const uint32_t k1 = (uint32_t)(E.seed >> 32) + E.run_id[r];
  const LogTables &LT = *sm.logt;
  const int g = r * E.cap + w;
  const int par = iter & 1;
  const int ld = E.R * E.cap;
  const int ps = live ? E.param_set[r] : 0;

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

  int32_t *xme = sm.xs + lane;
  const double *keff = sm.keff + ps * P;
  const double *Kn = sm.Kn + ps * P;
  const long long tau_bits = bits(E.tau);
  double t = 0.0;
  long long nev = 0;
  int nrec = 0, status = 0;
  bool done = !live;
  double t_stop = 0.0;
  double nd[2 * P];
  auto rebuild = [&]() {
#pragma unroll
    for (int j = 0; j < P; ++j) nd[P + j] = propensity(sm.meta[j], keff[j], Kn[j], xme, W);
#pragma unroll
    for (int k = P - 1; k >= 1; --k) nd[k] = __dadd_rn(nd[2 * k], nd[2 * k + 1]);
  };
  if (warp == 0 && live) {
    for (int s = 0; s < E.S; ++s) xme[s * W] = E.x[par][(size_t)s * ld + g];
    rebuild();
    if (E.feedback == 2 && in_target(E, r, xme, W)) done = true;   // already absorbed
  }

  for (int round = 0;; ++round) {
    const int b = round & 1;
    if (warp == 0) {
      for (int k = 0; k < kRoundDraws && !done; ++k) {
        const unsigned long long m2 = qm[(b * kRoundDraws + k) * W + lane];
        const float2 e = qe[(b * kRoundDraws + k) * W + lane];
        const double a0 = nd[1];
        if (bits(a0) == 0) { done = true; break; }
        const double tn = advance_clock(t, e, rcp_pos(a0));
        if (bits(tn) > tau_bits) { t_stop = tn; done = true; break; }
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
          if (E.feedback == 2) { done = true; break; }             // absorbed at its first passage
          for (int s = 0; s < E.S; ++s) xme[s * W] = E.recycle[r * E.S + s];
        }
        rebuild();
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
  if (warp == 0 && live) finish_walker(prm, r, g, par, xme, W, t, nev, nrec, status, near_tau_fp64(E.tau, t, t_stop));
  }
}

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

// State-indexed tables, pipelined.  The chain of states does not depend on the clock (a draw
// picks the reaction from the current row; the count moves; a recycle resets it), so a block
// splits each walker's events into three streams that run one round apart:
//   warp 0     the state chain of round p as if every draw fires: for each draw, the wait scale
//              of the current row and the count after the event, plus flags for a row that
//              cannot fire (a0 = 0), an event that would overflow, and an event that recycles;
//   warp 1     round p-1: every draw's waiting time in clock units (independent of one
//              another), then the clock in draw order -- the first draw that cannot fire (idle,
//              past tau, step cap, overflow) ends the interval and fixes the committed state;
//   warps 2-3  the draws (Philox + logarithm) of round p+1.
// A phase ends at one block barrier.  Draw buffers rotate over three rounds and the state
// buffers over two; done flags reach warp 0 one phase after warp 1 sets them, so warp 0 may
// run one round past a walker's end (that work is discarded).  The committed arithmetic is
// the same as the serial loop's: the same reaction for each draw, the same waiting time, the
// same order of clock additions.
template <int P, int LOG2P, int D>
__global__ void __launch_bounds__(128, 3) k_propagate_pipe(PropagateParams prm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Smem sm = load_smem<P>(prm, smem_raw);
  const EnsView &E = prm.ens;
  const TableView &TV = prm.tab;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int W = 32, K = kRoundDraws;
  int32_t *s_dx = sm.xs + E.S * W;                                       // P (species)
  int32_t *s_dy = s_dx + P;                                              // P (species2)
  unsigned long long *qm = reinterpret_cast<unsigned long long *>(
      (reinterpret_cast<uintptr_t>(s_dy + P) + 15) & ~(uintptr_t)15);    // [3][K][W]
  float2 *qe = reinterpret_cast<float2 *>(qm + 3 * K * W);              // [3][K][W]
  float2 *sw = qe + 3 * K * W;                                          // [2][K][W] wait scales
  int32_t *sx = reinterpret_cast<int32_t *>(sw + 2 * K * W);            // [2][K][W] counts
  int32_t *sy = sx + 2 * K * W;                                         // [2][K][W] (species2)
  uint32_t *sfl = reinterpret_cast<uint32_t *>(sy + 2 * K * W);         // [2][3][W] flag masks
  unsigned long long *s_tab = reinterpret_cast<unsigned long long *>(
      (reinterpret_cast<uintptr_t>(sfl + 2 * 3 * W) + 15) & ~(uintptr_t)15);
  __shared__ int s_more[2], s_win, s_win_n;
  __shared__ int s_done[2][W];
  for (int j = threadIdx.x; j < P; j += blockDim.x) {
    int dx = 0, dy = 0;
    for (int q = sm.meta[j].d_begin; q < sm.meta[j].d_end; ++q) {
      if (sm.dsp[q] == TV.species) dx += sm.dval[q];
      if (sm.dsp[q] == TV.species2) dy += sm.dval[q];
    }
    s_dx[j] = dx;
    s_dy[j] = dy;
  }
  // Persistent blocks: each takes groups of 32 walkers (vb) until every live walker is served,
  // so the shared prologue above is paid once per resident block, not once per capacity slot.
  const int n_live_all = E.run_off[E.R];
  for (int vb = blockIdx.x; vb * 32 < n_live_all; vb += gridDim.x) {
  __syncthreads();                                       // the previous group's buffers are free

  const int iter = *E.iter;
  const int total = E.run_off[E.R];
  const int f = vb * W + lane;
  const bool live = f < total;
  const int r = !live ? 0 : (E.R == 1 ? 0 : find_run(E.run_off, E.R, f));
  const int w = live ? f - E.run_off[r] : 0;
  const uint32_t k0 = (uint32_t)E.seed;
  const uint32_t k1 = (uint32_t)(E.seed >> 32) + E.run_id[r];
  const LogTables &LT = *sm.logt;
  const int g = r * E.cap + w;
  const int par = iter & 1;
  const int ld = E.R * E.cap;
  const int ps = live ? E.param_set[r] : 0;
  const unsigned long long *tab = TV.rows + (size_t)ps * TV.len * TV.lenB * P;

  // table rows for a window of counts around this block's walkers, in shared memory
  int win_lo = 0, win_n = 0;
  if (D == 1 && TV.smem_rows > 0) {
    if (warp == 0) {
      int lo = 0x7fffffff, hi = -1;
      if (live) lo = hi = E.x[par][(size_t)TV.species * ld + g];
      lo = __reduce_min_sync(0xffffffffu, lo);
      hi = __reduce_max_sync(0xffffffffu, hi);
      const int ps0 = __shfl_sync(0xffffffffu, ps, 0);
      const bool one_set = __all_sync(0xffffffffu, !live || ps == ps0);
      if (lane == 0) {
        const int n = min(TV.smem_rows, hi - lo + 1 + 2 * kWindowMargin);
        int start = (lo + hi) / 2 - n / 2;
        start = max(min(start, TV.len - n), 0);
        s_win = (one_set && hi >= 0) ? start : -1;           // no live walker: nothing to stage
        s_win_n = n;
      }
    }
    __syncthreads();
    if (s_win >= 0) {
      win_lo = s_win;
      win_n = s_win_n;
      const int ps0 = E.param_set[E.R == 1 ? 0 : find_run(E.run_off, E.R, vb * W)];
      const unsigned long long *src = TV.rows + ((size_t)ps0 * TV.len + win_lo) * P;
      for (int i = threadIdx.x; i < win_n * P; i += blockDim.x) s_tab[i] = src[i];
    }
  }

  auto produce = [&](int buf, uint32_t base, int first, int stride) {
    if (!live) return;
#pragma unroll 1
    for (int k = first; k < K; k += stride) {
      unsigned long long m2;
      float2 e;
      ssa_draw(base + (uint32_t)k, (uint32_t)iter, (uint32_t)w, k0, k1, LT, m2, e);
      qm[(buf * K + k) * W + lane] = m2;
      qe[(buf * K + k) * W + lane] = e;
    }
  };
  produce(0, 0u, warp, 4);                               // round 0: all four warps
  // absorbing target: a walker that starts the interval inside it fires nothing
  bool absorbed0 = false;
  if (warp == 1 && live && E.feedback == 2) {
    absorbed0 = true;
    for (int c = 0; c < E.n_clauses; ++c) {
      const int v = E.x[par][(size_t)E.tgt_species[c] * ld + g];
      const int thr = E.tgt_thr[r * E.n_clauses + c];
      absorbed0 = absorbed0 && (E.tgt_op[c] == 0 ? v >= thr : v <= thr);
    }
  }
  if (warp == 1) {
    s_done[1][lane] = !live || absorbed0;
    if (lane == 0) s_more[1] = 1;
  }

  int32_t *xme = sm.xs + lane;
  const double *keff = sm.keff + ps * P;
  const double *Kn = sm.Kn + ps * P;
  // warp 0: the speculative state chain
  int x = 0, y = 0, dxr[P], dyr[P];                      // y: count of species2 (D = 2)
  TableRow<P, LOG2P> row;
  double fb[2 * P];
  int xlo = -1, xhi = kMaxCount + 1, xrec = 0;
  int ylo = -1, yhi = kMaxCount + 1, yrec = 0;
  bool ok = false, ok_rec = false;
  auto in_table = [&](int xv, int yv) { return xv < TV.len && (D == 1 || yv < TV.lenB); };
  auto table_row = [&](int xv, int yv) { return tab + ((size_t)xv * TV.lenB + (D == 2 ? yv : 0)) * P; };
  auto load_row = [&](int xv, int yv) {
    const unsigned off = (unsigned)(xv - win_lo);
    if (D == 1 && off < (unsigned)win_n) {
      row.read(s_tab + (size_t)off * P);
    } else if (in_table(xv, yv)) {
      row.read(table_row(xv, yv));
    } else {
      xme[TV.species * W] = xv;
      if (D == 2) xme[TV.species2 * W] = yv;
      row.w = evaluate_row<P, LOG2P>(fb, sm.meta, keff, Kn, xme, W, TV.clock_scale);
      row.direct = true;
    }
  };
  // warp 1: the committed walker
  unsigned long long clk = 0;                           // clock units of tau / 2^62
  unsigned long long stop_u = 0;                        // clock of the first draw past tau (0: none)
  long long nev = 0;
  int xc = 0, yc = 0, nrec = 0, status = 0;
  bool done = !live || absorbed0, recycled = false;
  if (live && warp <= 1) {
    if (warp == 0)
      for (int s = 0; s < E.S; ++s) xme[s * W] = E.x[par][(size_t)s * ld + g];
    xc = E.x[par][(size_t)TV.species * ld + g];
    if (D == 2) yc = E.x[par][(size_t)TV.species2 * ld + g];
  }
  __syncthreads();
  if (warp == 0 && live) {
#pragma unroll
    for (int j = 0; j < P; ++j) { dxr[j] = s_dx[j]; dyr[j] = s_dy[j]; }
    x = xc;
    y = yc;
    if (E.feedback) {
      ok = true;
      ok_rec = true;
      for (int c = 0; c < E.n_clauses; ++c) {
        const int thr = E.tgt_thr[r * E.n_clauses + c];
        const int sp = E.tgt_species[c];
        if (sp == TV.species) {
          if (E.tgt_op[c] == 0) xlo = max(xlo, thr); else xhi = min(xhi, thr);
        } else if (D == 2 && sp == TV.species2) {
          if (E.tgt_op[c] == 0) ylo = max(ylo, thr); else yhi = min(yhi, thr);
        } else {
          const int v = xme[sp * W], vr = E.recycle[r * E.S + sp];
          ok = ok && (E.tgt_op[c] == 0 ? v >= thr : v <= thr);
          ok_rec = ok_rec && (E.tgt_op[c] == 0 ? vr >= thr : vr <= thr);
        }
      }
      xrec = E.recycle[r * E.S + TV.species];
      if (D == 2) yrec = E.recycle[r * E.S + TV.species2];
    }
    load_row(x, y);
  }

  for (int p = 0;; ++p) {
    if (warp == 0) {
      const int qb = p % 3, sb = p & 1;
      if (live && !s_done[sb ^ 1][lane]) {
        uint32_t idle_m = 0u, ovf_m = 0u, rec_m = 0u;
        // one draw of the chain; `fast` rows come from the table only (no calls in the
        // unrolled loop), rows beyond it are evaluated in the tail loop below
        auto step = [&](int k, bool fast) {
          const unsigned long long m2 = qm[(qb * K + k) * W + lane];
          sw[(sb * K + k) * W + lane] = row.w;
          if (row.idle()) idle_m |= 1u << k;
          const int j = (!fast && row.direct) ? descend_row<P, LOG2P>(fb, m2) : row.select_table(m2);
          int dx = dxr[0], dy = dyr[0];
#pragma unroll
          for (int i = 1; i < P; ++i) { dx = (j == i) ? dxr[i] : dx; dy = (j == i) ? dyr[i] : dy; }
          int nx = x + dx, ny = D == 2 ? y + dy : 0;
          if (nx > kMaxCount || ny > kMaxCount) { ovf_m |= 1u << k; nx = x; ny = y; }
          if (E.feedback && ok && nx >= xlo && nx <= xhi && (D == 1 || (ny >= ylo && ny <= yhi))) {
            rec_m |= 1u << k;
            if (E.feedback == 1) { nx = xrec; ny = yrec; ok = ok_rec; }   // absorbing: stays inside
          }
          sx[(sb * K + k) * W + lane] = nx;
          if (D == 2) sy[(sb * K + k) * W + lane] = ny;
          x = nx;
          y = ny;
        };
        int k = 0;
        if (!row.direct) {
          // the first draw after which the count leaves the table (its later draws in this
          // loop ran on a stale row and are redone below from the state saved here)
          int out_at = K;
          int x_out = 0, y_out = 0;
          bool ok_out = false;
#pragma unroll 4
          for (int kk = 0; kk < K; ++kk) {
            step(kk, true);
            const unsigned off = (unsigned)(x - win_lo);
            if (D == 1 && off < (unsigned)win_n) row.read(s_tab + (size_t)off * P);
            else if (in_table(x, y)) row.read(table_row(x, y));
            else if (out_at == K) { out_at = kk; x_out = x; y_out = y; ok_out = ok; }
          }
          k = K;
          if (out_at < K) {
            const uint32_t keep = (2u << out_at) - 1u;      // draws 0 .. out_at stand
            idle_m &= keep;
            ovf_m &= keep;
            rec_m &= keep;
            x = x_out;
            y = y_out;
            ok = ok_out;
            load_row(x, y);
            k = out_at + 1;
          }
        }
        for (; k < K; ++k) {                                // rows beyond the table
          step(k, false);
          load_row(x, y);
        }
        sfl[(sb * 3 + 0) * W + lane] = idle_m;
        sfl[(sb * 3 + 1) * W + lane] = ovf_m;
        sfl[(sb * 3 + 2) * W + lane] = rec_m;
      }
    } else if (warp == 1) {
      const int sb = p & 1;
      if (p >= 1) {
        const int qb = (p - 1) % 3, pb = sb ^ 1;
        if (!done) {
          // waiting times (independent), the clock after each draw, and the first draw that
          // cannot fire: idle row, waiting time or clock past tau (no status), else the step
          // cap, else an overflow -- the order of the checks in the serial loop
          unsigned long long dts[K];
          uint32_t far_m = 0u, over_m = 0u;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const float2 e = qe[(qb * K + k) * W + lane];
            const float2 wv = sw[(pb * K + k) * W + lane];
            if (!wait_units(e, wv, dts[k])) far_m |= 1u << k;
          }
          // the clock after each draw: exact up to the first draw that cannot fire (before it
          // the clock is at most 2^62 and a waiting time below 2^63 + 2^40, so no wrap)
          unsigned long long c = clk;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            c += dts[k];
            if (c > kClockTau) over_m |= 1u << k;
          }
          const uint32_t idle_m = sfl[(pb * 3 + 0) * W + lane];
          const uint32_t ovf_m = sfl[(pb * 3 + 1) * W + lane];
          const uint32_t rec_m = sfl[(pb * 3 + 2) * W + lane];
          const long long room = E.max_steps - nev;       // draws that may still fire
          const uint32_t cap_m = room >= K ? 0u : ((0xffffu << (int)room) & 0xffffu);
          // absorbing target: nothing fires after the draw that enters it
          const uint32_t absorb_m = E.feedback == 2 ? ((rec_m << 1) & 0xffffu) : 0u;
          const uint32_t quiet_m = idle_m | far_m | over_m | absorb_m;
          const uint32_t stop_m = (quiet_m | cap_m | ovf_m) & 0xffffu;
          const int kstop = stop_m ? __ffs(stop_m) - 1 : K;
          const uint32_t fired = (1u << kstop) - 1u;
          unsigned long long cs = clk;
#pragma unroll
          for (int k = 0; k < K; ++k) cs += (k < kstop) ? dts[k] : 0ull;
          clk = cs;
          nev += kstop;
          nrec += __popc(rec_m & fired);
          recycled = recycled || (rec_m & fired) != 0u;
          if (E.feedback == 2 && (rec_m & fired)) done = true;
          if (kstop > 0) {
            xc = sx[(pb * K + kstop - 1) * W + lane];
            if (D == 2) yc = sy[(pb * K + kstop - 1) * W + lane];
          }
          if (kstop < K) {
            done = true;
            const uint32_t bit = 1u << kstop;
            if (!(quiet_m & bit)) status = (cap_m & bit) ? kStatusStepCap : kStatusOverflow;
            else if ((over_m & bit) && !((idle_m | far_m | absorb_m) & bit)) {
              unsigned long long ds = 0;                 // the stopping draw's waiting time
#pragma unroll
              for (int k = 0; k < K; ++k) ds = (k == kstop) ? dts[k] : ds;
              stop_u = clk + ds;
            }
          }
        }
        s_done[sb][lane] = done;
        const int more = __any_sync(0xffffffffu, !done);
        if (lane == 0) s_more[sb] = more;
      } else {
        s_done[0][lane] = done;
        if (lane == 0) s_more[0] = 1;
      }
    } else {
      produce((p + 1) % 3, (uint32_t)((p + 1) * K), warp - 2, 2);
    }
    __syncthreads();
    if (!s_more[p & 1]) break;
  }
  if (warp == 1 && live) {
    if (recycled && E.feedback == 1)                     // the other species take the recycle state
      for (int s = 0; s < E.S; ++s) xme[s * W] = E.recycle[r * E.S + s];
    xme[TV.species * W] = xc;
    if (D == 2) xme[TV.species2 * W] = yc;
    finish_walker(prm, r, g, par, xme, W, clock_time(clk, E.tau), (long long)nev, nrec, status,
                  near_tau_units(clk, stop_u));
  }
  }
}

size_t propagate_thread_smem(const NetView &N, int block, bool table) {
  return sizeof(LogTables) + (size_t)N.P * sizeof(RxnMeta) +
         2 * (size_t)N.n_param_sets * N.P * sizeof(double) + 2 * (size_t)N.n_delta * sizeof(int32_t) +
         (size_t)N.S * block * sizeof(int32_t) + (table ? 2 * (size_t)N.P * sizeof(int32_t) : 0);
}

static size_t smem_prologue(const NetView &N) {
  return sizeof(LogTables) + (size_t)N.P * sizeof(RxnMeta) +
         2 * (size_t)N.n_param_sets * N.P * sizeof(double) + 2 * (size_t)N.n_delta * sizeof(int32_t) +
         (size_t)N.S * 32 * sizeof(int32_t);
}

size_t propagate_ws_smem(const NetView &N) {
  return smem_prologue(N) + 16 + 2 * (size_t)kRoundDraws * 32 * (sizeof(unsigned long long) + sizeof(float2));
}

size_t propagate_pipe_smem(const NetView &N, int table_rows) {
  return smem_prologue(N) + 2 * (size_t)N.P * sizeof(int32_t) + 16 +
         3 * (size_t)kRoundDraws * 32 * (sizeof(unsigned long long) + sizeof(float2)) +
         2 * (size_t)kRoundDraws * 32 * (sizeof(float2) + 2 * sizeof(int32_t)) + 2 * 3 * 32 * sizeof(uint32_t) + 16 +
         (size_t)table_rows * N.P * sizeof(unsigned long long);
}

cudaError_t launch_init_log_tables(LogTables *T, cudaStream_t st) {
  k_init_log_tables<<<1, 128, 0, st>>>(T);
  return cudaGetLastError();
}

template <int P, int L>
static cudaError_t build_table_p(const NetView &N, const int32_t *base, int species, int species2, int len,
                                 int lenB, double clock_scale, unsigned long long *rows, cudaStream_t st) {
  const int n_rows = len * lenB;
  int gx = (n_rows + 127) / 128;
  if (gx > 4096) gx = 4096;
  dim3 grid(gx, N.n_param_sets);
  k_build_table<P, L><<<grid, 128, 0, st>>>(N, base, species, species2, len, lenB, clock_scale, rows);
  return cudaGetLastError();
}

cudaError_t launch_build_table(const NetView &N, const int32_t *base, int species, int species2, int len,
                               int lenB, double clock_scale, unsigned long long *rows, cudaStream_t st) {
  switch (N.P) {
    case 1: return build_table_p<1, 0>(N, base, species, species2, len, lenB, clock_scale, rows, st);
    case 2: return build_table_p<2, 1>(N, base, species, species2, len, lenB, clock_scale, rows, st);
    case 4: return build_table_p<4, 2>(N, base, species, species2, len, lenB, clock_scale, rows, st);
    case 8: return build_table_p<8, 3>(N, base, species, species2, len, lenB, clock_scale, rows, st);
    case 16: return build_table_p<16, 4>(N, base, species, species2, len, lenB, clock_scale, rows, st);
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
static int pipe_table_rows(K kern, const PropagateParams &prm, int grid) {
  if (prm.tab.species < 0 || prm.tab.len <= 0 || prm.tab.species2 >= 0) return 0;   // 1-D window only
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) { cudaGetLastError(); return 0; }
  const int by_regs = std::max(1, 65536 / std::max(1, fa.numRegs * 128));
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
static int persistent_grid(K kern, int groups) {
  cudaFuncAttributes fa;
  int per_sm = 4;
  if (cudaFuncGetAttributes(&fa, kern) == cudaSuccess && fa.numRegs > 0)
    per_sm = std::max(1, std::min(16, 65536 / (fa.numRegs * 128)));
  else
    cudaGetLastError();
  return std::max(1, std::min(groups, per_sm * num_sms()));
}

template <typename K>
static cudaError_t launch_pipe(K kern, const PropagateParams &prm_in, int groups, cudaStream_t st) {
  PropagateParams prm = prm_in;
  const int grid = persistent_grid(kern, groups);
  prm.tab.smem_rows = pipe_table_rows(kern, prm, grid);
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

cudaError_t launch_propagate_ws(const PropagateParams &prm, bool table, cudaStream_t st) {
  const int total_slots = prm.ens.R * prm.ens.cap;
  const int grid = (total_slots + 31) / 32;
  const size_t smem = propagate_ws_smem(prm.net);
#define WE_CASE(PP, LL)                                                                  \
  case PP:                                                                               \
    return table ? (prm.tab.species2 >= 0 ? launch_pipe(k_propagate_pipe<PP, LL, 2>, prm, grid, st)       \
                                          : launch_pipe(k_propagate_pipe<PP, LL, 1>, prm, grid, st)) \
                 : launch_ws(k_propagate_ws<PP, LL>, prm, grid, smem, st);
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
