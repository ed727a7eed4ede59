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

#include "we_propagate_common.cuh"

namespace we {

cudaError_t launch_pipe_blocks3(const PropagateParams &prm, int groups, cudaStream_t st);
cudaError_t launch_pipe_blocks4(const PropagateParams &prm, int groups, cudaStream_t st);

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
// ------------------------------------------------------------------------------------------
// Direct evaluation: the canonical propensity tree (P leaves, node k = node 2k + node 2k+1,
// rounded) lives in registers; after unrolling every index into it is a compile-time constant
// and the descent picks children with predicated selects.  Counts sit in shared memory so that
// reactions can name them by runtime index.
// ------------------------------------------------------------------------------------------
template <int P, int LOG2P>
__global__ void __launch_bounds__(128) k_propagate_direct(PropagateParams prm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const EnsView &E = prm.ens;
  const int B = blockDim.x, tid = threadIdx.x;
  // the walker's run, slot and parameters first, so that their loads overlap the prologue
  const int iter = *E.iter;
  const int total = E.run_off[E.R];
  const int f = blockIdx.x * B + tid;
  const bool live = f < total;
  int r_start = 0;
  const int r = (!live || E.R == 1) ? 0 : find_run_start(E.run_off, E.R, f, r_start);
  const int ps = E.param_set[r];
  const uint32_t k0 = (uint32_t)E.seed;
  const uint32_t k1 = (uint32_t)(E.seed >> 32) + E.run_id[r];
  const Smem sm = load_smem<P>(prm, smem_raw);
  if (!live) return;
  const int w = f - r_start;
  const int g = r * E.cap + w;
  const int par = iter & 1;
  const int ld = E.R * E.cap;
  int32_t *xme = sm.xs + tid;
  for (int s = 0; s < E.S; ++s) xme[s * B] = E.x[par][(size_t)s * ld + g];
  const double *keff = sm.keff + ps * P;
  const double *Kn = sm.Kn + ps * P;

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
  finish_walker(prm, r, g, par, iter, xme, B, t, nev, nrec, status, near_tau_fp64(E.tau, t, t_stop));
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
  const EnsView &E = prm.ens;
  const TableView &TV = prm.tab;
  const int B = blockDim.x, tid = threadIdx.x;
  // the walker's run, slot and parameters first, so that their loads overlap the prologue
  const int iter = *E.iter;
  const int total = E.run_off[E.R];
  const int f = blockIdx.x * B + tid;
  const bool live = f < total;
  int r_start = 0;
  const int r = (!live || E.R == 1) ? 0 : find_run_start(E.run_off, E.R, f, r_start);
  const int ps = E.param_set[r];
  const uint32_t k0 = (uint32_t)E.seed;
  const uint32_t k1 = (uint32_t)(E.seed >> 32) + E.run_id[r];
  const int par = iter & 1;
  const int ld = E.R * E.cap;
  const int w = f - r_start;
  const int g = r * E.cap + w;
  const int sx = TV.species, sy = TV.species2;
  // ... and the table species' counts and their row (a count past the table is evaluated below)
  const int x0 = live ? E.x[par][(size_t)sx * ld + g] : 0;
  const int y0 = (live && sy >= 0) ? E.x[par][(size_t)sy * ld + g] : 0;
  const unsigned long long *tab = TV.rows + (size_t)ps * TV.len * TV.lenB * P;
  const bool in_table = x0 < TV.len && y0 < TV.lenB;
  TableRow<P, LOG2P> row;
  if (live && in_table) row.read(tab + ((size_t)x0 * TV.lenB + y0) * P);
  const Smem sm = load_smem<P>(prm, smem_raw);
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
  if (!live) return;
  int32_t *xme = sm.xs + tid;
  for (int s = 0; s < E.S; ++s) xme[s * B] = E.x[par][(size_t)s * ld + g];
  const double *keff = sm.keff + ps * P;
  const double *Kn = sm.Kn + ps * P;

  double fb[2 * P];
  auto load_row = [&](int xv, int yv) {           // xme holds the current counts
    if (xv < TV.len && yv < TV.lenB) row.read(tab + ((size_t)xv * TV.lenB + yv) * P);
    else row.evaluate(fb, sm.meta, keff, Kn, xme, B, TV.clock_scale);
  };
  int x = x0, y = y0;
  if (!in_table) load_row(x, y);

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
  finish_walker(prm, r, g, par, iter, xme, B, clock_time(clk, E.tau), nev, nrec, status, near_tau_units(clk, stop_u));
}

// ------------------------------------------------------------------------------------------
// Warp-specialised kernels: a block of four warps serves 32 walkers (one per lane), and the
// draws (Philox + logarithm, most of the instructions of an event) come from other warps than
// the event chain, through shared-memory buffers that alternate at block barriers.  Every
// wait is a block barrier that all warps reach; a loop ends when every walker is done.
// ------------------------------------------------------------------------------------------

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
  int r_start = 0;
  const int r = (!live || E.R == 1) ? 0 : find_run_start(E.run_off, E.R, f, r_start);
  const int w = live ? f - r_start : 0;
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
  if (warp == 0 && live) finish_walker(prm, r, g, par, iter, xme, W, t, nev, nrec, status, near_tau_fp64(E.tau, t, t_stop));
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

cudaError_t launch_propagate_ws(const PropagateParams &prm, bool table, cudaStream_t st) {
  const int total_slots = prm.ens.R * prm.ens.cap;
  const int grid = (total_slots + 31) / 32;
  // few walker groups (at most four per SM): the launch is set by its slowest group, which the
  // 3-blocks-per-SM build runs faster; more groups: the 4-blocks-per-SM build's throughput
  const bool few = grid <= 4 * num_sms();
  const size_t smem = propagate_ws_smem(prm.net);
  if (table) return few ? launch_pipe_blocks3(prm, grid, st) : launch_pipe_blocks4(prm, grid, st);
#define WE_CASE(PP, LL)                                                                  \
  case PP:                                                                               \
    return launch_ws(k_propagate_ws<PP, LL>, prm, grid, smem, st);
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
