// we_pipe.cuh -- the pipelined SSA kernel for networks with state-indexed tables, a template
// on the table shape and on the blocks per SM it is compiled for.  Its two builds live in
// translation units of their own (we_pipe3.cu, we_pipe4.cu) so that they compile in parallel.
#pragma once
#include "we_propagate_common.cuh"

namespace we {

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
//
// MINB, the blocks per SM the kernel is compiled for: 3 (155 registers) when the launch has few
// walker groups and the slowest group's chain sets its time; 4 (128 registers) when groups
// outnumber the resident blocks and the SMs' throughput does.
template <int P, int LOG2P, int D, int MINB>
__global__ void __launch_bounds__(128, MINB) k_propagate_pipe(PropagateParams prm) {
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
  __shared__ int s_win, s_win_n, s_rwin, s_rwin_n;
  __shared__ int s_done[2][W];
  // Roles by sub-partition (the 3-blocks build, for launches whose slowest chain sets the time):
  // the state chain goes to this block's warp on the lowest scheduler index, then the clock,
  // then the draws, so that in every block the same role lands on the same sub-partition and a
  // chain warp does not share its scheduler with another block's draw warps (measured: SSA launch
  // 0.0889 -> 0.0857 ms on the Schloegl MFPT workload; the 4-blocks build, whose launches are
  // throughput-bound, keeps the roles by warp index: 3 % faster there).  Only performance
  // depends on this (a warp's slot may change after a preemption); every assignment of the four
  // roles gives the same results.
  __shared__ int s_role[4], s_sp[4];
  if (MINB <= 3) {
    unsigned wid;
    asm volatile("mov.u32 %0, %%warpid;" : "=r"(wid));
    if (lane == 0) s_sp[warp] = (int)(wid & 3u);
    __syncthreads();
    if (threadIdx.x == 0) {
      int taken = 0;
      for (int k = 0; k < 4; ++k) {                        // role k: the free warp on the lowest index
        int best = -1;
        for (int w = 0; w < 4; ++w)
          if (!((taken >> w) & 1) && (best < 0 || s_sp[w] < s_sp[best])) best = w;
        s_role[best] = k;
        taken |= 1 << best;
      }
    }
    __syncthreads();
  }
  const int role = MINB <= 3 ? s_role[warp] : warp;
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
  const unsigned long long *tab = TV.rows + (size_t)ps * TV.len * TV.lenB * P;

  // table rows for a window of counts around this block's walkers, in shared memory, and a
  // second one around the recycle count: a walker that enters the target mid-interval goes on
  // from there, and one lane reading its rows from global memory would hold up the whole chain
  int win_lo = 0, win_n = 0, rec_lo = 0, rec_n = 0;
  if (D == 1 && TV.smem_rows > 0) {
    if (warp == 0) {
      int lo = 0x7fffffff, hi = -1, rlo = 0x7fffffff, rhi = -1;
      if (live) lo = hi = E.x[par][(size_t)TV.species * ld + g];
      if (live && E.feedback == 1) rlo = rhi = E.recycle[r * E.S + TV.species];
      lo = __reduce_min_sync(0xffffffffu, lo);
      hi = __reduce_max_sync(0xffffffffu, hi);
      rlo = __reduce_min_sync(0xffffffffu, rlo);
      rhi = __reduce_max_sync(0xffffffffu, rhi);
      const int ps0 = __shfl_sync(0xffffffffu, ps, 0);
      const bool one_set = __all_sync(0xffffffffu, !live || ps == ps0);
      if (lane == 0) {
        int n2 = (rhi >= 0 && rlo == rhi) ? min(2 * kWindowMargin + 1, TV.smem_rows / 4) : 0;
        const int n = min(TV.smem_rows - n2, hi - lo + 1 + 2 * kWindowMargin);
        int start = (lo + hi) / 2 - n / 2;
        start = max(min(start, TV.len - n), 0);
        s_win = (one_set && hi >= 0) ? start : -1;           // no live walker: nothing to stage
        s_win_n = n;
        if (rhi - kWindowMargin >= start && rhi + kWindowMargin < start + n) n2 = 0;   // in the first
        s_rwin = max(min(rhi - n2 / 2, TV.len - n2), 0);
        s_rwin_n = n2;
      }
    }
    __syncthreads();
    if (s_win >= 0) {
      win_lo = s_win;
      win_n = s_win_n;
      rec_lo = s_rwin;
      rec_n = s_rwin_n;
      const int ps0 = E.param_set[E.R == 1 ? 0 : find_run(E.run_off, E.R, vb * W)];
      const unsigned long long *src = TV.rows + ((size_t)ps0 * TV.len + win_lo) * P;
      for (int i = threadIdx.x; i < win_n * P; i += blockDim.x) s_tab[i] = src[i];
      const unsigned long long *src2 = TV.rows + ((size_t)ps0 * TV.len + rec_lo) * P;
      for (int i = threadIdx.x; i < rec_n * P; i += blockDim.x) s_tab[(size_t)win_n * P + i] = src2[i];
    }
  }
  // position of count xv's row among the staged rows, or -1
  auto staged = [&](int xv) {
    const unsigned o1 = (unsigned)(xv - win_lo), o2 = (unsigned)(xv - rec_lo);
    return o1 < (unsigned)win_n ? (int)o1 : (o2 < (unsigned)rec_n ? win_n + (int)o2 : -1);
  };

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
  produce(0, 0u, role, 4);                               // round 0: all four warps
  // absorbing target: a walker that starts the interval inside it fires nothing
  bool absorbed0 = false;
  if (role == 1 && live && E.feedback == 2) {
    absorbed0 = true;
    for (int c = 0; c < E.n_clauses; ++c) {
      const int v = E.x[par][(size_t)E.tgt_species[c] * ld + g];
      const int thr = E.tgt_thr[r * E.n_clauses + c];
      absorbed0 = absorbed0 && (E.tgt_op[c] == 0 ? v >= thr : v <= thr);
    }
  }
  if (role == 1) s_done[1][lane] = !live || absorbed0;

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
    const int at = D == 1 ? staged(xv) : -1;
    if (at >= 0) {
      row.read(s_tab + (size_t)at * P);
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
  if (live && role <= 1) {
    if (role == 0)
      for (int s = 0; s < E.S; ++s) xme[s * W] = E.x[par][(size_t)s * ld + g];
    xc = E.x[par][(size_t)TV.species * ld + g];
    if (D == 2) yc = E.x[par][(size_t)TV.species2 * ld + g];
  }
  __syncthreads();
  if (role == 0 && live) {
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

  // One loop per role, each ending its phase at the same block barrier, whose OR (from the
  // clock warp) tells every warp whether any walker goes on.
  if (role == 0) {
    for (int p = 0;; ++p) {
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
            const int at = D == 1 ? staged(x) : -1;
            if (at >= 0) row.read(s_tab + (size_t)at * P);
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
      if (!__syncthreads_or(0)) break;
    }
  } else if (role == 1) {
    for (int p = 0;; ++p) {
      int go = 0;                                        // this walker goes on
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
        go = !done;
      } else {
        s_done[0][lane] = done;
        go = 1;
      }
      if (!__syncthreads_or(go)) break;
    }
  } else {
    for (int p = 0;; ++p) {
      produce((p + 1) % 3, (uint32_t)((p + 1) * K), role - 2, 2);
      if (!__syncthreads_or(0)) break;
    }
  }
  if (role == 1 && live) {
    if (recycled && E.feedback == 1)                     // the other species take the recycle state
      for (int s = 0; s < E.S; ++s) xme[s * W] = E.recycle[r * E.S + s];
    xme[TV.species * W] = xc;
    if (D == 2) xme[TV.species2 * W] = yc;
    finish_walker(prm, r, g, par, iter, xme, W, clock_time(clk, E.tau), (long long)nev, nrec, status,
                  near_tau_units(clk, stop_u));
  }
  }
}

// Launch the pipelined kernel compiled for MINB blocks per SM for the ensemble's table shape.
template <int MINB>
static cudaError_t launch_pipe_minb(const PropagateParams &prm, int groups, cudaStream_t st) {
  const bool two = prm.tab.species2 >= 0;
  switch (prm.net.P) {
    case 1: return two ? launch_pipe(k_propagate_pipe<1, 0, 2, MINB>, prm, groups, st, MINB)
                       : launch_pipe(k_propagate_pipe<1, 0, 1, MINB>, prm, groups, st, MINB);
    case 2: return two ? launch_pipe(k_propagate_pipe<2, 1, 2, MINB>, prm, groups, st, MINB)
                       : launch_pipe(k_propagate_pipe<2, 1, 1, MINB>, prm, groups, st, MINB);
    case 4: return two ? launch_pipe(k_propagate_pipe<4, 2, 2, MINB>, prm, groups, st, MINB)
                       : launch_pipe(k_propagate_pipe<4, 2, 1, MINB>, prm, groups, st, MINB);
    case 8: return two ? launch_pipe(k_propagate_pipe<8, 3, 2, MINB>, prm, groups, st, MINB)
                       : launch_pipe(k_propagate_pipe<8, 3, 1, MINB>, prm, groups, st, MINB);
    case 16: return two ? launch_pipe(k_propagate_pipe<16, 4, 2, MINB>, prm, groups, st, MINB)
                        : launch_pipe(k_propagate_pipe<16, 4, 1, MINB>, prm, groups, st, MINB);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace we
