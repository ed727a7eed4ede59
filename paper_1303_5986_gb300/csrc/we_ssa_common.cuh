// we_ssa_common.cuh -- device helpers shared by the SSA kernels: the counter-based generator,
// uniforms, propensities, bins, the target test, waiting-time pieces (a table-driven -log u and
// a Newton reciprocal).
//
// Floating-point rules: every operation that decides which reaction fires (propensities, tree
// nodes, the target u2*a0 and the descent subtractions) is one IEEE double operation with an
// explicit round-to-nearest intrinsic, so no multiply-add is ever fused there and the device
// reaches the same bits as the definition.  Comparisons between non-negative doubles use their
// bit patterns (for non-negative doubles the IEEE order is the integer order of the bits), which
// keeps compares off the FP64 pipe.  The waiting time only decides when the interval ends; it is
// computed to about one part in 1e15 (see neg_log_u01 and rcp_pos).
#pragma once
#include "we_internal.cuh"

namespace we {

constexpr int32_t kStatusStepCap = -5;
constexpr int32_t kStatusOverflow = -4;

// Philox-4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two 32x32->64 multiplies
// whose high halves are xored with the other counter words and the key; the key advances by
// the Weyl constants between rounds.
__device__ __forceinline__ void philox4x32_10(uint32_t &c0, uint32_t &c1, uint32_t &c2,
                                              uint32_t &c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// (2m+1)/2^53 with m = hi<<20 | lo>>12: the double 1 + m/2^52 built from bits, minus
// (1 - 2^-53).  The difference is representable, so the subtraction is exact.
__device__ __forceinline__ double u01(uint32_t hi, uint32_t lo) {
  const unsigned long long m = ((unsigned long long)hi << 20) | (unsigned long long)(lo >> 12);
  const double one_plus = __longlong_as_double((long long)(0x3FF0000000000000ull | m));
  return __dsub_rn(one_plus, 0x1.fffffffffffffp-1);
}

__device__ __forceinline__ long long bits(double x) { return __double_as_longlong(x); }

__device__ __forceinline__ long long binom_small(long long x, int m) {
  return m == 1 ? x : (m == 2 ? x * (x - 1) / 2 : x * (x - 1) * (x - 2) / 6);
}

// Propensity of one reaction from counts held at xs[species * stride].
__device__ __forceinline__ double propensity(const RxnMeta &mt, double keff, double Kn,
                                             const int32_t *xs, int stride) {
  if (mt.law == 1) {
    const long long y = xs[mt.hsp * stride];
    long long yn = y;
    if (mt.hn >= 2) yn *= y;
    if (mt.hn >= 3) yn *= y;
    const double den = __dadd_rn(Kn, __ll2double_rn(yn));
    return __ddiv_rn(keff, den);
  }
  long long h = 1;
  for (int k = 0; k < mt.n_reac; ++k) h *= binom_small(xs[mt.sp[k] * stride], mt.m[k]);
  return __dmul_rn(keff, __ll2double_rn(h));
}

__device__ __forceinline__ float bf16_to_f32(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

__device__ __forceinline__ float silu_f(float a) { return __fdiv_rn(a, __fadd_rn(1.0f, expf(-a))); }

// First layer of the learned coordinate (see MlpView) for one state: h1 = silu(W1 phi + b1),
// accumulated input by input so that each log1p is taken once; zero beyond the hidden width,
// and all zero for an invalid sample (whose counts are not read).  Hidden width at most 64.
__device__ __forceinline__ void mlp_layer1(const MlpView &m, const int32_t *xs, int stride, bool valid,
                                           float (&h1)[64]) {
#pragma unroll
  for (int o = 0; o < 64; ++o) h1[o] = 0.0f;
  if (!valid) return;
  for (int i = 0; i < m.n_in; ++i) {
    const float phi = log1pf((float)xs[i * stride]);
#pragma unroll
    for (int o = 0; o < 64; ++o)
      if (o < m.hidden) h1[o] = __fmaf_rn(bf16_to_f32(m.w1[o * m.n_in + i]), phi, h1[o]);
  }
#pragma unroll
  for (int o = 0; o < 64; ++o)
    if (o < m.hidden) h1[o] = silu_f(__fadd_rn(h1[o], m.b1[o]));
}

// Bin of a z value among n_bins intervals [zedges[k], zedges[k+1]) (clamped at both ends).
__device__ __forceinline__ int z_bin(const BinView &bv, float z) {
  int lo = 0, hi = bv.n_bins - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bv.zedges[mid] <= z) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Grid bin of a state (learned bins are assigned by k_learned_bins after the SSA kernel).
__device__ __forceinline__ int bin_of(const BinView &bv, const int32_t *xs, int stride) {
  int flat = 0;
#pragma unroll 1
  for (int d = 0; d < bv.ndim; ++d) {
    const int xv = xs[bv.species[d] * stride];
    int lo = 0;
    if (bv.ustep[d] > 0) {
      // the last k in 1..nb-1 with e_k = e_1 + (k - 1) h <= x, else 0 (the search below, exactly)
      if (xv >= bv.ufirst[d]) {
        const unsigned q = ((unsigned)xv - (unsigned)bv.ufirst[d]) / (unsigned)bv.ustep[d];
        lo = q >= (unsigned)(bv.nb[d] - 2) ? bv.nb[d] - 1 : (int)q + 1;
      }
    } else {
      const double v = (double)xv;
      const double *e = bv.edges + bv.edge_off[d];
      int hi = bv.nb[d] - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (e[mid] <= v) lo = mid; else hi = mid - 1;
      }
    }
    flat = flat * bv.nb[d] + lo;
  }
  return flat;
}

__device__ __forceinline__ bool in_target(const EnsView &E, int r, const int32_t *xs, int stride) {
  bool in = true;
#pragma unroll 1
  for (int c = 0; c < E.n_clauses; ++c) {
    const int v = xs[E.tgt_species[c] * stride];
    const int thr = E.tgt_thr[r * E.n_clauses + c];
    in = in && (E.tgt_op[c] == 0 ? v >= thr : v <= thr);
  }
  return in;
}

// Absorbing runs (feedback 2; the brute-force transition-time runs of Sec. II.C): the first-
// passage time of the walker in slot g from the run's start, fl(fl(iter tau) + t) for an
// entrance at time t of this interval.  A walker inside the target set that did not enter it in
// this interval was inside at the interval's start: its time is the start, fl(iter tau).
__device__ __forceinline__ void record_first_passage(const EnsView &E, int r, int g, const int32_t *xs,
                                                     int stride, int nrec, double t) {
  if (!(E.fpt[g] < 0.0)) return;
  const double t0 = __dmul_rn((double)*E.iter, E.tau);
  if (nrec) E.fpt[g] = __dadd_rn(t0, t);
  else if (in_target(E, r, xs, stride)) E.fpt[g] = t0;
}

// Stop decisions near the end of the interval.  The waiting times carry a relative error of
// ~1e-14 (float-float logarithm), the oracle's its own rounding, so an event that falls within
// about that of tau may fire in one and not in the other.  A walker's interval counts as near
// when its last fired event or its first draw past tau lies within 2^-40 tau (9.1e-13 tau) of
// tau; such walkers are counted per iteration (WE_OUT_NEAR_TAU) so that a comparison can tell
// a flip from a fault.
__device__ __forceinline__ int near_tau_fp64(double tau, double t_last, double t_stop) {
  const double thr = __dmul_rn(tau, 0x1p-40);
  return (__dsub_rn(tau, t_last) < thr) || (t_stop > 0.0 && __dsub_rn(t_stop, tau) < thr);
}

__device__ __forceinline__ int find_run(const int32_t *run_off, int R, int f) {
  int lo = 0, hi = R;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (run_off[mid] <= f) lo = mid; else hi = mid;
  }
  return lo;
}

// The run holding flat walker index f and the run's first index (run_off ascending from
// run_off[0] = 0).  Up to 16 runs: every offset loaded at once and counted (the last one at or
// below f is the start), one memory latency instead of a chain of log2(R) dependent loads.
__device__ __forceinline__ int find_run_start(const int32_t *run_off, int R, int f, int &start) {
  if (R <= 16) {
    int r = 0, s = 0;
#pragma unroll
    for (int k = 1; k < 16; ++k) {
      const int v = k < R ? run_off[k] : 0x7FFFFFFF;
      if (v <= f) { ++r; s = v; }
    }
    start = s;
    return r;
  }
  const int r = find_run(run_off, R, f);
  start = run_off[r];
  return r;
}

// ------------------------------------------------------------------------------------------
// -log u for u = (2m+1)/2^53, the waiting time in units of 1/a0.
//
// GB300 issues one FP64 instruction of a warp in about 64 cycles per SM sub-partition, so an
// FP64 logarithm (~29 issue slots in the library) would dominate every event.  Here it is
// evaluated in float-float arithmetic -- pairs of floats whose unevaluated sum carries ~48
// bits, with Dekker's and Knuth's error-free sum and the FMA-based error-free product (T. J.
// Dekker, "A floating-point technique for extending the available precision", Numer. Math.
// 18, 1971) -- on the FP32 and integer pipes, following the table-driven method of P. T. P.
// Tang ("Table-driven implementation of the logarithm function in IEEE floating-point
// arithmetic", ACM TOMS 16, 1990):
//   2m+1 = 2^k f with f in [1,2); c_j = 1 + (2j+1)/256 is the centre of the 1/128-wide
//   interval holding f, so f - c_j is an exact integer multiple of 2^-52 and r = (f-c_j)/c_j
//   has |r| <= 2^-8;  log f = log c_j + log1p(r), with log1p(r) = r - r^2/2 + r^3/3 - ...
//   (float-float through r^2, plain float for r^3 onwards: the truncation and rounding are
//   below 4e-15 of the result);
//   -log u = (52-k) ln 2 + B_j - log1p(r),  B_j = -log(c_j/2) > 0.
// Writing the constant as B_j rather than (53-k) ln 2 - log c_j keeps u near 1 (k = 52, f
// near 2) free of cancellation.  Tables hold 1/c_j, B_j and i ln 2, filled once per ensemble
// from CUDA's double log and division.  The result is returned as a float-float; its error is
// below 1.2e-14 max(1, e) (measured against the C library's log over 2e7 draws, including
// the extremes u = 2^-53 and u = 1 - 2^-53), so event times stay within ~1e-14 relative of
// the definition's (the parity tests check them against the CPU oracle).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float2 ff_fast_two_sum(float a, float b) {   // needs |a| >= |b|
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ float2 ff_mul(float2 x, float2 y) {
  const float p = __fmul_rn(x.x, y.x);
  float e = __fmaf_rn(x.x, y.x, -p);
  e = __fmaf_rn(x.x, y.y, e);
  e = __fmaf_rn(x.y, y.x, e);
  return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ float2 ff_add(float2 x, float2 y) {
  const float2 s = ff_two_sum(x.x, y.x);
  return ff_fast_two_sum(s.x, __fadd_rn(s.y, __fadd_rn(x.y, y.y)));
}

// The double equal to a normal float (or zero), built with integer operations so that the
// conversion does not occupy the FP64 pipe.
__device__ __forceinline__ double f2d_bits(float f) {
  const uint32_t b = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
  if ((b & 0x7fffffffu) == 0u) return __longlong_as_double((long long)sign);
  const unsigned long long ex = ((b >> 23) & 0xffu) - 127u + 1023u;
  const unsigned long long man = (unsigned long long)(b & 0x7fffffu) << 29;
  return __longlong_as_double((long long)(sign | (ex << 52) | man));
}

__device__ __forceinline__ float2 neg_log_u01(uint32_t hi, uint32_t lo, const LogTables &T) {
  const unsigned long long m = ((unsigned long long)hi << 20) | (unsigned long long)(lo >> 12);
  const unsigned long long v = 2ull * m + 1ull;               // odd, in [1, 2^53)
  const int lz = __clzll((long long)v);                       // 11..63
  const int k = 63 - lz;                                      // v = 2^k f
  const unsigned long long mant = ((v << lz) << 1) >> 12;     // 52 bits of f - 1
  const int j = (int)(mant >> 45);                            // top 7 of them
  // f - c_j = diff * 2^-52 exactly, |diff| <= 2^44; split into two exact floats
  const long long diff = (long long)mant - (long long)((unsigned long long)(2 * j + 1) << 44);
  // |dh| <= 2^22 and 0 <= dl < 2^22 become floats exactly through the 2^23-offset bit patterns
  const int dh = (int)(diff >> 22);
  const int dl = (int)(diff - ((long long)dh << 22));
  const float fh = __fsub_rn(__int_as_float(0x4B400000 + dh), 12582912.0f);   // 1.5 * 2^23
  const float fl = __fsub_rn(__int_as_float(0x4B000000 | dl), 8388608.0f);    // 2^23
  const float2 d = ff_fast_two_sum(__fmul_rn(fh, 0x1p-30f), __fmul_rn(fl, 0x1p-52f));
  const float4 cb = T.cb[j];                                  // (1/c_j, -log(c_j / 2))
  const float2 r = ff_mul(d, make_float2(cb.x, cb.y));
  const float2 r2 = ff_mul(r, r);
  const float rh = r.x;
  // r^3/3 - r^4/4 + r^5/5 - r^6/6 in float
  const float tail = __fmul_rn(__fmul_rn(__fmul_rn(rh, rh), rh),
                               __fmaf_rn(rh, __fmaf_rn(rh, __fmaf_rn(rh, -1.0f / 6.0f, 0.2f), -0.25f),
                                         1.0f / 3.0f));
  float2 p = ff_add(r, make_float2(-0.5f * r2.x, -0.5f * r2.y));
  p = ff_add(p, make_float2(tail, 0.0f));                     // log1p(r)
  float2 e = ff_add(T.n_ln2[52 - k], make_float2(cb.z, cb.w));
  return ff_add(e, make_float2(-p.x, -p.y));
}

// 1/a for a > 0: the FP32 reciprocal refined by two Newton steps r <- r + r(1 - a r) (each
// doubles the correct bits: ~23 -> 46 -> full), or a division outside FP32's normal range.
__device__ __forceinline__ double rcp_pos(double a) {
  const long long ab = bits(a);
  if (ab > bits(1e-36) && ab < bits(1e36)) {
    double r = (double)__frcp_rn(__double2float_rn(a));
    double e = __fma_rn(-a, r, 1.0);
    r = __fma_rn(r, e, r);
    e = __fma_rn(-a, r, 1.0);
    return __fma_rn(r, e, r);
  }
  return __ddiv_rn(1.0, a);
}

// (2m+1)/2^53 for a 52-bit index m (the same value u01 builds from two words).
__device__ __forceinline__ double u01_index(unsigned long long m) {
  return __dsub_rn(__longlong_as_double((long long)(0x3FF0000000000000ull | m)), 0x1.fffffffffffffp-1);
}

// One SSA draw: Philox counter (d, iter, slot, 0) -> the 52-bit index m2 of u2 (which reaction)
// and e = -log u1 (the waiting time in units of 1/a0) as a float-float.
__device__ __forceinline__ void ssa_draw(uint32_t d, uint32_t iter, uint32_t slot, uint32_t k0,
                                         uint32_t k1, const LogTables &T, unsigned long long &m2,
                                         float2 &e) {
  uint32_t c0 = d, c1 = iter, c2 = slot, c3 = 0u;
  philox4x32_10(c0, c1, c2, c3, k0, k1);
  e = neg_log_u01(c0, c1, T);
  m2 = ((unsigned long long)c2 << 20) | (unsigned long long)(c3 >> 12);
}

// Clock after a waiting time e (float-float) at rate inverse inv_a0: t + (e_hi + e_lo) inv_a0,
// two FP64 fused operations (the float halves become doubles exactly by integer operations).
__device__ __forceinline__ double advance_clock(double t, float2 e, double inv_a0) {
  return __fma_rn(f2d_bits(e.y), inv_a0, __fma_rn(f2d_bits(e.x), inv_a0, t));
}

// ------------------------------------------------------------------------------------------
// Fixed-point clock of the table kernels.  Within an interval the clock runs in integer units
// of tau / 2^62: waiting times are added exactly (no rounding per event), the event-fires test
// t + dt <= tau is an integer compare, and no FP64 operation is left on the event-to-event
// chain.  A waiting time dt = e / a0 comes from e (float-float) times the row's float-float
// (2^62 / tau) / a0, an error-free float product plus the cross terms (relative error about
// 2^-47, below the logarithm's), rounded to the nearest unit.  The float product alone never
// decides whether an event fires: near the end of the interval it can round up to 2^62 while
// the full product is below it, so only products of 2^63 and more are set aside, and the fire
// test is made on the exact unsigned sum.
// ------------------------------------------------------------------------------------------
constexpr uint32_t kClockFarBits = (uint32_t)(127 + 63) << 23;    // float bits of 2^63

// Nearest integer to a float f with |f| < 2^63, by integer operations on its bits and without
// branches: |f| = m 2^(E-150) = (m 2^39) / 2^(189-E), one rounding right shift of m 2^39 (below
// 2^63, so adding the rounding half, at most 2^62, cannot wrap), or none for E = 189.  The shift
// is held at 63 at most; only |f| < 1/2 is affected by that limit, which then gives 1, not 0.
__device__ __forceinline__ long long f2ll_near(float f) {
  const uint32_t b = __float_as_uint(f);
  const int ex = (int)((b >> 23) & 0xffu);
  const unsigned long long mm = (unsigned long long)((b & 0x7fffffu) | 0x800000u) << 39;
  const int sh = min(max(189 - ex, 0), 63);
  const unsigned long long v = sh ? (mm + (1ull << (sh - 1))) >> sh : mm;
  const long long sv = (long long)v;
  return (b >> 31) ? -sv : sv;
}

// Waiting time in clock units for e = -log u1 and w = (2^62 / tau) / a0 (both float-float,
// non-negative).  Returns false when it is 2^63 units or more (far beyond the interval,
// including an infinite w); dt is then unspecified.  Otherwise 0 <= dt < 2^63 + 2^40.
__device__ __forceinline__ bool wait_units(float2 e, float2 w, unsigned long long &dt) {
  const float p = __fmul_rn(e.x, w.x);
  const bool near = (__float_as_uint(p) & 0x7fffffffu) < kClockFarBits;
  const float err = __fmaf_rn(e.x, w.x, -p);
  const float lo = __fmaf_rn(e.x, w.y, __fmaf_rn(e.y, w.x, err));
  dt = (unsigned long long)(f2ll_near(p) + f2ll_near(lo));
  return near;
}

// Clock units back to time: t = units * tau / 2^62 (one rounding).
__device__ __forceinline__ double clock_time(unsigned long long units, double tau) {
  return __dmul_rn(__ull2double_rn(units), ldexp(tau, -kClockBits));
}

// near_tau_fp64 on the fixed-point clock: 2^-40 tau is 2^22 units.
__device__ __forceinline__ int near_tau_units(unsigned long long clk, unsigned long long stop_u) {
  constexpr unsigned long long thr = 1ull << (kClockBits - 40);
  return (kClockTau - clk < thr) || (stop_u > kClockTau && stop_u - kClockTau < thr);
}

// Draws do not depend on the state, so they are made kDrawBatch at a time: the batch's
// independent Philox and logarithm chains interleave in one instruction stream (each chain
// alone is a few hundred cycles of dependent integer and FP32 operations), instead of one
// serial chain per event.  At most kDrawBatch - 1 draws per walker and interval go unused.
constexpr int kDrawBatch = 4;
struct DrawQueue {
  unsigned long long m[kDrawBatch];
  float2 e[kDrawBatch];
  uint32_t base;                                    // counter of draw m[0]
  int used;                                         // draws of this batch already taken

  __device__ __forceinline__ void refill(uint32_t iter, uint32_t slot, uint32_t k0, uint32_t k1,
                                         const LogTables &T) {
#pragma unroll
    for (int i = 0; i < kDrawBatch; ++i) ssa_draw(base + (uint32_t)i, iter, slot, k0, k1, T, m[i], e[i]);
    used = 0;
  }
  __device__ __forceinline__ void init(uint32_t iter, uint32_t slot, uint32_t k0, uint32_t k1,
                                       const LogTables &T) {
    base = 0;
    refill(iter, slot, k0, k1, T);
  }
  // The next draw in counter order (entry 0; the rest move down, so every index is a
  // compile-time constant and the queue stays in registers).
  __device__ __forceinline__ void pop(uint32_t iter, uint32_t slot, uint32_t k0, uint32_t k1,
                                      const LogTables &T, unsigned long long &m2, float2 &e2) {
    if (used == kDrawBatch) {
      base += kDrawBatch;
      refill(iter, slot, k0, k1, T);
    }
    m2 = m[0];
    e2 = e[0];
#pragma unroll
    for (int i = 0; i + 1 < kDrawBatch; ++i) { m[i] = m[i + 1]; e[i] = e[i + 1]; }
    ++used;
  }
};

}  // namespace we
