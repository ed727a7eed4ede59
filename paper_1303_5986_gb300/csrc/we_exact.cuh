// we_exact.cuh -- exact integer forms of the two floating-point decisions of split/merge, so
// that the warp loops of k_resample need no FP64 division (a multi-instruction subroutine on
// the FP64 unit, which GB300 has little of):
//
//   merge:  u < fl(w_p / s), s = fl(w_p + w_q)   -- the survivor draw of Sec. II.B
//   split:  fl(w / c) for a copy count c         -- the per-copy weight
//
// Both give the same bits as IEEE round-to-nearest-even double arithmetic (checked on the
// host against the C library's double division in tests/test_exact_arith.py).  Inputs are
// positive normal doubles; callers route other cases to the plain floating-point path.  The
// merge decision also has an FP32 screen that answers only where its error bound allows and
// otherwise defers to the exact test (checked the same way).
#pragma once
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define WE_HD __host__ __device__ __forceinline__
#else
#define WE_HD inline
#endif

namespace we {

WE_HD unsigned long long ex_mulhi64(unsigned long long a, unsigned long long b) {
#if defined(__CUDA_ARCH__)
  return __umul64hi(a, b);
#else
  return (unsigned long long)(((unsigned __int128)a * b) >> 64);
#endif
}

WE_HD int ex_clz64(unsigned long long v) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)v);
#else
  return v ? __builtin_clzll(v) : 64;
#endif
}

// 128-bit unsigned as (hi, lo)
struct U128 {
  unsigned long long hi, lo;
};
WE_HD bool ex_lt(U128 a, U128 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
WE_HD bool ex_eq(U128 a, U128 b) { return a.hi == b.hi && a.lo == b.lo; }

// Significand (with the implicit bit) and exponent field of a positive normal double.
WE_HD unsigned long long ex_mant(unsigned long long bits) { return (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52); }
WE_HD int ex_field(unsigned long long bits) { return (int)(bits >> 52); }

// u < fl(w / s) for positive normal doubles u (< 1), w and s.  With x = m 2^(F-1075) for each,
// in units of 2^(eu+es-1):  u s = A = 2 mu ms,  (u + ulp(u)/2) s = B = A + ms,  w = C = mw 2^t,
// t = Fw - Fu - Fs + 1076.  Then fl(w/s) > u iff w/s > u + ulp/2, or w/s = u + ulp/2 and the
// tie rounds up to the even neighbour (mu odd); fl(w/s) <= u otherwise.  (The next double above
// u is u + ulp(u), so a quotient strictly above the midpoint rounds to it or beyond.)
WE_HD bool ex_u_below_quotient(unsigned long long u_bits, unsigned long long w_bits, unsigned long long s_bits) {
  const unsigned long long mu = ex_mant(u_bits), ms = ex_mant(s_bits), mw = ex_mant(w_bits);
  const int t = ex_field(w_bits) - ex_field(u_bits) - ex_field(s_bits) + 1076;
  if (t < 0) return false;                                 // w < u s: quotient below u
  if (t > 75) return true;                                 // w > 2^127 units > B
  const unsigned long long plo = mu * ms, phi = ex_mulhi64(mu, ms);
  U128 A{(phi << 1) | (plo >> 63), plo << 1};
  U128 B{A.hi + ((A.lo + ms) < A.lo ? 1ull : 0ull), A.lo + ms};
  U128 C;
  if (t == 0) C = U128{0ull, mw};
  else if (t < 64) C = U128{mw >> (64 - t), mw << t};
  else C = U128{mw << (t - 64), 0ull};
  if (ex_lt(C, A)) return false;
  if (ex_lt(B, C)) return true;
  return ex_eq(C, B) && (mu & 1ull);   // exact midpoint (needs a 54-bit w; kept for completeness)
}

// A float with the given exponent field whose significand is the first 23 fraction bits of the
// double `dbits` (truncated: relative error below 2^-23).
WE_HD float ex_f32_of(int f32_field, unsigned long long dbits) {
  const unsigned int fb = ((unsigned int)f32_field << 23) | (unsigned int)((dbits >> 29) & 0x7FFFFFull);
#if defined(__CUDA_ARCH__)
  return __uint_as_float(fb);
#else
  float f;
  std::memcpy(&f, &fb, 4);
  return f;
#endif
}

WE_HD float ex_fmul(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}

// The same decision u < fl(w / s) screened in FP32 (u < 1, w <= s, all positive doubles):
// 1 or 0 where FP32 settles it, -1 where it does not (u below 2^-60, w subnormal, or u within
// about 2^-19 of the quotient; the caller then takes the exact test).  Both sides are divided
// by 2^(Fs-1023): with d = Fw - Fs, W = w 2^-(Fs-1023) and S = s 2^-(Fs-1023) in [1, 2) as
// truncated floats, U the truncated float of u, and P = fl(U S), each within 5 2^-24 of its
// real value relatively.  P < fl(W (1 - 2^-19)) then gives u < q (1 - 26 2^-24) < fl(q), and
// P > fl(W (1 + 2^-19)) gives u > q (1 + 27 2^-24) > fl(q) (q = w / s).  For d < -100 the
// quotient is below 2^-99 and u (>= 2^-60) is not below it.
WE_HD int ex_u_below_quotient_f32(unsigned long long u_bits, unsigned long long w_bits,
                                  unsigned long long s_bits) {
  const int fu = ex_field(u_bits), fw = ex_field(w_bits), d = fw - ex_field(s_bits);
  if (fu < 1023 - 60 || fw == 0 || d > 0) return -1;
  if (d < -100) return 0;
  const float U = ex_f32_of(fu - 1023 + 127, u_bits), S = ex_f32_of(127, s_bits),
              W = ex_f32_of(127 + d, w_bits);
  const float P = ex_fmul(U, S);
  if (P < ex_fmul(W, 1.0f - 0x1p-19f)) return 1;
  if (P > ex_fmul(W, 1.0f + 0x1p-19f)) return 0;
  return -1;
}

// floor((2^64 - 1) / c) for 2 <= c: the reciprocal used by ex_div_small (host side).
inline unsigned long long ex_div_magic(unsigned int c) { return ~0ull / (unsigned long long)c; }

// fl(w / c) for a positive normal double w and 2 <= c <= 2048 whose quotient is normal
// (w >= 2^-1000 suffices).  magic = ex_div_magic(c).  N = m 2^11 is in [2^63, 2^64); q =
// floor(N / c) from the reciprocal (at most two corrections), then rounding to 53 bits with the
// discarded bits of q and the remainder as the exact fraction.
WE_HD unsigned long long ex_div_small(unsigned long long w_bits, unsigned int c, unsigned long long magic) {
  const unsigned long long N = ex_mant(w_bits) << 11;
  unsigned long long q = ex_mulhi64(N, magic);
  unsigned long long r = N - q * c;
  if (r >= c) { ++q; r -= c; }
  if (r >= c) { ++q; r -= c; }
  const int nb = 64 - ex_clz64(q);                         // 53 .. 63 for c <= 2048
  const int sh = nb - 53;
  unsigned long long mant = q >> sh;
  const unsigned long long low = sh ? (q & ((1ull << sh) - 1ull)) : 0ull;
  const unsigned long long num2 = 2ull * (low * c + r);    // 2 * (fraction * c * 2^sh)
  const unsigned long long half = (unsigned long long)c << sh;
  if (num2 > half || (num2 == half && (mant & 1ull))) ++mant;
  int field = ex_field(w_bits) + sh - 11;
  if (mant == (1ull << 53)) { mant >>= 1; ++field; }
  return ((unsigned long long)field << 52) | (mant & 0xFFFFFFFFFFFFFull);
}

}  // namespace we
