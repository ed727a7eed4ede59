// Host check of the exact integer split/merge decisions (paper_1303_5986_gb300/csrc/we_exact.cuh)
// against IEEE double arithmetic of the host (round to nearest even, no contraction).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <random>
#include "../paper_1303_5986_gb300/csrc/we_exact.cuh"

static unsigned long long B(double x) { unsigned long long b; std::memcpy(&b, &x, 8); return b; }
static double D(unsigned long long b) { double x; std::memcpy(&x, &b, 8); return x; }

int main() {
  std::mt19937_64 g(12345);
  long fails = 0, n_div = 0, n_cmp = 0, n_tie = 0;
  // fl(w / c): random normal w over the exponent range the kernel admits, every c in 2..2048
  for (unsigned c = 2; c <= 2048; ++c) {
    const unsigned long long mg = we::ex_div_magic(c);
    for (int k = 0; k < 2000; ++k) {
      const int field = 24 + (int)(g() % 2000);            // w from 2^-999 up
      const unsigned long long wb = ((unsigned long long)field << 52) | (g() & 0xFFFFFFFFFFFFFull);
      const double w = D(wb);
      const volatile double cd = (double)c;
      const unsigned long long want = B(w / cd);
      const unsigned long long got = we::ex_div_small(wb, c, mg);
      ++n_div;
      if (want != got) { if (fails++ < 10) std::printf("div w=%a c=%u want %a got %a\n", w, c, D(want), D(got)); }
    }
    // mantissas all ones and exact multiples
    for (int k = 0; k < 64; ++k) {
      const unsigned long long wb = ((unsigned long long)(1000 + k) << 52) | (k & 1 ? 0xFFFFFFFFFFFFFull : 0ull);
      const volatile double cd = (double)c;
      if (B(D(wb) / cd) != we::ex_div_small(wb, c, mg)) { if (fails++ < 10) std::printf("div edge c=%u\n", c); }
      ++n_div;
    }
  }
  // u < fl(w / s), s = fl(w + q): random weights over a wide range and random uniforms
  for (long k = 0; k < 4000000; ++k) {
    const int fw = 24 + (int)(g() % 1900), dq = (int)(g() % 120) - 60;
    const unsigned long long wb = ((unsigned long long)fw << 52) | (g() & 0xFFFFFFFFFFFFFull);
    const int fq = fw + dq < 24 ? 24 : fw + dq;
    const unsigned long long qb = ((unsigned long long)fq << 52) | (g() & 0xFFFFFFFFFFFFFull);
    const double w = D(wb), q = D(qb);
    const volatile double s = w + q;
    const volatile double prob = w / s;
    double u;
    switch (k % 4) {
      case 0: u = (double)(2 * (g() >> 12) + 1) * 0x1p-53; break;   // the generator's uniforms
      case 1: u = prob; break;                                      // u equal to the quotient
      case 2: u = std::nextafter((double)prob, 0.0); break;         // just below
      default: u = std::nextafter((double)prob, 1.0); break;        // just above
    }
    if (!(u > 0.0 && u < 1.0)) continue;
    const bool want = u < prob;
    const bool got = we::ex_u_below_quotient(B(u), wb, B((double)s));
    ++n_cmp;
    if (want != got) { if (fails++ < 10) std::printf("cmp u=%a w=%a s=%a want %d got %d\n", u, w, (double)s, want, got); }
  }
  // The FP32 screen: where it answers, the answer is the double comparison's; it leaves few
  // of the generator's uniforms undecided.  Weights over the whole normal range (and subnormal
  // ones), w <= s, uniforms of the generator and at, just below and just above the quotient.
  long n_f32 = 0, n_f32_open = 0, n_f32_gen = 0, n_f32_gen_open = 0;
  for (long k = 0; k < 4000000; ++k) {
    const int fw = (int)(g() % 2047), dq = (int)(g() % 240) - 120;
    const unsigned long long wb = ((unsigned long long)fw << 52) | (g() & 0xFFFFFFFFFFFFFull);
    const int fq0 = fw + dq, fq = fq0 < 0 ? 0 : (fq0 > 2000 ? 2000 : fq0);
    const unsigned long long qb = ((unsigned long long)fq << 52) | (g() & 0xFFFFFFFFFFFFFull);
    const double w = D(wb), q = D(qb);
    const volatile double s = w + q;
    if (!(s < INFINITY) || !(s > 0.0) || !(w > 0.0)) continue;
    const volatile double prob = w / s;
    double u;
    switch (k % 5) {
      case 0: u = (double)(2 * (g() >> 12) + 1) * 0x1p-53; break;
      case 1: u = prob; break;
      case 2: u = std::nextafter((double)prob, 0.0); break;
      case 3: u = std::nextafter((double)prob, 1.0); break;
      default: u = (double)prob * (1.0 + std::ldexp((double)(g() % 64) - 32.0, -24)); break;
    }
    if (!(u > 0.0 && u < 1.0)) continue;
    const int got = we::ex_u_below_quotient_f32(B(u), wb, B((double)s));
    ++n_f32;
    if (k % 5 == 0) ++n_f32_gen;
    if (got < 0) { ++n_f32_open; if (k % 5 == 0) ++n_f32_gen_open; continue; }
    const bool want = u < prob;
    if (want != (got == 1)) { if (fails++ < 10) std::printf("f32 u=%a w=%a s=%a want %d got %d\n", u, w, (double)s, want, got); }
  }
  if (n_f32_gen_open * 1000 > n_f32_gen) { ++fails; std::printf("f32 screen leaves %ld of %ld uniforms open\n", n_f32_gen_open, n_f32_gen); }
  // quotients exactly equal to u (s a power of two, w = u s exact).  An exact midpoint
  // w/s = u + ulp(u)/2 cannot occur: it needs the 54-bit odd significand 2 mu + 1 in w.
  for (long k = 0; k < 200000; ++k) {
    const unsigned long long mu = g() & 0xFFFFFFFFFFFFFull;
    const int fu = 1000 + (int)(g() % 22);
    const double u = D(((unsigned long long)fu << 52) | mu);
    const double s = std::ldexp(1.0, (int)(g() % 40) - 20);
    const double w = u * s;
    const bool want = u < w / s;                            // false: the quotient is u
    const bool got = we::ex_u_below_quotient(B(u), B(w), B(s));
    ++n_tie;
    if (want != got) { if (fails++ < 10) std::printf("eq u=%a w=%a s=%a\n", u, w, s); }
  }
  std::printf("%s div=%ld cmp=%ld eq=%ld f32=%ld (open %ld; uniforms %ld open %ld) fails=%ld\n", fails ? "FAIL" : "ok",
              n_div, n_cmp, n_tie, n_f32, n_f32_open, n_f32_gen, n_f32_gen_open, fails);
  return fails ? 1 : 0;
}
