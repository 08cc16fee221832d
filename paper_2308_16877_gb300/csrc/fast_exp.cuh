// Double-precision exponential in 10 FP64 operations, by P. T. P. Tang's
// table-driven method ("Table-driven implementation of the exponential
// function in IEEE floating-point arithmetic", ACM TOMS 15(2), 1989):
//   x = (64 m + j) ln2/64 + r,  |r| <= ln2/128,
//   exp(x) = 2^m 2^(j/64) e^r,
// with e^r - 1 by its Taylor polynomial to r^5 (the r^6 term is below 4e-17
// relative), 2^(j/64) from a 64-entry table of doubles and 2^m added to the
// exponent field on the integer pipes. k = 64 m + j comes out of the low word
// of x 64/ln2 + 1.5 2^52, which the addition has rounded to an integer, so no
// float-to-integer conversion runs on the FP64 pipe. The reduction is
// Cody-Waite's: ln2/64 = l1 + l2 with l1 short enough that k l1 is exact.
// Valid for |x| <= 700, where the result is normal; callers take another path
// outside that range (and for NaN). Error: about one ulp (the table entry's
// rounding, the polynomial's and the final multiply-add's).
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

namespace hpac {

struct ExpTang {
  double t[64];   // 2^(j/64), j = 0..63
  double inv_l;   // 64 / ln 2
  double l1, l2;  // ln2 / 64 = l1 + l2; l1 keeps 32 significant bits
};

// The constants, from long-double arithmetic on the host, each rounded once.
inline ExpTang exp_tang_constants() {
  ExpTang c;
  for (int j = 0; j < 64; ++j) c.t[j] = (double)exp2l((long double)j / 64.0L);
  const long double L = logl(2.0L) / 64.0L;
  const double ld = (double)L;
  uint64_t b;
  memcpy(&b, &ld, sizeof b);
  b &= ~((1ull << 21) - 1);  // 53 - 21 = 32 significant bits: |k| l1 < 2^49 is exact
  memcpy(&c.l1, &b, sizeof b);
  c.l2 = (double)(L - (long double)c.l1);
  c.inv_l = (double)(64.0L / logl(2.0L));
  return c;
}

// |x| <= 700 (and not NaN) as an integer test on the bits.
__device__ __forceinline__ bool exp_tang_in_range(double x) {
  const unsigned long long ax = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  return ax <= 0x4085e00000000000ull;  // 700.0
}

// exp(x) for |x| <= 700; tab: the 64 table entries (shared memory).
__device__ __forceinline__ double exp_tang(double x, const double *tab, double inv_l, double l1,
                                           double l2) {
  const double shift = 6755399441055744.0;  // 1.5 * 2^52
  const double t = fma(x, inv_l, shift);
  const double kd = t - shift;
  const int k = __double2loint(t);
  double r = fma(-kd, l1, x);
  r = fma(-kd, l2, r);
  double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  q = fma(r, q, 1.0 / 6.0);
  q = fma(r, q, 0.5);
  const double p = fma(r * r, q, r);
  const double tj = tab[k & 63];
  const double y = fma(tj, p, tj);
  const unsigned long long m = (unsigned long long)(long long)(k >> 6);
  return __longlong_as_double((long long)((unsigned long long)__double_as_longlong(y) + (m << 52)));
}

}  // namespace hpac
