// FP64 device building blocks shared by the 2D and 3D volume kernels, written to
// spend few FP64 issue slots (GB300 issues ~2 FP64 FMAs per clock per SM).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace perk {

// Reciprocal: two Newton-Raphson steps y <- y + y (1 - x y) from the hardware's
// approximate reciprocal (PTX rcp.approx.ftz.f64); the relative error is
// squared by each step, which brings the seed to full double precision
// (within ~1 ulp, not correctly rounded).  Positive normal x only.
__device__ __forceinline__ double rcp_nr(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

// Natural logarithm, table-driven (P. T. P. Tang, "Table-driven implementation
// of the logarithm function in IEEE floating-point arithmetic", ACM TOMS 16,
// 1990): x = 2^k m, m in [1, 2); with c_j the midpoint of the j-th of 128
// mantissa intervals, ln x = k ln 2 + ln(1/inv_c[j]) + ln(1 + r),
// r = m inv_c[j] - 1 (|r| < 2^-8), ln(1 + r) by its Taylor series to r^8.
// The table (inv_c[j] = fl(1/c_j), ln_c[j] = -ln(inv_c[j]) rounded from
// extended precision) is built on the host.  Positive normal x; any other
// input (zero, negative, infinite, NaN) returns NaN.
constexpr int LOG_TABLE = 128;
constexpr double LN2_HI = 0.6931471805599453;
constexpr double LN2_LO = 2.3190468138462996e-17;

__device__ __forceinline__ double log_tab(double x, const double* __restrict__ inv_c,
                                          const double* __restrict__ ln_c) {
  const long long bits = __double_as_longlong(x);
  const int hi = (int)(bits >> 32);
  const int j = (hi >> 13) & (LOG_TABLE - 1);
  const long long eb = (bits >> 52) & 0x7FF;
  const double m = __longlong_as_double((bits & 0x000FFFFFFFFFFFFFLL) | 0x3FF0000000000000LL);
  // k as a double without an int->double conversion: 2^52 + eb, minus 2^52 + 1023
  const double kd = __longlong_as_double(0x4330000000000000LL | eb) - (4503599627370496.0 + 1023.0);
  const double r = fma(m, inv_c[j], -1.0);
  double q = -1.0 / 8.0;
  q = fma(q, r, 1.0 / 7.0);
  q = fma(q, r, -1.0 / 6.0);
  q = fma(q, r, 1.0 / 5.0);
  q = fma(q, r, -1.0 / 4.0);
  q = fma(q, r, 1.0 / 3.0);
  q = fma(q, r, -0.5);
  const double l1p = fma(r * r, q, r);
  const double v = fma(kd, LN2_HI, ln_c[j] + fma(kd, LN2_LO, l1p));
  // positive finite x has a bit pattern in (0, +inf): an integer test, off the FP64 pipe
  return (bits > 0 && bits < 0x7FF0000000000000LL) ? v : __longlong_as_double(0x7FF8000000000000LL);
}

// Whether the logarithmic means of a pair take their series: for positive normal a, b whose
// bit patterns differ by less than NEAR_BITS = 0.06 * 2^52.  The bit pattern grows by at least
// 2^52 (b/a - 1) from a to b (it is a concave, piecewise-linear function of x that matches
// 2^52 log2 x at powers of two), so the test implies b/a < 1.06, |f| = |b - a|/(a + b) < 0.0292;
// it fails only for |f| > 0.015, where the difference of the node logarithms is well conditioned.
// Integer arithmetic keeps the decision off the FP64 pipe.
constexpr long long NEAR_BITS = 270215977642229LL;   // floor(0.06 * 2^52)
__device__ __forceinline__ bool near_pair(double a, double b) {
  const long long d = __double_as_longlong(b) - __double_as_longlong(a);
  return (d < 0 ? -d : d) < NEAR_BITS;
}

// Series of the logarithmic mean in u = f^2, f = (b - a)/(b + a), used where near_pair holds:
//   ln(b/a) = 2 f A(u),  A(u) = sum_k u^k / (2k+1);   {{x}}_ln = (a + b) / (2 A(u)) = (a + b) H(u)
// with H = 1/(2A) expanded term by term (exact rationals), both to u^4: for |f| < 0.0292 the
// truncation is below 1e-17 (H) and 5e-17 (2A) relative.
__device__ __forceinline__ double series_H(double u) {
  double r = -214.0 / 14175.0;
  r = fma(r, u, -22.0 / 945.0);
  r = fma(r, u, -2.0 / 45.0);
  r = fma(r, u, -1.0 / 6.0);
  return fma(r, u, 0.5);
}
__device__ __forceinline__ double series_2A(double u) {
  double r = 2.0 / 9.0;
  r = fma(r, u, 2.0 / 7.0);
  r = fma(r, u, 2.0 / 5.0);
  r = fma(r, u, 2.0 / 3.0);
  return fma(r, u, 2.0);
}

// Positive doubles order like their bit patterns: element-wide extremes by integer min/max.
__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ double bitsd(unsigned long long b) { return __longlong_as_double((long long)b); }

// Whether every node pair of an element takes the series branch of both logarithmic means
// (near_pair for rho and for rho/p), judged from the element's extremes of the two variables'
// bit patterns: when they lie within NEAR_BITS, so does every pair, no node logarithm is read
// and the element's logarithms need not be computed.  A zero, negative, infinite or NaN value
// anywhere makes the test fail, and the logarithms are then computed as usual.
__device__ __forceinline__ bool series_only(unsigned long long rmin, unsigned long long rmax, unsigned long long bmin,
                                            unsigned long long bmax) {
  constexpr unsigned long long INF = 0x7FF0000000000000ull;
  return rmin > 0 && rmax < INF && bmin > 0 && bmax < INF && rmax - rmin < (unsigned long long)NEAR_BITS &&
         bmax - bmin < (unsigned long long)NEAR_BITS;
}

}  // namespace perk
