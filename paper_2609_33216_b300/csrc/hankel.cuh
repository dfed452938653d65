// Hankel functions H_0^(1)(x) and H_1^(1)(x) = J_n(x) + i Y_n(x) for real x > 0,
// evaluated together in FP64 to about 1e-15 relative accuracy.
//
// Three regions, each a published method written out here:
//   x <= 4        power series (DLMF 10.2.2, 10.8.1):
//                 J0 = sum (-1)^k t^k / (k!)^2,  J1 = (x/2) sum (-1)^k t^k / (k!(k+1)!),  t = x^2/4
//                 Y0 = (2/pi) [(ln(x/2) + gamma) J0 + sum (-1)^(k+1) H_k t^k / (k!)^2]
//                 Y1 = (2/pi)(ln(x/2) + gamma) J1 - 2/(pi x) - (x/(2 pi)) sum (-1)^k (H_k + H_(k+1)) t^k / (k!(k+1)!)
//                 (H_k the harmonic numbers), 16 terms;
//   4 < x < 20    Taylor expansions of J0, Y0, J1, Y1 of degree 15 about the centres
//                 4.5 + m of the sixteen unit intervals (kHankelMid, hankel_table.inc,
//                 written by gen_hankel_table.py from mpmath): 64 fused multiply-adds,
//                 about 2e-16 relative;
//   x >= 20       Hankel's asymptotic expansion (DLMF 10.17.5)
//                 H_n(x) = sqrt(2/(pi x)) e^{i(x - n pi/2 - pi/4)} sum_k i^k a_k(n) / x^k,
//                 a_k(n) = prod_{j<=k} (4n^2 - (2j-1)^2) / (8j), 28 terms; one sincos(x)
//                 serves both orders.
// The coefficient tables are generated at compile time from these formulas.
#pragma once

#include <cuda_runtime.h>

namespace symhss {
namespace hk {

#include "hankel_table.inc"


constexpr double factd(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= (double)i;
  return f;
}
constexpr double harm(int k) {
  double s = 0.0;
  for (int i = 1; i <= k; ++i) s += 1.0 / (double)i;
  return s;
}
constexpr double sgn(int k) { return (k & 1) ? -1.0 : 1.0; }
constexpr double cj0(int k) { return sgn(k) / (factd(k) * factd(k)); }
constexpr double cj1(int k) { return sgn(k) / (factd(k) * factd(k + 1)); }
constexpr double cy0(int k) { return -sgn(k) * harm(k) / (factd(k) * factd(k)); }
constexpr double cy1(int k) { return sgn(k) * (harm(k) + harm(k + 1)) / (factd(k) * factd(k + 1)); }
constexpr double ak(int n, int k) {
  double a = 1.0;
  for (int j = 1; j <= k; ++j) a *= (4.0 * n * n - (2.0 * j - 1.0) * (2.0 * j - 1.0)) / (8.0 * j);
  return a;
}
constexpr double pk(int n, int m) { return sgn(m) * ak(n, 2 * m); }
constexpr double qk(int n, int m) { return sgn(m) * ak(n, 2 * m + 1); }

#define SYMHSS_T16(f) \
  { f(0), f(1), f(2), f(3), f(4), f(5), f(6), f(7), f(8), f(9), f(10), f(11), f(12), f(13), f(14), f(15) }
#define SYMHSS_T14(f) \
  { f(0), f(1), f(2), f(3), f(4), f(5), f(6), f(7), f(8), f(9), f(10), f(11), f(12), f(13) }
#define SYMHSS_P0(m) pk(0, m)
#define SYMHSS_Q0(m) qk(0, m)
#define SYMHSS_P1(m) pk(1, m)
#define SYMHSS_Q1(m) qk(1, m)

constexpr int kSeries = 16;
constexpr int kAsym = 14;
constexpr double kSeriesMax = 4.0;
constexpr double kAsymMin = 20.0;
constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kGamma = 0.577215664901532860606512090082402431;

static __constant__ double cJ0[kSeries] = SYMHSS_T16(cj0);
static __constant__ double cJ1[kSeries] = SYMHSS_T16(cj1);
static __constant__ double cY0[kSeries] = SYMHSS_T16(cy0);
static __constant__ double cY1[kSeries] = SYMHSS_T16(cy1);
static __constant__ double cP0[kAsym] = SYMHSS_T14(SYMHSS_P0);
static __constant__ double cQ0[kAsym] = SYMHSS_T14(SYMHSS_Q0);
static __constant__ double cP1[kAsym] = SYMHSS_T14(SYMHSS_P1);
static __constant__ double cQ1[kAsym] = SYMHSS_T14(SYMHSS_Q1);

template <int K>
__device__ __forceinline__ double horner(const double* c, double t) {
  double s = c[K - 1];
#pragma unroll
  for (int k = K - 2; k >= 0; --k) s = fma(s, t, c[k]);
  return s;
}

}  // namespace hk

// h0 = H_0^(1)(x), h1 = H_1^(1)(x) for x > 0 (x = re, y = im), given
// lh = log(x / 2) and ix = 1 / x (callers evaluating several x from one distance
// share the logarithm and the reciprocal).
__device__ __forceinline__ void hankel01(double x, double lh, double ix, double2& h0, double2& h1) {
  using namespace hk;
  if (x <= kSeriesMax) {
    const double t = 0.25 * x * x;
    const double j0v = horner<kSeries>(cJ0, t);
    const double j1v = 0.5 * x * horner<kSeries>(cJ1, t);
    const double L = lh + kGamma;
    const double y0v = (2.0 / kPi) * fma(L, j0v, horner<kSeries>(cY0, t));
    const double y1v = (2.0 / kPi) * (L * j1v - ix) - (x * (0.5 / kPi)) * horner<kSeries>(cY1, t);
    h0 = make_double2(j0v, y0v);
    h1 = make_double2(j1v, y1v);
    return;
  }
  if (x >= kAsymMin) {
    const double ix2 = ix * ix;
    const double p0 = horner<kAsym>(cP0, ix2), q0 = ix * horner<kAsym>(cQ0, ix2);
    const double p1 = horner<kAsym>(cP1, ix2), q1 = ix * horner<kAsym>(cQ1, ix2);
    double s, c;
    sincos(x, &s, &c);
    const double amp = sqrt(ix * (1.0 / kPi));
    // e^{i(x - pi/4)} sqrt2 = (c + s) + i (s - c);  e^{i(x - 3pi/4)} sqrt2 = (s - c) - i (s + c)
    const double e0r = c + s, e0i = s - c;
    const double e1r = s - c, e1i = -(s + c);
    h0 = make_double2(amp * (e0r * p0 - e0i * q0), amp * (e0r * q0 + e0i * p0));
    h1 = make_double2(amp * (e1r * p1 - e1i * q1), amp * (e1r * q1 + e1i * p1));
    return;
  }
  // 4 < x < 20: Horner in t = x - (4.5 + m) with the interval's Taylor coefficients
  int m = (int)x - 4;
  m = m < 0 ? 0 : (m > 15 ? 15 : m);
  const double t = x - (4.5 + (double)m);
  const double* c = &kHankelMid[m][0][0];
  double j0v = __ldg(c + 15), y0v = __ldg(c + 31), j1v = __ldg(c + 47), y1v = __ldg(c + 63);
#pragma unroll
  for (int n = 14; n >= 0; --n) {
    j0v = fma(j0v, t, __ldg(c + n));
    y0v = fma(y0v, t, __ldg(c + 16 + n));
    j1v = fma(j1v, t, __ldg(c + 32 + n));
    y1v = fma(y1v, t, __ldg(c + 48 + n));
  }
  h0 = make_double2(j0v, y0v);
  h1 = make_double2(j1v, y1v);
}

__device__ __forceinline__ void hankel01(double x, double2& h0, double2& h1) {
  hankel01(x, log(0.5 * x), 1.0 / x, h0, h1);
}

}  // namespace symhss
