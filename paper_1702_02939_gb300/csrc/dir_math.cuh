// Table-driven FP64 sine/cosine and logarithm for the director terms of Eq. 3.
//
// The director step needs, per cell and step, n(theta) = (cos theta, sin theta)
// and one standard normal by the Box-Muller transform, sqrt(-2 ln u1) cos(2 pi u2).
// On this GPU FP64 runs at 1/74 of the FP32 rate and these three functions
// are most of the director kernel's FP64 work, so they are evaluated with the
// table-driven method of P. T. P. Tang (ACM TOMS 15(2), 1989, for the
// trigonometric functions; ACM TOMS 16(4), 1990, for the logarithm): the
// argument is reduced to a small remainder around one of 256 table points and
// short Taylor polynomials of the remainder are combined with the tabulated
// values.  Every coefficient is a Taylor coefficient (1/k!, 1/k); the split of
// pi/128 and the other constants are derived from pi and ln 2.
//
// Accuracy (checked against CUDA's sincos/log/cospi in the tests):
//   dm_sincos  absolute error <= 4 * 2^-53 for |theta| < 2^20 (CUDA's sincos
//              beyond, and for non-finite theta);
//   dm_cospi   absolute error <= 4 * 2^-53 on [0, 2];
//   dm_log     relative error <= 4 * 2^-53 on (0, 1] (normal numbers).
#pragma once
#include <cuda_runtime.h>

namespace cgk {

// Table layout: 256 entries (sin(j pi/128), cos(j pi/128)), then 256 entries
// (1/c_j, -ln(1/c_j)) for the logarithm's reduction intervals.
constexpr int kDirTabEntries = 512;

// The logarithm reduces u = 2^k m with m in [M0, 2 M0), M0 = 0.708 (bit
// pattern kLogOff), so that ln m never cancels against k ln 2; the octave is
// cut into 256 intervals of equal width in the bit pattern (2^44 units), and
// interval 149 is centred on 1.0 (its reciprocal is exactly 1, so ln u for u
// near 1 is the polynomial alone).
constexpr long long kLogOff = 0x3FE6A80000000000LL;
constexpr int kLogOne = 149;

// Exact v * 2^k as a double for |v| < 2^53 (and a result in the normal
// range), built on the integer pipes alone: sign, leading-zero count, the
// leading one shifted to bit 52, the exponent field added on top (the leading
// one carries into it).  No FP64 instruction: in the geometry kernels the FP64
// pipe is the bottleneck while the integer pipes are mostly idle.
__device__ __forceinline__ double i2d_int(long long v, int k = 0) {
  const unsigned long long sgn = (unsigned long long)v & 0x8000000000000000ull;
  const unsigned long long a = (v < 0) ? (0ull - (unsigned long long)v) : (unsigned long long)v;
  const int lz = __clzll((long long)a);  // 11 <= lz for |v| < 2^53; 64 for v = 0
  const unsigned long long m = a << (lz - 11);
  const unsigned long long e = (unsigned long long)(1022 + 63 - lz + k) << 52;
  return a ? __longlong_as_double((long long)(sgn | (e + m))) : 0.0;
}

__device__ __forceinline__ double dm_i2d(long long v) { return i2d_int(v); }  // exact for |v| < 2^53

// sin(r) - r and cos(r) - 1 for |r| <= 0.0125 (Taylor to r^7 and r^6; the
// first omitted terms are below 2^-70).
__device__ __forceinline__ void dm_small(double r, double& s_minus_r, double& c_minus_1) {
  const double r2 = r * r;
  const double ps = fma(r2, fma(r2, -1.0 / 5040.0, 1.0 / 120.0), -1.0 / 6.0);
  s_minus_r = (r * r2) * ps;
  const double pc = fma(r2, fma(r2, -1.0 / 720.0, 1.0 / 24.0), -0.5);
  c_minus_1 = r2 * pc;
}

// (sin theta, cos theta).  theta = j pi/128 + r with j = rint(128 theta / pi)
// and r by a three-term Cody-Waite reduction (the first two parts of pi/128
// carry 27 significant bits, so j * part is exact for |j| < 2^26).
__device__ __forceinline__ void dm_sincos(double th, const double2* __restrict__ tab, double& s, double& c) {
  if (!((__double_as_longlong(th) & 0x7FFFFFFFFFFFFFFFLL) < 0x4130000000000000LL)) {  // |theta| >= 2^20 or NaN
    sincos(th, &s, &c);
    return;
  }
  const double kMagic = 0x1.8p52;
  const double jm = fma(th, 0x1.45f306dc9c883p+5, kMagic);  // 128/pi
  const double jd = jm - kMagic;
  const int j = __double2loint(jm) & 255;
  double r = fma(-jd, 0x1.921fb54000000p-6, th);  // pi/128, part 1
  r = fma(-jd, 0x1.10b4610000000p-36, r);          // part 2
  r = fma(-jd, 0x1.a62633145c06ep-64, r);          // part 3
  double sr, cm;
  dm_small(r, sr, cm);
  sr += r;
  const double2 t = __ldg(&tab[j]);  // (S, C) = (sin, cos)(j pi/128)
  // sin(a + r) = S + (S (cos r - 1) + C sin r), cos(a + r) = C + (C (cos r - 1) - S sin r)
  s = t.x + fma(t.y, sr, t.x * cm);
  c = t.y + fma(-t.x, sr, t.y * cm);
}

// cos(pi t) for t in [0, 2]: t = j/128 + r exactly (t is a multiple of
// 2^-52), then the angle pi r.
__device__ __forceinline__ double dm_cospi(double t, const double2* __restrict__ tab) {
  const double kMagic = 0x1.8p52;
  const double jm = fma(t, 128.0, kMagic);
  const double jd = jm - kMagic;
  const int j = __double2loint(jm) & 255;
  const double rr = fma(-jd, 0x1p-7, t);   // exact
  const double r = rr * 0x1.921fb54442d18p+1;  // pi
  double sr, cm;
  dm_small(r, sr, cm);
  sr += r;
  const double2 tt = __ldg(&tab[j]);
  return tt.y + fma(-tt.x, sr, tt.y * cm);
}

// cos(pi t) for t = v 2^-52, v in [1, 2^53] (t in (0, 2]) given as the
// integer v: the reduction t = j/128 + r is done on the integer pipes
// (j = v / 2^45 rounded to nearest, ties to even, as the FP64 reduction of
// dm_cospi rounds; r = (v - j 2^45) 2^-52 exactly), then as dm_cospi.
__device__ __forceinline__ double dm_cospi_grid52(unsigned long long v, const double2* __restrict__ tab) {
  const unsigned long long half = 1ull << 44;
  const unsigned long long q = v >> 45, rem = v & ((1ull << 45) - 1);
  const unsigned long long jr = q + ((rem > half || (rem == half && (q & 1))) ? 1ull : 0ull);
  const int j = (int)(jr & 255);
  const double rr = i2d_int((long long)v - (long long)(jr << 45), -52);  // exact, |rr| <= 2^-8
  const double r = rr * 0x1.921fb54442d18p+1;                            // pi
  double sr, cm;
  dm_small(r, sr, cm);
  sr += r;
  const double2 tt = __ldg(&tab[j]);
  return tt.y + fma(-tt.x, sr, tt.y * cm);
}

// ln u for a positive normal u: u = 2^k m, m in [M0, 2 M0).  With c_j the
// centre of m's interval, ln m = -ln(1/c_j) + ln(1 + r) where r = m (1/c_j) - 1
// is formed in one rounding (|r| <= 2^-9); ln(1 + r) by Taylor to r^7.
__device__ __forceinline__ double dm_log(double u, const double2* __restrict__ tab) {
  const long long b = __double_as_longlong(u);
  const long long d = b - kLogOff;
  const long long k = d >> 52;  // floor
  const int j = (int)((d >> 44) & 255);
  const double m = __longlong_as_double(b - (k << 52));
  const double2 t = __ldg(&tab[256 + j]);  // (1/c_j, -ln(1/c_j))
  const double r = fma(m, t.x, -1.0);
  double q = fma(r, 1.0 / 7.0, -1.0 / 6.0);
  q = fma(r, q, 1.0 / 5.0);
  q = fma(r, q, -0.25);
  q = fma(r, q, 1.0 / 3.0);
  q = fma(r, q, -0.5);
  const double l1p = fma(r * r, q, r);
  return fma(dm_i2d(k), 0x1.62e42fefa39efp-1, t.y + l1p);  // + k ln 2
}

}  // namespace cgk
