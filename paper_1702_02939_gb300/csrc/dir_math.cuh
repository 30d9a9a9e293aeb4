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
// The argument reductions run in FP64 (or, for the Box-Muller cosine, on the
// integer pipes); the polynomials and the combination with the table run in
// 64-bit fixed point (Q1.62: value x 2^62 in a signed 64-bit integer; products
// by the 128-bit integer multiply), rounded to double once at the end.  The
// integer pipes are mostly idle in the FP64-bound step kernels, and a
// fixed-point polynomial carries ~2^-60 absolute error against ~2^-53 per
// FP64 operation.
//
// Accuracy (the tests allow 4 units of 2^-53 against numpy and the oracle;
// an exact-arithmetic check of the same formulas found at most 1 unit for
// sin/cos, absolute, and 2 units for ln(1 + r), relative):
//   dm_sincos        for |theta| < 2^20 (CUDA's sincos beyond, and for
//                    non-finite theta);
//   dm_cospi_grid52  on (0, 2];
//   dm_log           on (0, 1] (normal numbers).
#pragma once
#include <cuda_runtime.h>

namespace cgk {

// Table layout: 256 entries (sin(j pi/128), cos(j pi/128)), then 256 entries
// (1/c_j, -ln(1/c_j)) for the logarithm's reduction intervals, then the 256
// (sin, cos)(j pi/128) again as Q1.62 integers (the doubles times 2^62, exact).
constexpr int kDirTabEntries = 768;
constexpr int kDirTabQ = 512;

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

// ---- 64-bit fixed point, Q1.62 ----
constexpr long long kQOne = 1LL << 62;
// round(2^62 / d)
__host__ __device__ constexpr long long qdiv(long long d) { return (kQOne + d / 2) / d; }
// a b in Q1.62 (|a b| < 2), the product truncated toward minus infinity
__device__ __forceinline__ long long mulq(long long a, long long b) {
  return (long long)(((__int128)a * (__int128)b) >> 62);
}
// x 2^62 for |x| < 2, truncated toward zero, on the integer pipes
__device__ __forceinline__ long long d2q(double x) {
  const long long b = __double_as_longlong(x);
  const int ef = (int)((b >> 52) & 0x7ff);
  if (ef == 0) return 0;  // zero (or subnormal, below 2^-1022)
  const long long m = (b & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;
  const int sh = ef - 1023 + 10;  // m 2^(e - 52) 2^62
  const long long v = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> -sh) : 0);
  return b < 0 ? -v : v;
}
// v 2^k rounded to the nearest double (ties to even), any int64 v, on the
// integer pipes: the leading bits kept, the dropped ones rounded (a carry out
// of the mantissa lands in the exponent field)
__device__ __forceinline__ double q2d(long long v, int k) {
  const unsigned long long sgn = (unsigned long long)v & 0x8000000000000000ull;
  const unsigned long long a = (v < 0) ? (0ull - (unsigned long long)v) : (unsigned long long)v;
  if (!a) return 0.0;
  const int lz = __clzll((long long)a);
  const int nb = 64 - lz;  // significant bits
  unsigned long long m;
  if (nb <= 53) {
    m = a << (53 - nb);
  } else {
    const int sh = nb - 53;
    m = a >> sh;
    const unsigned long long rem = a & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (m & 1))) m += 1;
  }
  const unsigned long long e = (unsigned long long)(1022 + nb - 1 + k) << 52;
  return __longlong_as_double((long long)(sgn | (e + m)));
}

// sin(r) and cos(r) - 1 in Q1.62 for r (Q1.62) with |r| <= 0.0125 (Taylor to
// r^7 and r^6; the first omitted terms are below 2^-70).
__device__ __forceinline__ void dm_small_q(long long r, long long& s, long long& c_minus_1) {
  const long long r2 = mulq(r, r);
  const long long ps = -qdiv(6) + mulq(r2, qdiv(120) - mulq(r2, qdiv(5040)));
  s = r + mulq(mulq(r2, r), ps);
  const long long pc = -(kQOne / 2) + mulq(r2, qdiv(24) - mulq(r2, qdiv(720)));
  c_minus_1 = mulq(r2, pc);
}

// (sin theta, cos theta).  theta = j pi/128 + r with j = rint(128 theta / pi)
// and r by a three-term Cody-Waite reduction in FP64 (the first two parts of
// pi/128 carry 27 significant bits, so j * part is exact for |j| < 2^26);
// sin r, cos r - 1 and the combination with the table in fixed point:
// sin(a + r) = S + S (cos r - 1) + C sin r, cos(a + r) = C + C (cos r - 1) - S sin r.
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
  long long sr, cm;
  dm_small_q(d2q(r), sr, cm);
  const longlong2 t = __ldg(reinterpret_cast<const longlong2*>(tab + kDirTabQ) + j);  // (S, C) in Q1.62
  s = q2d(t.x + mulq(t.x, cm) + mulq(t.y, sr), -62);
  c = q2d(t.y + mulq(t.y, cm) - mulq(t.x, sr), -62);
}

// cos(pi t) for t = v 2^-52, v in [1, 2^53] (t in (0, 2]) given as the
// integer v, on the integer pipes: t = j/128 + r with j = v / 2^45 rounded to
// nearest (ties to even) and r = (v - j 2^45) 2^-52 exactly, |r| <= 2^-8;
// the angle pi r in Q1.62 from pi in Q2.61; then as dm_sincos.
__device__ __forceinline__ double dm_cospi_grid52(unsigned long long v, const double2* __restrict__ tab) {
  const unsigned long long half = 1ull << 44;
  const unsigned long long q = v >> 45, rem = v & ((1ull << 45) - 1);
  const unsigned long long jr = q + ((rem > half || (rem == half && (q & 1))) ? 1ull : 0ull);
  const int j = (int)(jr & 255);
  const long long rr = (long long)v - (long long)(jr << 45);  // r 2^52, |rr| <= 2^44
  const long long kPiQ61 = 0x6487ED5110B4611ALL;             // round(pi 2^61)
  const long long rq = (long long)(((__int128)rr * kPiQ61) >> 51);  // pi r 2^62
  long long sr, cm;
  dm_small_q(rq, sr, cm);
  const longlong2 tt = __ldg(reinterpret_cast<const longlong2*>(tab + kDirTabQ) + j);
  return q2d(tt.y + mulq(tt.y, cm) - mulq(tt.x, sr), -62);
}

// ln u for a positive normal u: u = 2^k m, m in [M0, 2 M0).  With c_j the
// centre of m's interval, ln m = -ln(1/c_j) + ln(1 + r) where r = m (1/c_j) - 1
// is formed in one FP64 rounding (|r| <= 2^-9); ln(1 + r) = r P(r) with
// P(r) = 1 - r/2 + r^2/3 - ... + r^6/7 (Taylor to r^7) in fixed point, so that
// r P keeps full relative precision when u is near 1 (r tiny, c_j = 1).
__device__ __forceinline__ double dm_log(double u, const double2* __restrict__ tab) {
  const long long b = __double_as_longlong(u);
  const long long d = b - kLogOff;
  const long long k = d >> 52;  // floor
  const int j = (int)((d >> 44) & 255);
  const double m = __longlong_as_double(b - (k << 52));
  const double2 t = __ldg(&tab[256 + j]);  // (1/c_j, -ln(1/c_j))
  const double r = fma(m, t.x, -1.0);
  const long long rq = d2q(r);
  long long p = qdiv(7);
  p = -qdiv(6) + mulq(rq, p);
  p = qdiv(5) + mulq(rq, p);
  p = -(kQOne / 4) + mulq(rq, p);
  p = qdiv(3) + mulq(rq, p);
  p = -(kQOne / 2) + mulq(rq, p);
  p = kQOne + mulq(rq, p);
  const double l1p = r * q2d(p, -62);
  return fma(dm_i2d(k), 0x1.62e42fefa39efp-1, t.y + l1p);  // + k ln 2
}

}  // namespace cgk
