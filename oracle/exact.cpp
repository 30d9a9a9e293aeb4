// Oracle: exact geometric predicates. TEST INFRASTRUCTURE ONLY.
//
// The paper (Sec. 2.C.3) decides whether the triangulation is still valid by
// the empty-circumcircle property of every Delaunay triangle.  Here those
// decisions are made exactly: every coordinate is an integer number of grid
// units (positions are kept on the dyadic grid 2^-q), so the orientation and
// in-circle determinants are evaluated in exact integer arithmetic
// (128-bit products, 256-bit sums).  A cheap double-precision evaluation is
// accepted only when its magnitude exceeds a conservative error bound.
//
// Exactly cocircular inputs are resolved by a symbolic perturbation of the
// lifting map: point p is lifted to |p|^2 + eps_p with eps_p infinitesimal
// and larger for larger `key`.  The perturbed determinant's sign is then the
// sign of the cofactor of the highest-key point (never zero: four distinct
// cocircular points have no three collinear).
#include "internal.h"
#include <cmath>
#include <cstdlib>

namespace cgo {

namespace {

struct I256 {
  uint64_t w[4];
};

I256 i256_neg(const I256& a) {
  I256 r;
  uint64_t carry = 1;
  for (int k = 0; k < 4; ++k) {
    uint64_t v = ~a.w[k];
    u128 s = (u128)v + carry;
    r.w[k] = (uint64_t)s;
    carry = (uint64_t)(s >> 64);
  }
  return r;
}

I256 i256_add(const I256& a, const I256& b) {
  I256 r;
  u128 carry = 0;
  for (int k = 0; k < 4; ++k) {
    u128 s = (u128)a.w[k] + b.w[k] + carry;
    r.w[k] = (uint64_t)s;
    carry = s >> 64;
  }
  return r;
}

// Exact product of two signed 128-bit integers (|a|,|b| < 2^127).
I256 i256_mul(i128 a, i128 b) {
  bool neg = (a < 0) != (b < 0);
  u128 ua = a < 0 ? (u128)0 - (u128)a : (u128)a;
  u128 ub = b < 0 ? (u128)0 - (u128)b : (u128)b;
  uint64_t a0 = (uint64_t)ua, a1 = (uint64_t)(ua >> 64);
  uint64_t b0 = (uint64_t)ub, b1 = (uint64_t)(ub >> 64);
  uint64_t r[4] = {0, 0, 0, 0};
  auto add_at = [&](int k, u128 v) {
    u128 s = (u128)r[k] + (uint64_t)v;
    r[k] = (uint64_t)s;
    u128 c = (s >> 64) + (v >> 64);
    for (int m = k + 1; m < 4 && c != 0; ++m) {
      u128 t = (u128)r[m] + (uint64_t)c;
      r[m] = (uint64_t)t;
      c = (t >> 64) + (c >> 64);
    }
  };
  add_at(0, (u128)a0 * b0);
  add_at(1, (u128)a0 * b1);
  add_at(1, (u128)a1 * b0);
  add_at(2, (u128)a1 * b1);
  I256 out{{r[0], r[1], r[2], r[3]}};
  return neg ? i256_neg(out) : out;
}

int i256_sign(const I256& a) {
  if ((a.w[0] | a.w[1] | a.w[2] | a.w[3]) == 0) return 0;
  return (a.w[3] >> 63) ? -1 : 1;
}

int sgn128(i128 v) { return (v > 0) - (v < 0); }

}  // namespace

// orient2d(a,b,c) = (b-a) x (c-a); > 0 iff a,b,c counter-clockwise.
// Differences are < 2^62 in magnitude, products < 2^124: exact in i128.
int orient2d_exact(const Pt& a, const Pt& b, const Pt& c) {
  i128 bax = (i128)b.X - a.X, bay = (i128)b.Y - a.Y;
  i128 cax = (i128)c.X - a.X, cay = (i128)c.Y - a.Y;
  return sgn128(bax * cay - bay * cax);
}

// incircle(a,b,c,d) = det[[a-d, |a-d|^2],[b-d, |b-d|^2],[c-d, |c-d|^2]].
// > 0 iff d lies strictly inside the circle through a,b,c when a,b,c are CCW.
int incircle_exact(const Pt& a, const Pt& b, const Pt& c, const Pt& d) {
  const int64_t adx = a.X - d.X, ady = a.Y - d.Y;
  const int64_t bdx = b.X - d.X, bdy = b.Y - d.Y;
  const int64_t cdx = c.X - d.X, cdy = c.Y - d.Y;

  // Double-precision filter.  Each difference is rounded once on conversion,
  // then at most five further roundings occur along any product/sum chain, so
  // |err| <= ~10 eps * permanent; 1e-14 (~ 90 eps) is a safe margin.
  {
    double ax = (double)adx, ay = (double)ady, bx = (double)bdx, by = (double)bdy;
    double cx = (double)cdx, cy = (double)cdy;
    double al = ax * ax + ay * ay, bl = bx * bx + by * by, cl = cx * cx + cy * cy;
    double bc = bx * cy - by * cx, ca = cx * ay - cy * ax, ab = ax * by - ay * bx;
    double det = al * bc + bl * ca + cl * ab;
    double perm = al * (std::fabs(bx * cy) + std::fabs(by * cx)) +
                  bl * (std::fabs(cx * ay) + std::fabs(cy * ax)) +
                  cl * (std::fabs(ax * by) + std::fabs(ay * bx));
    double bound = 1.0e-14 * perm;
    if (det > bound) return 1;
    if (det < -bound) return -1;
  }

  // Exact: |differences| < 2^62 -> squares < 2^124; lifts < 2^125.
  i128 al = (i128)adx * adx + (i128)ady * ady;
  i128 bl = (i128)bdx * bdx + (i128)bdy * bdy;
  i128 cl = (i128)cdx * cdx + (i128)cdy * cdy;
  i128 bc = (i128)bdx * cdy - (i128)bdy * cdx;
  i128 ca = (i128)cdx * ady - (i128)cdy * adx;
  i128 ab = (i128)adx * bdy - (i128)ady * bdx;
  I256 s = i256_add(i256_add(i256_mul(al, bc), i256_mul(bl, ca)), i256_mul(cl, ab));
  return i256_sign(s);
}

// Symbolically perturbed in-circle: never returns 0 for distinct points.
// With lifted heights |p|^2 + eps_p, the perturbed determinant is
//   incircle + eps_a*o(b,c,d) + eps_b*o(c,a,d) + eps_c*o(a,b,d) - eps_d*o(a,b,c)
// (o = orient2d), and the highest-key point's term dominates.
int incircle_sos(const Pt& a, const Pt& b, const Pt& c, const Pt& d) {
  int s = incircle_exact(a, b, c, d);
  if (s != 0) return s;
  const Pt* p[4] = {&a, &b, &c, &d};
  int top = 0;
  for (int k = 1; k < 4; ++k)
    if (p[k]->key > p[top]->key) top = k;
  switch (top) {
    case 0: return orient2d_exact(b, c, d);
    case 1: return orient2d_exact(c, a, d);
    case 2: return orient2d_exact(a, b, d);
    default: return -orient2d_exact(a, b, c);
  }
}

}  // namespace cgo
