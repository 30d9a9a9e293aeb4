// Oracle: adjoint (reverse-mode gradient) of an SPV run. TEST INFRASTRUCTURE ONLY.
//
// Step map of Eq. 3 with the director noise fixed (replayed from the seed):
//   r_{t+1} = r_t + dt (mu F(r_t; p0, K_A, K_P) + v0 n(theta_t)),  F = -grad E.
// Its transposed Jacobian is I - dt mu H(r_t) with H the (symmetric) Hessian of
// E, so the cotangent of the positions runs backwards as
//   g_t = g_{t+1} - dt mu H(r_t) g_{t+1}.
// H v is the forward-mode derivative of -F along v, computed here by running
// the oracle's own force code (spv_core.h, pinned by finite differences of E)
// on dual numbers.  Parameter cotangents, from the same forward derivative of
// the areas and perimeters along g = g_{t+1} (Adot, Pdot):
//   dL/dp0_i += dt mu 2 K_P sqrt(A0) Pdot_i            (dF/dp0_i = 2K_P sqrt(A0) grad P_i)
//   dL/dK_A  += -dt mu sum_c 2 (A_c - A0) Adot_c       (dF/dK_A = -sum_c 2(A_c-A0) grad A_c)
//   dL/dK_P  += -dt mu sum_c 2 (P_c - P0_c) Pdot_c
//   dL/dv0_i += dt g_i . n(theta_i)
// A loss on the final areas and perimeters enters through the force machinery
// with per-cell coefficients (dL/dA_c, dL/dP_c) in place of 2K(A-A0), 2K(P-P0).
// Topology is frozen within each step (the triangulation of r_t).
#include "internal.h"
#include "spv_core.h"

#include <cmath>
#include <cstring>

extern "C" int cgo_triangulate(int n, double Lx, double Ly, const double* x, const double* y, int max_ring,
                               int32_t* cnt, int32_t* nbr, int32_t* off);
extern "C" int cgo_integrate(int n, double Lx, double Ly, double* x, double* y, double* theta, const double* Fx,
                             const double* Fy, const double* v0, const double* par, uint64_t seed, int64_t step);

namespace cgo {

// Forward-mode dual number v + d eps.
struct Dual {
  double v, d;
  Dual(double a = 0.0, double b = 0.0) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator+(Dual a, double b) { return Dual(a.v + b, a.d); }
inline Dual operator+(double a, Dual b) { return Dual(a + b.v, b.d); }
inline Dual operator-(Dual a, double b) { return Dual(a.v - b, a.d); }
inline Dual operator-(double a, Dual b) { return Dual(a - b.v, -b.d); }
inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
inline Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
inline Dual operator/(double a, Dual b) { return Dual(a / b.v, -a * b.d / (b.v * b.v)); }
inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}

namespace {

struct Topo {
  std::vector<int32_t> cnt, nbr, off;
};

// H v, and the derivatives of A and P along v, at the state (x, y) with the
// given topology.
int hvp(int n, double Lx, double Ly, const double* x, const double* y, const Topo& t, int R, const double* p0,
        const double* mech, const double* vx, const double* vy, double* Hvx, double* Hvy, double* Adot,
        double* Pdot) {
  std::vector<Dual> dx(n), dy(n), Fx(n), Fy(n), A(n), P(n);
  for (int i = 0; i < n; ++i) {
    dx[i] = Dual(x[i], vx[i]);
    dy[i] = Dual(y[i], vy[i]);
  }
  GeoT<Dual> g{n, Lx, Ly, R, dx.data(), dy.data(), t.cnt.data(), t.nbr.data(), t.off.data()};
  MechT<Dual> mp{mech[0], mech[1], mech[2], p0};
  int rc = forces_t(g, mp, Fx.data(), Fy.data(), A.data(), P.data(), (Dual*)nullptr);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {
    if (Hvx) Hvx[i] = -Fx[i].d;
    if (Hvy) Hvy[i] = -Fy[i].d;
    if (Adot) Adot[i] = A[i].d;
    if (Pdot) Pdot[i] = P[i].d;
  }
  return 0;
}

int triangulate_topo(int n, double Lx, double Ly, const double* x, const double* y, int R, Topo& t) {
  t.cnt.assign(n, 0);
  t.nbr.assign((size_t)n * R, -1);
  t.off.assign((size_t)n * R * 2, 0);
  return cgo_triangulate(n, Lx, Ly, x, y, R, t.cnt.data(), t.nbr.data(), t.off.data());
}

}  // namespace
}  // namespace cgo

using namespace cgo;

extern "C" {

// H v (Hessian of E times v) and the derivatives of A, P along v, on a given
// topology.  mech = {A0, KA, KP}.
int cgo_hvp(int n, double Lx, double Ly, const double* x, const double* y, const int32_t* cnt, const int32_t* nbr,
            const int32_t* off, int max_ring, const double* p0, const double* mech, const double* vx,
            const double* vy, double* Hvx, double* Hvy, double* Adot, double* Pdot) {
  Topo t;
  t.cnt.assign(cnt, cnt + n);
  t.nbr.assign(nbr, nbr + (size_t)n * max_ring);
  t.off.assign(off, off + (size_t)n * max_ring * 2);
  return hvp(n, Lx, Ly, x, y, t, max_ring, p0, mech, vx, vy, Hvx, Hvy, Adot, Pdot);
}

// Gradient of sum_c (cA_c A_c + cP_c P_c) with respect to the positions.
int cgo_geom_grad(int n, double Lx, double Ly, const double* x, const double* y, const int32_t* cnt,
                  const int32_t* nbr, const int32_t* off, int max_ring, const double* cA, const double* cP,
                  double* gx, double* gy) {
  std::vector<double> p0(n, 0.0), A(n), P(n);
  GeoT<double> g{n, Lx, Ly, max_ring, x, y, cnt, nbr, off};
  MechT<double> mp{1.0, 0.0, 0.0, p0.data()};
  int rc = forces_t(g, mp, gx, gy, A.data(), P.data(), (double*)nullptr, nullptr, cA, cP);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {
    gx[i] = -gx[i];
    gy[i] = -gy[i];
  }
  return 0;
}

// Forward run of nsteps (triangulating from scratch every step) and the
// reverse pass for the cotangents (gx_T, gy_T, gA_T, gP_T) of the final
// positions, areas and perimeters.  par = {A0, KA, KP, mu, Dr, dt}.
// Outputs: final state (xT, yT, AT, PT), cotangents of the initial positions
// (gx0, gy0), of per-cell p0 and v0 (gp0, gv0), and of (K_A, K_P) (gK[2]).
int cgo_spv_backward(int n, double Lx, double Ly, const double* x0, const double* y0, const double* theta0,
                     const double* p0, const double* v0, const double* par, uint64_t seed, int64_t step0,
                     int64_t nsteps, const double* gxT, const double* gyT, const double* gAT, const double* gPT,
                     double* xT, double* yT, double* AT, double* PT, double* gx0, double* gy0, double* gp0,
                     double* gv0, double* gK) {
  const int R = 16;
  const double A0 = par[0], KA = par[1], KP = par[2], mu = par[3], dt = par[5];
  const double sqA0 = std::sqrt(A0);
  const double mech[3] = {A0, KA, KP};
  const double ipar[3] = {par[3], par[4], par[5]};
  std::vector<std::vector<double>> xs(nsteps + 1), ys(nsteps + 1), ths(nsteps + 1);
  std::vector<Topo> topo(nsteps + 1);
  xs[0].assign(x0, x0 + n);
  ys[0].assign(y0, y0 + n);
  ths[0].assign(theta0, theta0 + n);
  std::vector<double> Fx(n), Fy(n), A(n), P(n);
  for (int64_t t = 0; t < nsteps; ++t) {
    int rc = triangulate_topo(n, Lx, Ly, xs[t].data(), ys[t].data(), R, topo[t]);
    if (rc) return rc;
    GeoT<double> g{n, Lx, Ly, R, xs[t].data(), ys[t].data(), topo[t].cnt.data(), topo[t].nbr.data(),
                   topo[t].off.data()};
    MechT<double> mp{A0, KA, KP, p0};
    rc = forces_t(g, mp, Fx.data(), Fy.data(), A.data(), P.data(), (double*)nullptr);
    if (rc) return rc;
    xs[t + 1] = xs[t];
    ys[t + 1] = ys[t];
    ths[t + 1] = ths[t];
    rc = cgo_integrate(n, Lx, Ly, xs[t + 1].data(), ys[t + 1].data(), ths[t + 1].data(), Fx.data(), Fy.data(), v0,
                       ipar, seed, step0 + t);
    if (rc) return rc;
  }
  int rc = triangulate_topo(n, Lx, Ly, xs[nsteps].data(), ys[nsteps].data(), R, topo[nsteps]);
  if (rc) return rc;
  {
    GeoT<double> g{n, Lx, Ly, R, xs[nsteps].data(), ys[nsteps].data(), topo[nsteps].cnt.data(),
                   topo[nsteps].nbr.data(), topo[nsteps].off.data()};
    std::vector<double> hx, hy;
    polygons_t(g, hx, hy, A.data(), P.data());
  }
  for (int i = 0; i < n; ++i) {
    xT[i] = xs[nsteps][i];
    yT[i] = ys[nsteps][i];
    AT[i] = A[i];
    PT[i] = P[i];
  }
  // cotangent of the final positions: direct part + the area/perimeter loss terms
  std::vector<double> gx(n), gy(n);
  rc = cgo_geom_grad(n, Lx, Ly, xs[nsteps].data(), ys[nsteps].data(), topo[nsteps].cnt.data(),
                     topo[nsteps].nbr.data(), topo[nsteps].off.data(), R, gAT, gPT, gx.data(), gy.data());
  if (rc) return rc;
  for (int i = 0; i < n; ++i) {
    gx[i] += gxT[i];
    gy[i] += gyT[i];
    gp0[i] = 0.0;
    gv0[i] = 0.0;
  }
  gK[0] = gK[1] = 0.0;
  std::vector<double> Hx(n), Hy(n), Ad(n), Pd(n), At(n), Pt(n);
  for (int64_t t = nsteps - 1; t >= 0; --t) {
    rc = hvp(n, Lx, Ly, xs[t].data(), ys[t].data(), topo[t], R, p0, mech, gx.data(), gy.data(), Hx.data(),
             Hy.data(), Ad.data(), Pd.data());
    if (rc) return rc;
    {
      GeoT<double> g{n, Lx, Ly, R, xs[t].data(), ys[t].data(), topo[t].cnt.data(), topo[t].nbr.data(),
                     topo[t].off.data()};
      std::vector<double> hx, hy;
      polygons_t(g, hx, hy, At.data(), Pt.data());
    }
    double sKA = 0.0, sKP = 0.0;
    for (int c = 0; c < n; ++c) {
      gp0[c] += dt * mu * 2.0 * KP * sqA0 * Pd[c];
      sKA += 2.0 * (At[c] - A0) * Ad[c];
      sKP += 2.0 * (Pt[c] - p0[c] * sqA0) * Pd[c];
      gv0[c] += dt * (gx[c] * std::cos(ths[t][c]) + gy[c] * std::sin(ths[t][c]));
    }
    gK[0] += -dt * mu * sKA;
    gK[1] += -dt * mu * sKP;
    for (int i = 0; i < n; ++i) {
      gx[i] -= dt * mu * Hx[i];
      gy[i] -= dt * mu * Hy[i];
    }
  }
  for (int i = 0; i < n; ++i) {
    gx0[i] = gx[i];
    gy0[i] = gy[i];
  }
  return 0;
}

}  // extern "C"
