// Oracle: self-propelled Voronoi (SPV) model, one plain CPU step at a time.
// TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the timed CPU
// baseline of bench.py; never by the library.
//
// What is computed, with the passage of Sussman, arXiv 1702.02939 it follows:
//  * periodic Delaunay triangulation from scratch (3x3 image tiling +
//    Bowyer-Watson, exact predicates)                      -- Sec. 2.C.3
//  * Voronoi vertices as circumcentres h = r_i + z/d       -- Eqs. A8-A12
//  * areas A_i (shoelace) and perimeters P_i               -- Sec. 2.C.1
//  * energy E = sum K_A (A_i - A0)^2 + K_P (P_i - P0_i)^2  -- Eq. 1 / A1
//  * force sets dE_c/dh per (cell, vertex)                 -- Eqs. A3-A5
//  * net force F_i = -sum_t (dh_t/dr_i)^T G_t              -- Eqs. A6, A7, A16
//  * overdamped active update dr/dt = mu F + v0 n(theta),
//    dtheta/dt = eta with variance 2 D_r (Euler-Maruyama)  -- Eq. 3, Sec. 2.C.3
// Readings of garbled/silent passages (each also stated in the design notes):
//  - Eq. 2 prints F = +grad E; Eq. A6 has the minus sign: F = -grad E.
//  - Eq. A5 prints dP/dh = -(t_ij + t_ik); with t_ij = h_ijk - h_gij and
//    t_ik = h_ikl - h_ijk the derivative of sum |t| is  t^_ij - t^_ik.
//  - Eq. A14 must read  d(gamma d)/dr_i = -2 (r_ik.r_jk) r_ij - |r_ij|^2 r_jk,
//    and Eq. A15 must read (1/d) dd/dr_i = (2/c) (r_jk,y, -r_jk,x) for c as
//    defined in Eq. A8 (both re-derived; pinned by finite differences).
//  - P0_i = p0_i * sqrt(A0) (p0 is the dimensionless target shape index).
//  - positions are kept on the dyadic grid 2^-q, q = 50 - ceil(log2 max(Lx,Ly)),
//    so coordinate differences are exact and predicates are decidable exactly.
#include "internal.h"
#include "spv_core.h"
#include <chrono>
#include <cmath>
#include <cstring>

namespace cgo {
namespace {

using Geo = GeoT<double>;
using Mech = MechT<double>;

// Periodic reduction of a finite coordinate (any move size): v' = fmod(v, L)
// is exact, v' is rounded to the grid 2^-q, and the grid integer is wrapped
// into [0, L 2^q).  Returns false for a non-finite v.
inline bool snap_wrap_ok(double v, double L, int q, double& out) {
  if (!std::isfinite(v)) return false;
  double r = std::fmod(v, L);
  double X = std::rint(std::ldexp(r, q));
  double LX = std::ldexp(L, q);
  if (X < 0.0) X += LX;
  else if (X >= LX) X -= LX;
  out = std::ldexp(X, -q) + 0.0;
  return true;
}
inline double snap_wrap(double v, double L, int q) {
  double out = 0.0;
  snap_wrap_ok(v, L, q, out);
  return out;
}

int grid_exponent(double Lx, double Ly) {
  double m = Lx > Ly ? Lx : Ly;
  int ex;
  double fr = std::frexp(m, &ex);  // m = fr * 2^ex, fr in [0.5, 1)
  int e = (fr == 0.5) ? ex - 1 : ex;
  return 50 - e;
}

// uniform in (0, 1]: (53 high bits of (hi:lo) + 1) * 2^-53
inline double u53(uint32_t hi, uint32_t lo) {
  uint64_t k = ((((uint64_t)hi) << 32) | lo) >> 11;
  return std::ldexp((double)(k + 1), -53);
}

double director_noise(uint64_t seed, int32_t tag, int64_t step) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr[4] = {(uint32_t)tag, (uint32_t)(uint64_t)step, (uint32_t)((uint64_t)step >> 32), 0u};
  uint32_t out[4];
  philox4x32_10(ctr, key, out);
  double u1 = u53(out[0], out[1]), u2 = u53(out[2], out[3]);
  // Box-Muller, cosine branch
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

int triangulate(int n, double Lx, double Ly, const double* x, const double* y, int max_ring,
                int32_t* cnt, int32_t* nbr, int32_t* off) {
  int q = grid_exponent(Lx, Ly);
  int64_t LX = (int64_t)std::ldexp(Lx, q), LY = (int64_t)std::ldexp(Ly, q);
  std::vector<Pt> pts;
  std::vector<char> central;
  pts.reserve((size_t)9 * n);
  for (int oy = -1; oy <= 1; ++oy)
    for (int ox = -1; ox <= 1; ++ox)
      for (int i = 0; i < n; ++i) {
        int64_t X = (int64_t)std::ldexp(x[i], q), Y = (int64_t)std::ldexp(y[i], q);
        int img = (oy + 1) * 3 + (ox + 1);
        pts.push_back(Pt{X + ox * LX, Y + oy * LY, i, ox, oy, (int64_t)i * 16 + img});
        central.push_back(ox == 0 && oy == 0);
      }
  std::vector<Ring> rings;
  int rc = bowyer_watson_rings(pts, central, rings);
  if (rc) return rc;
  for (size_t p = 0; p < pts.size(); ++p) {
    if (!central[p]) continue;
    int i = pts[p].tag;
    const Ring& r = rings[p];
    if ((int)r.tag.size() > max_ring) return -5;  // ring overflow
    cnt[i] = (int32_t)r.tag.size();
    for (int a = 0; a < max_ring; ++a) {
      bool on = a < (int)r.tag.size();
      nbr[i * max_ring + a] = on ? r.tag[a] : -1;
      off[(i * max_ring + a) * 2 + 0] = on ? r.ox[a] : 0;
      off[(i * max_ring + a) * 2 + 1] = on ? r.oy[a] : 0;
    }
  }
  return 0;
}

}  // namespace
}  // namespace cgo

using namespace cgo;

extern "C" {

int cgo_grid_exponent(double Lx, double Ly) { return grid_exponent(Lx, Ly); }

double cgo_snap_length(double L, int q) { return std::ldexp(std::rint(std::ldexp(L, q)), -q); }

// Snaps positions onto the grid and wraps them into [0, L). Inputs must lie in [-L, 2L).
int cgo_snap_positions(int n, double Lx, double Ly, double* x, double* y) {
  int q = grid_exponent(Lx, Ly);
  for (int i = 0; i < n; ++i) {
    if (!(x[i] >= -Lx && x[i] < 2 * Lx && y[i] >= -Ly && y[i] < 2 * Ly)) return -1;
    x[i] = snap_wrap(x[i], Lx, q);
    y[i] = snap_wrap(y[i], Ly, q);
  }
  return 0;
}

void cgo_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  philox4x32_10(ctr, key, out);
}

double cgo_director_noise(uint64_t seed, int32_t tag, int64_t step) {
  return director_noise(seed, tag, step);
}

static Pt mkpt(const int64_t* p, int64_t key) { return Pt{p[0], p[1], 0, 0, 0, key}; }

int cgo_orient2d(const int64_t* a, const int64_t* b, const int64_t* c) {
  return orient2d_exact(mkpt(a, 0), mkpt(b, 0), mkpt(c, 0));
}

int cgo_incircle(const int64_t* a, const int64_t* b, const int64_t* c, const int64_t* d) {
  return incircle_exact(mkpt(a, 0), mkpt(b, 0), mkpt(c, 0), mkpt(d, 0));
}

int cgo_incircle_sos(const int64_t* a, const int64_t* b, const int64_t* c, const int64_t* d,
                     const int64_t* keys) {
  return incircle_sos(mkpt(a, keys[0]), mkpt(b, keys[1]), mkpt(c, keys[2]), mkpt(d, keys[3]));
}

// Delaunay triangulation of a plain (non-periodic) point set given in grid
// units; rings of every interior point (CCW, starting at the smallest index);
// hull points get cnt = 0.
int cgo_delaunay_plain(int m, const int64_t* X, const int64_t* Y, int max_ring, int32_t* cnt,
                       int32_t* nbr) {
  std::vector<Pt> pts(m);
  std::vector<char> central(m, 1);
  for (int i = 0; i < m; ++i) pts[i] = Pt{X[i], Y[i], i, 0, 0, (int64_t)i};
  std::vector<Ring> rings;
  int rc = bowyer_watson_rings(pts, central, rings, true);
  if (rc) return rc;
  for (int i = 0; i < m; ++i) {
    if ((int)rings[i].tag.size() > max_ring) return -5;
    cnt[i] = (int32_t)rings[i].tag.size();
    for (int a = 0; a < max_ring; ++a)
      nbr[i * max_ring + a] = a < cnt[i] ? rings[i].tag[a] : -1;
  }
  return 0;
}

int cgo_triangulate(int n, double Lx, double Ly, const double* x, const double* y, int max_ring,
                    int32_t* cnt, int32_t* nbr, int32_t* off) {
  return triangulate(n, Lx, Ly, x, y, max_ring, cnt, nbr, off);
}

// Voronoi vertices (relative to each cell), areas and perimeters.
int cgo_geometry(int n, double Lx, double Ly, const double* x, const double* y,
                 const int32_t* cnt, const int32_t* nbr, const int32_t* off, int max_ring,
                 double* A, double* P, double* hx, double* hy) {
  Geo g{n, Lx, Ly, max_ring, x, y, cnt, nbr, off};
  std::vector<double> vx, vy;
  polygons_t(g, vx, vy, A, P);
  if (hx) std::memcpy(hx, vx.data(), sizeof(double) * vx.size());
  if (hy) std::memcpy(hy, vy.data(), sizeof(double) * vy.size());
  return 0;
}

// mech = {A0, KA, KP}
int cgo_forces(int n, double Lx, double Ly, const double* x, const double* y, const int32_t* cnt,
               const int32_t* nbr, const int32_t* off, int max_ring, const double* p0,
               const double* mech, double* Fx, double* Fy, double* A, double* P, double* E) {
  Geo g{n, Lx, Ly, max_ring, x, y, cnt, nbr, off};
  Mech mp{mech[0], mech[1], mech[2], p0};
  return forces_t(g, mp, Fx, Fy, A, P, E);
}

// One Euler-Maruyama update (Eq. 3) from given forces; positions snapped/wrapped.
// par = {mu, Dr, dt}
// The same update for cells whose noise counters are tag0 + i: the cells of
// one system placed from index tag0 on in a larger numbering (the tag is the
// cell's index in the Philox counter of the director noise).
int cgo_integrate_tagged(int n, double Lx, double Ly, double* x, double* y, double* theta,
                         const double* Fx, const double* Fy, const double* v0, const double* par,
                         uint64_t seed, int64_t step, int64_t tag0) {
  int q = grid_exponent(Lx, Ly);
  double mu = par[0], Dr = par[1], dt = par[2];
  double s = std::sqrt(2.0 * Dr * dt);
  for (int i = 0; i < n; ++i) {
    double vx = mu * Fx[i] + v0[i] * std::cos(theta[i]);
    double vy = mu * Fy[i] + v0[i] * std::sin(theta[i]);
    double xn = x[i] + dt * vx, yn = y[i] + dt * vy;
    if (!snap_wrap_ok(xn, Lx, q, x[i]) || !snap_wrap_ok(yn, Ly, q, y[i])) return -6;  // non-finite move
    theta[i] = theta[i] + s * director_noise(seed, (int)(tag0 + i), step);
  }
  return 0;
}

int cgo_integrate(int n, double Lx, double Ly, double* x, double* y, double* theta,
                  const double* Fx, const double* Fy, const double* v0, const double* par,
                  uint64_t seed, int64_t step) {
  return cgo_integrate_tagged(n, Lx, Ly, x, y, theta, Fx, Fy, v0, par, seed, step, 0);
}

// nsteps full oracle steps: triangulate from scratch, forces, update.
// par = {A0, KA, KP, mu, Dr, dt}.  Final forces/areas/perimeters of the last
// step's starting state are left in Fx, Fy, A, P (may be NULL).
int cgo_spv_run(int n, double Lx, double Ly, double* x, double* y, double* theta,
                const double* p0, const double* v0, const double* par, uint64_t seed,
                int64_t step0, int64_t nsteps, double* Fx, double* Fy, double* A, double* P) {
  const int R = 16;
  std::vector<int32_t> cnt(n), nbr((size_t)n * R), off((size_t)n * R * 2);
  std::vector<double> fx(n), fy(n), a(n), p(n);
  Mech mp{par[0], par[1], par[2], p0};
  double ipar[3] = {par[3], par[4], par[5]};
  for (int64_t s = 0; s < nsteps; ++s) {
    int rc = triangulate(n, Lx, Ly, x, y, R, cnt.data(), nbr.data(), off.data());
    if (rc) return rc;
    Geo g{n, Lx, Ly, R, x, y, cnt.data(), nbr.data(), off.data()};
    rc = forces_t(g, mp, fx.data(), fy.data(), a.data(), p.data(), (double*)nullptr);
    if (rc) return rc;
    if (Fx) std::memcpy(Fx, fx.data(), sizeof(double) * n);
    if (Fy) std::memcpy(Fy, fy.data(), sizeof(double) * n);
    if (A) std::memcpy(A, a.data(), sizeof(double) * n);
    if (P) std::memcpy(P, p.data(), sizeof(double) * n);
    rc = cgo_integrate(n, Lx, Ly, x, y, theta, fx.data(), fy.data(), v0, ipar, seed, step0 + s);
    if (rc) return rc;
  }
  return 0;
}

// One oracle step restricted to a square window of the periodic system: the
// cells within hw + margin of (cx, cy) are triangulated from scratch (plain
// Bowyer-Watson), and the cells within hw of the centre get their exact force
// and update (their rings and their neighbours' rings lie well inside the
// triangulated patch when margin >= 6 mean spacings).  Used as a bounded
// sample of a large workload for CPU timing.  (cx, cy) must lie on the grid.
// Returns the number of updated (interior) cells, or a negative error code.
int cgo_spv_window_step(int n, double Lx, double Ly, double* x, double* y, double* theta,
                        const double* p0, const double* v0, const double* par, uint64_t seed,
                        int64_t step, double cx, double cy, double hw, double margin) {
  const int q = grid_exponent(Lx, Ly);
  const int R = 16;
  std::vector<int> ids;
  std::vector<double> lx, ly;
  for (int i = 0; i < n; ++i) {
    double dx = x[i] - cx, dy = y[i] - cy;
    if (dx >= 0.5 * Lx) dx -= Lx; else if (dx < -0.5 * Lx) dx += Lx;
    if (dy >= 0.5 * Ly) dy -= Ly; else if (dy < -0.5 * Ly) dy += Ly;
    if (std::fabs(dx) < hw + margin && std::fabs(dy) < hw + margin) {
      ids.push_back(i);
      lx.push_back(dx);
      ly.push_back(dy);
    }
  }
  const int m = (int)ids.size();
  std::vector<Pt> pts(m);
  std::vector<char> central(m, 1);
  for (int k = 0; k < m; ++k)
    pts[k] = Pt{(int64_t)std::ldexp(lx[k], q), (int64_t)std::ldexp(ly[k], q), ids[k], 0, 0,
                (int64_t)ids[k] * 16};
  std::vector<Ring> rings;
  int rc = bowyer_watson_rings(pts, central, rings, true);
  if (rc) return rc;
  // local tags -> local indices
  std::vector<int> local_of(n, -1);
  for (int k = 0; k < m; ++k) local_of[ids[k]] = k;
  std::vector<int32_t> cnt(m, 0), nbr((size_t)m * R, -1), off((size_t)m * R * 2, 0);
  std::vector<char> interior(m, 0);
  int n_int = 0;
  const double valid = hw + margin - 3.0;
  for (int k = 0; k < m; ++k) {
    interior[k] = std::fabs(lx[k]) < hw && std::fabs(ly[k]) < hw;
    n_int += interior[k];
    if (!(std::fabs(lx[k]) < valid && std::fabs(ly[k]) < valid)) continue;
    const Ring& r = rings[k];
    if (r.tag.empty()) continue;
    if ((int)r.tag.size() > R) return -5;
    cnt[k] = (int32_t)r.tag.size();
    for (size_t a = 0; a < r.tag.size(); ++a) nbr[(size_t)k * R + a] = local_of[r.tag[a]];
  }
  Geo g{m, 2.0 * Lx, 2.0 * Ly, R, lx.data(), ly.data(), cnt.data(), nbr.data(), off.data()};
  std::vector<double> lp0(m), fx(m, 0.0), fy(m, 0.0), A(m), P(m);
  for (int k = 0; k < m; ++k) lp0[k] = p0[ids[k]];
  Mech mp{par[0], par[1], par[2], lp0.data()};
  rc = forces_t(g, mp, fx.data(), fy.data(), A.data(), P.data(), (double*)nullptr, interior.data());
  if (rc) return rc;
  const double mu = par[3], Dr = par[4], dt = par[5];
  const double s = std::sqrt(2.0 * Dr * dt);
  for (int k = 0; k < m; ++k) {
    if (!interior[k]) continue;
    const int i = ids[k];
    double vx = mu * fx[k] + v0[i] * std::cos(theta[i]);
    double vy = mu * fy[k] + v0[i] * std::sin(theta[i]);
    x[i] = snap_wrap(x[i] + dt * vx, Lx, q);
    y[i] = snap_wrap(y[i] + dt * vy, Ly, q);
    theta[i] = theta[i] + s * director_noise(seed, i, step);
  }
  return n_int;
}

}  // extern "C"
