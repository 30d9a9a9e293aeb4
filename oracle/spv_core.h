// Oracle: SPV geometry and forces, written once for any scalar type T
// (double, or the forward-mode dual number of adjoint.cpp).  TEST
// INFRASTRUCTURE ONLY.
//
// Follows Sussman, arXiv 1702.02939:
//  * Voronoi vertices as circumcentres h = r_i + z/d            Eqs. A8-A12
//  * areas (shoelace) and perimeters                            Sec. 2.C.1
//  * force sets dE_c/dh = 2K_A(A_c-A0) dA_c/dh + 2K_P(P_c-P0_c) dP_c/dh,
//    dA/dh = 1/2 (l_ij n_ij + l_ik n_ik), dP/dh = t^_ij - t^_ik   Eqs. A3-A5
//  * net force F_i = -sum_t (dh_t/dr_i)^T G_t with dh/dr_i of Eq. A16
//    (Eqs. A14, A15 corrected)                                  Eqs. A6, A7, A13-A16
// Optional per-cell coefficients (cA_c, cP_c) replace 2K_A(A_c-A0) and
// 2K_P(P_c-P0_c); the result is then -sum_c (cA_c grad A_c + cP_c grad P_c),
// the gradient of any function of the areas and perimeters.
#pragma once
#include <cmath>
#include <cstdint>
#include <vector>

namespace cgo {

template <class T>
struct GeoT {
  int n = 0;
  double Lx = 0, Ly = 0;
  int max_ring = 16;
  const T *x = nullptr, *y = nullptr;
  const int32_t *cnt = nullptr, *nbr = nullptr, *off = nullptr;
};

template <class T>
struct MechT {
  double A0, KA, KP;
  const double* p0;
};

// Vector from cell i to the image of ring entry a of cell i.
template <class T>
inline void rel_t(const GeoT<T>& g, int i, int a, T& dx, T& dy) {
  int j = g.nbr[i * g.max_ring + a];
  int ox = g.off[(i * g.max_ring + a) * 2 + 0];
  int oy = g.off[(i * g.max_ring + a) * 2 + 1];
  dx = (g.x[j] - g.x[i]) + ox * g.Lx;
  dy = (g.y[j] - g.y[i]) + oy * g.Ly;
}

// Circumcentre of (r_i, r_j, r_k) relative to r_i, written as in Eqs. A8-A12:
//   c = r_ij x r_kj, d = 2c^2, beta d = -|r_ik|^2 (r_ij . r_jk),
//   gamma d = |r_ij|^2 (r_ik . r_jk), z = beta d r_ij + gamma d r_ik, h - r_i = z/d.
template <class T>
void circumcentre_rel_t(const T& rijx, const T& rijy, const T& rikx, const T& riky, T& hx, T& hy) {
  T rjkx = rikx - rijx, rjky = riky - rijy;
  T rkjx = -rjkx, rkjy = -rjky;
  T c = rijx * rkjy - rijy * rkjx;
  T d = 2.0 * c * c;
  T betad = -(rikx * rikx + riky * riky) * (rijx * rjkx + rijy * rjky);
  T gammad = (rijx * rijx + rijy * rijy) * (rikx * rjkx + riky * rjky);
  T zx = betad * rijx + gammad * rikx;
  T zy = betad * rijy + gammad * riky;
  hx = zx / d;
  hy = zy / d;
}

// Voronoi polygon of every cell (vertices relative to the cell), A and P.
template <class T>
void polygons_t(const GeoT<T>& g, std::vector<T>& hx, std::vector<T>& hy, T* A, T* P) {
  using std::sqrt;
  hx.assign((size_t)g.n * g.max_ring, T(0.0));
  hy.assign((size_t)g.n * g.max_ring, T(0.0));
  for (int i = 0; i < g.n; ++i) {
    int m = g.cnt[i];
    for (int a = 0; a < m; ++a) {
      T ax, ay, bx, by;
      rel_t(g, i, a, ax, ay);
      rel_t(g, i, (a + 1) % m, bx, by);
      circumcentre_rel_t(ax, ay, bx, by, hx[i * g.max_ring + a], hy[i * g.max_ring + a]);
    }
    T area(0.0), per(0.0);
    for (int a = 0; a < m; ++a) {
      T x0 = hx[i * g.max_ring + a], y0 = hy[i * g.max_ring + a];
      T x1 = hx[i * g.max_ring + (a + 1) % m], y1 = hy[i * g.max_ring + (a + 1) % m];
      area = area + (x0 * y1 - x1 * y0);
      per = per + sqrt((x1 - x0) * (x1 - x0) + (y1 - y0) * (y1 - y0));
    }
    A[i] = 0.5 * area;
    P[i] = per;
  }
}

// Slot b of cell c's ring such that ring(c)[b] = (u, ou) and ring(c)[b+1] = (w, ow).
template <class T>
int find_pair_t(const GeoT<T>& g, int c, int u, int oux, int ouy, int w, int owx, int owy) {
  int m = g.cnt[c];
  for (int b = 0; b < m; ++b) {
    int e0 = c * g.max_ring + b, e1 = c * g.max_ring + (b + 1) % m;
    if (g.nbr[e0] == u && g.off[2 * e0] == oux && g.off[2 * e0 + 1] == ouy && g.nbr[e1] == w &&
        g.off[2 * e1] == owx && g.off[2 * e1 + 1] == owy)
      return b;
  }
  return -1;
}

// Forces on every cell (or on the cells with only[i] set).  Returns 0, or -10
// for inconsistent rings.
template <class T>
int forces_t(const GeoT<T>& g, const MechT<T>& mp, T* Fx, T* Fy, T* A, T* P, T* energy,
             const char* only = nullptr, const T* coefA = nullptr, const T* coefP = nullptr) {
  using std::sqrt;
  std::vector<T> hx, hy;
  polygons_t(g, hx, hy, A, P);
  const double sqA0 = std::sqrt(mp.A0);
  T E(0.0);
  // force sets dE_c/dh at every vertex of every cell (Eq. A3 with A4, A5)
  std::vector<T> sx((size_t)g.n * g.max_ring, T(0.0)), sy((size_t)g.n * g.max_ring, T(0.0));
  for (int c = 0; c < g.n; ++c) {
    double P0 = mp.p0[c] * sqA0;
    T ka = coefA ? coefA[c] : 2.0 * mp.KA * (A[c] - mp.A0);
    T kp = coefP ? coefP[c] : 2.0 * mp.KP * (P[c] - P0);
    E = E + mp.KA * (A[c] - mp.A0) * (A[c] - mp.A0) + mp.KP * (P[c] - P0) * (P[c] - P0);
    int m = g.cnt[c];
    for (int a = 0; a < m; ++a) {
      int ip = c * g.max_ring + (a + m - 1) % m, ia = c * g.max_ring + a,
          in = c * g.max_ring + (a + 1) % m;
      T tinx = hx[ia] - hx[ip], tiny = hy[ia] - hy[ip];   // t_ij (incoming edge)
      T toutx = hx[in] - hx[ia], touty = hy[in] - hy[ia];  // t_ik (outgoing edge)
      // Eq. A4: dA/dh = 1/2 (l_ij n_ij + l_ik n_ik), outward normal l n = (t_y, -t_x)
      T dAx = 0.5 * (tiny + touty), dAy = 0.5 * (-tinx - toutx);
      // Eq. A5 (corrected): dP/dh = t^_ij - t^_ik
      T lin = sqrt(tinx * tinx + tiny * tiny);
      T lout = sqrt(toutx * toutx + touty * touty);
      T dPx = tinx / lin - toutx / lout, dPy = tiny / lin - touty / lout;
      sx[ia] = ka * dAx + kp * dPx;
      sy[ia] = ka * dAy + kp * dPy;
    }
  }
  if (energy) *energy = E;
  // net force (Eqs. A6, A7): F_i = - sum_{t ni i} (dh_t/dr_i)^T G_t
  for (int i = 0; i < g.n; ++i) {
    if (only && !only[i]) continue;
    int m = g.cnt[i];
    T fx(0.0), fy(0.0);
    for (int a = 0; a < m; ++a) {
      int ea = i * g.max_ring + a, eb = i * g.max_ring + (a + 1) % m;
      int j = g.nbr[ea], k = g.nbr[eb];
      int ojx = g.off[2 * ea], ojy = g.off[2 * ea + 1];
      int okx = g.off[2 * eb], oky = g.off[2 * eb + 1];
      // triangle (i, j, k) appears as (j, k, i) around j and as (k, i, j) around k
      int bj = find_pair_t(g, j, k, okx - ojx, oky - ojy, i, -ojx, -ojy);
      int bk = find_pair_t(g, k, i, -okx, -oky, j, ojx - okx, ojy - oky);
      if (bj < 0 || bk < 0) return -10;  // inconsistent rings
      T Gx = sx[ea] + sx[j * g.max_ring + bj] + sx[k * g.max_ring + bk];
      T Gy = sy[ea] + sy[j * g.max_ring + bj] + sy[k * g.max_ring + bk];
      // Jacobian dh/dr_i (Eqs. A8-A16, corrected)
      T rijx, rijy, rikx, riky;
      rel_t(g, i, a, rijx, rijy);
      rel_t(g, i, (a + 1) % m, rikx, riky);
      T rjkx = rikx - rijx, rjky = riky - rijy;
      T c = rijx * (-rjky) - rijy * (-rjkx);
      T d = 2.0 * c * c;
      T rij2 = rijx * rijx + rijy * rijy, rik2 = rikx * rikx + riky * riky;
      T ij_jk = rijx * rjkx + rijy * rjky, ik_jk = rikx * rjkx + riky * rjky;
      T betad = -rik2 * ij_jk, gammad = rij2 * ik_jk;
      T zx = betad * rijx + gammad * rikx, zy = betad * rijy + gammad * riky;
      T gbx = 2.0 * ij_jk * rikx + rik2 * rjkx, gby = 2.0 * ij_jk * riky + rik2 * rjky;
      T ggx = -2.0 * ik_jk * rijx - rij2 * rjkx, ggy = -2.0 * ik_jk * rijy - rij2 * rjky;
      T gdx = (2.0 / c) * rjky, gdy = (2.0 / c) * (-rjkx);
      T J[2][2];
      const T rv[2] = {rijx, rijy}, kv[2] = {rikx, riky}, zv[2] = {zx, zy};
      const T gb[2] = {gbx, gby}, gg[2] = {ggx, ggy}, gd[2] = {gdx, gdy};
      for (int al = 0; al < 2; ++al)
        for (int be = 0; be < 2; ++be) {
          T diag = (al == be) ? betad + gammad : T(0.0);
          J[al][be] = (al == be ? 1.0 : 0.0) + (rv[al] * gb[be] + kv[al] * gg[be] - diag - zv[al] * gd[be]) / d;
        }
      fx = fx - (J[0][0] * Gx + J[1][0] * Gy);
      fy = fy - (J[0][1] * Gx + J[1][1] * Gy);
    }
    Fx[i] = fx;
    Fy[i] = fy;
  }
  return 0;
}

}  // namespace cgo
