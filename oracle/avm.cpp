// Oracle: active vertex model (AVM). TEST INFRASTRUCTURE ONLY.
//
// Sussman, arXiv 1702.02939, Sec. 2.D and Eq. 4:
//  * degrees of freedom: the vertices h_v of a degree-3 network (2N vertices
//    for N cells); here the initial network is the Voronoi tessellation of
//    cell seed positions (the circumcentres of the Delaunay triangles);
//  * energy of Eq. 1 from the polygon areas and perimeters;
//  * vertex force F_v = -(dE_i + dE_j + dE_k)/dh_v over the vertex's three
//    cells (Eq. A2) with dA/dh, dP/dh of Eqs. A4, A5 (A5 corrected);
//  * motion dh_v/dt = mu F_v + (v0 / 3) sum_{cells c of v} n(theta_c) (Eq. 4, n = 3),
//    then the directors rotate (a separate update, Sec. 2.D);
//  * T1 transitions (Fig. 1): an edge shorter than a threshold is rotated by
//    90 degrees about its midpoint and the neighbours are exchanged; at most
//    one transition per cell per pass, passes repeated until none is called
//    for (Sec. 2.D);
//  * T2 transitions (cell removal, named in Sec. 2.A; the paper's code has
//    only T1s): a triangular cell whose area is below a threshold is removed
//    and its three vertices merge into one at their centroid; per-cell
//    preferred areas A0_c (a dying cell gets a small A0_c) drive the cell
//    down to it.
// Conventions (shared definitions with the library, each written separately):
//  * vertex v stores its cells (c0, c1, c2) counter-clockwise around it and
//    its neighbours (n0, n1, n2), where the edge v-n_k separates c_k and c_{k+1};
//  * cell vertex lists are counter-clockwise;
//  * vertex ids: the Delaunay triangles of each cell o whose smallest cell is
//    o, in o's ring order, numbered consecutively in increasing o;
//  * T1 candidates: edges (v, n_s) with v < n_s and squared length below the
//    squared threshold (products and sums rounded separately, no fused
//    multiply-add); edge id = 3 v + s; for the edge, i = c_s, k = c_{s+1}
//    (the cells that share it), j = c_{s+2}, l = the third cell of n_s;
//    a transition needs |i|, |k| > 3 vertices and |j|, |l| < 16;
//    a candidate applies in a pass when its edge id is the smallest among the
//    candidates touching each of i, j, k, l;
//  * the rotated edge gets length 1.5 x threshold; v becomes the endpoint on
//    cell i's side (cells j, i, l; neighbours A_ll, A_lr, n_s), n_s the one
//    on cell k's side (cells k, j, l; neighbours A_ul, v, A_ur);
//  * T2 candidates: cells c with exactly 3 vertices (v0, v1, v2 = its list)
//    and d < 2 x threshold_T2, d = px1 py2 - px2 py1 (each product and the
//    difference rounded separately; p = minimum-image offsets from v0), id
//    3V + c; its cells are c and the three cells across its edges, which must
//    be distinct with more than 3 vertices each; the three outer vertices
//    must be distinct; the same lock rule as T1 (smallest id among the
//    candidates touching each cell);
//  * a T2 keeps the smallest of the three vertex ids at the centroid
//    v0 + (p1 + p2)/3 (wrapped); the other two become free (vc, vn = -1),
//    the cell is emptied (cc = 0, cv = -1); around the kept vertex the
//    outer edges keep their order; each neighbour cell loses one vertex;
//  * free vertices and empty cells take no part in forces, moves or
//    transitions (their positions stay); P0_c = p0_c sqrt(A0_c);
//  * division of cell c along direction u (cell division, named in Sec. 2.A
//    as a feature of vertex models; the paper's code has none): with p the
//    minimum-image offsets of its vertices from its first vertex, m their
//    mean (sum in list order, then / count), q = p - m and s_a = u x q_a, an
//    edge a -> a+1 is cut where s changes sign (s > 0 against s <= 0) at
//    X = q_a + t (q_{a+1} - q_a), t = s_a / (s_a - s_{a+1}) clamped to
//    [1/16, 15/16]; of the cuts, the one with the smallest u.X > 0 (new
//    vertex A, edge a1) and the one with the largest u.X < 0 (new vertex B,
//    edge a2) are taken (every product, sum and quotient rounded on its own);
//    c keeps A, v_{a1+1} .. v_{a2}, B and the new cell B, v_{a2+1} ..
//    v_{a1}, A (the lowest empty cell slot; A, B the two lowest free vertex
//    slots); the cells across the cut edges gain A and B; the new cell
//    copies c's director, p0, v0 and A0.  Refused (no change) when a cut is
//    missing, a daughter would exceed 16 vertices or a neighbour could not
//    take the new vertex.
#include "internal.h"

#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

extern "C" int cgo_triangulate(int n, double Lx, double Ly, const double* x, const double* y, int max_ring,
                               int32_t* cnt, int32_t* nbr, int32_t* off);
extern "C" double cgo_director_noise(uint64_t seed, int32_t tag, int64_t step);

namespace cgo {
namespace {

constexpr int kR = 16;

inline double mimg(double d, double L) {
  if (d > 0.5 * L) d -= L;
  else if (d < -0.5 * L) d += L;
  return d;
}
inline double wrapL(double v, double L) {
  double r = std::fmod(v, L);
  if (r < 0.0) r += L;
  if (r >= L) r -= L;
  return r + 0.0;
}

struct Net {
  int N, V;
  double Lx, Ly;
  double* hx;
  double* hy;
  int32_t *vc, *vn, *cc, *cv;
};

inline bool vertex_free(const Net& g, int v) { return g.vc[3 * v] < 0; }

// Squared edge length, every product and sum rounded on its own.
double edge_len2(const Net& g, int v, int w) {
  volatile double dx = mimg(g.hx[w] - g.hx[v], g.Lx);
  volatile double dy = mimg(g.hy[w] - g.hy[v], g.Ly);
  volatile double a = dx * dx;
  volatile double b = dy * dy;
  return a + b;
}

void polygon_geometry(const Net& g, int c, double& A, double& P) {
  int m = g.cc[c];
  if (m == 0) {  // removed by a T2
    A = P = 0.0;
    return;
  }
  int v0 = g.cv[c * kR];
  std::vector<double> px(m), py(m);
  for (int a = 0; a < m; ++a) {
    int v = g.cv[c * kR + a];
    px[a] = mimg(g.hx[v] - g.hx[v0], g.Lx);
    py[a] = mimg(g.hy[v] - g.hy[v0], g.Ly);
  }
  double area = 0.0, per = 0.0;
  for (int a = 0; a < m; ++a) {
    int b = (a + 1) % m;
    area += px[a] * py[b] - px[b] * py[a];
    per += std::sqrt((px[b] - px[a]) * (px[b] - px[a]) + (py[b] - py[a]) * (py[b] - py[a]));
  }
  A = 0.5 * area;
  P = per;
}

// F_v = -sum_c dE_c/dh_v, accumulated cell by cell over each cell's vertex list.
void vertex_forces(const Net& g, const double* p0, const double* a0, double KA, double KP, double* Fx,
                   double* Fy, double* A, double* P, double* energy) {
  double E = 0.0;
  for (int v = 0; v < g.V; ++v) Fx[v] = Fy[v] = 0.0;
  for (int c = 0; c < g.N; ++c) {
    polygon_geometry(g, c, A[c], P[c]);
    int m = g.cc[c];
    if (m == 0) continue;
    const double A0 = a0[c], P0 = p0[c] * std::sqrt(A0);
    E += KA * (A[c] - A0) * (A[c] - A0) + KP * (P[c] - P0) * (P[c] - P0);
    double ka = 2.0 * KA * (A[c] - A0), kp = 2.0 * KP * (P[c] - P0);
    for (int a = 0; a < m; ++a) {
      int vp = g.cv[c * kR + (a + m - 1) % m], v = g.cv[c * kR + a], vn = g.cv[c * kR + (a + 1) % m];
      double tinx = mimg(g.hx[v] - g.hx[vp], g.Lx), tiny = mimg(g.hy[v] - g.hy[vp], g.Ly);    // t_ij
      double toutx = mimg(g.hx[vn] - g.hx[v], g.Lx), touty = mimg(g.hy[vn] - g.hy[v], g.Ly);  // t_ik
      // Eq. A4 with outward normals l n = (t_y, -t_x); Eq. A5 (corrected)
      double dAx = 0.5 * (tiny + touty), dAy = 0.5 * (-tinx - toutx);
      double lin = std::sqrt(tinx * tinx + tiny * tiny), lout = std::sqrt(toutx * toutx + touty * touty);
      double dPx = tinx / lin - toutx / lout, dPy = tiny / lin - touty / lout;
      Fx[v] -= ka * dAx + kp * dPx;
      Fy[v] -= ka * dAy + kp * dPy;
    }
  }
  if (energy) *energy = E;
}

int slot_of(const int32_t* arr, int v, int val) {
  for (int s = 0; s < 3; ++s)
    if (arr[3 * v + s] == val) return s;
  return -1;
}

void remove_vertex(Net& g, int c, int v) {
  int m = g.cc[c], w = 0;
  for (int a = 0; a < m; ++a)
    if (g.cv[c * kR + a] != v) g.cv[c * kR + w++] = g.cv[c * kR + a];
  for (int a = w; a < kR; ++a) g.cv[c * kR + a] = -1;
  g.cc[c] = w;
}

void insert_after(Net& g, int c, int after, int v) {
  int m = g.cc[c];
  int pos = -1;
  for (int a = 0; a < m; ++a)
    if (g.cv[c * kR + a] == after) pos = a;
  for (int a = m; a > pos + 1; --a) g.cv[c * kR + a] = g.cv[c * kR + a - 1];
  g.cv[c * kR + pos + 1] = v;
  g.cc[c] = m + 1;
}

struct Cand {
  int v, s, w, i, j, k, l, id;
};

// A T2 candidate: the triangular cell c, its vertices v[3] (its list), the
// cells nb[a] across its edges (v[a], v[a+1]), the outer vertices w[a] of
// v[a] and the cells cp[a], cpp[a] on either side of the edge v[a] - w[a]
// (counter-clockwise around v[a]).
struct T2Cand {
  int c, id;
  int v[3], nb[3], w[3], cp[3], cpp[3];
};

// The T2 area test: twice the signed area of the triangle, each product and
// the difference rounded separately, below twice the threshold.
bool t2_small(const Net& g, int c, double t2_area) {
  const int v0 = g.cv[c * kR], v1 = g.cv[c * kR + 1], v2 = g.cv[c * kR + 2];
  volatile double px1 = mimg(g.hx[v1] - g.hx[v0], g.Lx), py1 = mimg(g.hy[v1] - g.hy[v0], g.Ly);
  volatile double px2 = mimg(g.hx[v2] - g.hx[v0], g.Lx), py2 = mimg(g.hy[v2] - g.hy[v0], g.Ly);
  volatile double a = px1 * py2;
  volatile double b = px2 * py1;
  volatile double d = a - b;
  return d < 2.0 * t2_area;
}

// Cell other than c that has both vertices va and vb, or -1.
int across(const Net& g, int c, int va, int vb) {
  for (int s = 0; s < 3; ++s) {
    const int x = g.vc[3 * va + s];
    if (x != c && x >= 0 && (x == g.vc[3 * vb] || x == g.vc[3 * vb + 1] || x == g.vc[3 * vb + 2])) return x;
  }
  return -1;
}

// Fills a T2 candidate for the triangular cell c; false when the removal is
// not allowed (a neighbour with 3 vertices, neighbours or outer vertices not
// distinct); -1 in *broken for an inconsistent network.
bool t2_candidate(const Net& g, int c, T2Cand& t, int* broken) {
  t.c = c;
  t.id = 3 * g.V + c;
  for (int a = 0; a < 3; ++a) t.v[a] = g.cv[c * kR + a];
  for (int a = 0; a < 3; ++a) {
    const int va = t.v[a];
    const int s = slot_of(g.vc, va, c);
    if (s < 0) {
      *broken = 1;
      return false;
    }
    t.w[a] = g.vn[3 * va + (s + 1) % 3];
    t.cp[a] = g.vc[3 * va + (s + 1) % 3];
    t.cpp[a] = g.vc[3 * va + (s + 2) % 3];
    t.nb[a] = across(g, c, va, t.v[(a + 1) % 3]);
    if (t.nb[a] < 0) {
      *broken = 1;
      return false;
    }
  }
  for (int a = 0; a < 3; ++a) {
    if (g.cc[t.nb[a]] <= 3) return false;
    for (int b2 = a + 1; b2 < 3; ++b2)
      if (t.nb[a] == t.nb[b2] || t.w[a] == t.w[b2]) return false;
    for (int b2 = 0; b2 < 3; ++b2)
      if (t.w[a] == t.v[b2]) return false;
  }
  return true;
}

// Replaces v0, v1, v2 by vk in cell x's list and drops the repeat this makes
// (the cell shared one edge with the removed triangle).
void merge_in_cell(Net& g, int x, const int* v, int vk) {
  const int m = g.cc[x];
  std::vector<int> out;
  for (int a = 0; a < m; ++a) {
    int e = g.cv[x * kR + a];
    if (e == v[0] || e == v[1] || e == v[2]) e = vk;
    if (!out.empty() && e == vk && out.back() == vk) continue;
    out.push_back(e);
  }
  if (out.size() > 1 && out.front() == vk && out.back() == vk) out.pop_back();
  for (int a = 0; a < kR; ++a) g.cv[x * kR + a] = a < (int)out.size() ? out[a] : -1;
  g.cc[x] = (int)out.size();
}

// Applies a T2; -1 on an inconsistent network.
int apply_t2(Net& g, const T2Cand& t) {
  const int vk = std::min(t.v[0], std::min(t.v[1], t.v[2]));
  // centroid relative to the first vertex of the list
  const int u0 = t.v[0], u1 = t.v[1], u2 = t.v[2];
  const double dx1 = mimg(g.hx[u1] - g.hx[u0], g.Lx), dy1 = mimg(g.hy[u1] - g.hy[u0], g.Ly);
  const double dx2 = mimg(g.hx[u2] - g.hx[u0], g.Lx), dy2 = mimg(g.hy[u2] - g.hy[u0], g.Ly);
  const double cx = wrapL(g.hx[u0] + (dx1 + dx2) / 3.0, g.Lx);
  const double cy = wrapL(g.hy[u0] + (dy1 + dy2) / 3.0, g.Ly);
  // the kept vertex: outer edges in the order a0 = 0, then the one whose
  // first cell is the previous edge's second cell
  int ord[3] = {0, -1, -1};
  for (int q = 1; q < 3; ++q)
    for (int a = 0; a < 3; ++a)
      if (t.cp[a] == t.cpp[ord[q - 1]] && a != ord[0] && (q < 2 || a != ord[1])) ord[q] = a;
  if (ord[1] < 0 || ord[2] < 0 || t.cpp[ord[2]] != t.cp[ord[0]]) return -1;
  for (int a = 0; a < 3; ++a) {
    const int s = slot_of(g.vn, t.w[a], t.v[a]);
    if (s < 0) return -1;
    g.vn[3 * t.w[a] + s] = vk;
  }
  for (int a = 0; a < 3; ++a) merge_in_cell(g, t.nb[a], t.v, vk);
  for (int q = 0; q < 3; ++q) {
    g.vc[3 * vk + q] = t.cp[ord[q]];
    g.vn[3 * vk + q] = t.w[ord[q]];
  }
  g.hx[vk] = cx;
  g.hy[vk] = cy;
  for (int a = 0; a < 3; ++a) {
    if (t.v[a] == vk) continue;
    for (int q = 0; q < 3; ++q) g.vc[3 * t.v[a] + q] = g.vn[3 * t.v[a] + q] = -1;
  }
  for (int a = 0; a < kR; ++a) g.cv[t.c * kR + a] = -1;
  g.cc[t.c] = 0;
  return 0;
}

// One pass of topological transitions (T1 and, with t2_area > 0, T2);
// returns the number applied (T1s in *n_t1, T2s in *n_t2) or -1 on a broken
// network; *remaining = candidates proposed.
int topo_pass(Net& g, double thr, double newlen, double t2_area, int* remaining, int* n_t1, int* n_t2) {
  std::vector<Cand> cands;
  std::vector<T2Cand> t2s;
  const double thr2 = thr * thr;
  for (int v = 0; v < g.V; ++v) {
    if (vertex_free(g, v)) continue;
    for (int s = 0; s < 3; ++s) {
      int w = g.vn[3 * v + s];
      if (w <= v) continue;
      if (!(edge_len2(g, v, w) < thr2)) continue;
      int i = g.vc[3 * v + s], k = g.vc[3 * v + (s + 1) % 3], j = g.vc[3 * v + (s + 2) % 3];
      int l = -1;
      for (int t = 0; t < 3; ++t) {
        int c = g.vc[3 * w + t];
        if (c != i && c != k) l = c;
      }
      if (l < 0) return -1;
      if (g.cc[i] <= 3 || g.cc[k] <= 3 || g.cc[j] >= kR || g.cc[l] >= kR) continue;
      cands.push_back(Cand{v, s, w, i, j, k, l, 3 * v + s});
    }
  }
  if (t2_area > 0.0) {
    for (int c = 0; c < g.N; ++c) {
      if (g.cc[c] != 3 || !t2_small(g, c, t2_area)) continue;
      T2Cand t;
      int broken = 0;
      if (t2_candidate(g, c, t, &broken)) t2s.push_back(t);
      if (broken) return -1;
    }
  }
  *remaining = (int)(cands.size() + t2s.size());
  *n_t1 = *n_t2 = 0;
  if (*remaining == 0) return 0;
  std::vector<int> lock(g.N, INT_MAX);
  for (const Cand& c : cands)
    for (int cell : {c.i, c.j, c.k, c.l}) lock[cell] = std::min(lock[cell], c.id);
  for (const T2Cand& t : t2s)
    for (int cell : {t.c, t.nb[0], t.nb[1], t.nb[2]}) lock[cell] = std::min(lock[cell], t.id);
  int applied = 0;
  for (const Cand& c : cands) {
    if (lock[c.i] != c.id || lock[c.j] != c.id || lock[c.k] != c.id || lock[c.l] != c.id) continue;
    const int v1 = c.v, v2 = c.w, a = c.s;
    const int Aul = g.vn[3 * v1 + (a + 1) % 3], All = g.vn[3 * v1 + (a + 2) % 3];
    const int b = slot_of(g.vn, v2, v1);
    if (b < 0 || g.vc[3 * v2 + b] != c.k || g.vc[3 * v2 + (b + 1) % 3] != c.i) return -1;
    const int Alr = g.vn[3 * v2 + (b + 1) % 3], Aur = g.vn[3 * v2 + (b + 2) % 3];
    // geometry: rotate the edge by 90 degrees about its midpoint
    double ex = mimg(g.hx[v2] - g.hx[v1], g.Lx), ey = mimg(g.hy[v2] - g.hy[v1], g.Ly);
    double mx = g.hx[v1] + 0.5 * ex, my = g.hy[v1] + 0.5 * ey;
    double len = std::sqrt(ex * ex + ey * ey);
    double px = -ey / len * 0.5 * newlen, py = ex / len * 0.5 * newlen;
    g.hx[v1] = wrapL(mx - px, g.Lx);
    g.hy[v1] = wrapL(my - py, g.Ly);
    g.hx[v2] = wrapL(mx + px, g.Lx);
    g.hy[v2] = wrapL(my + py, g.Ly);
    // topology
    int* c1 = g.vc + 3 * v1;
    int* n1 = g.vn + 3 * v1;
    int* c2 = g.vc + 3 * v2;
    int* n2 = g.vn + 3 * v2;
    c1[0] = c.j; c1[1] = c.i; c1[2] = c.l;
    n1[0] = All; n1[1] = Alr; n1[2] = v2;
    c2[0] = c.k; c2[1] = c.j; c2[2] = c.l;
    n2[0] = Aul; n2[1] = v1; n2[2] = Aur;
    int su = slot_of(g.vn, Aul, v1);
    int sl = slot_of(g.vn, Alr, v2);
    if (su < 0 || sl < 0) return -1;
    g.vn[3 * Aul + su] = v2;
    g.vn[3 * Alr + sl] = v1;
    remove_vertex(g, c.i, v2);
    remove_vertex(g, c.k, v1);
    insert_after(g, c.j, v1, v2);
    insert_after(g, c.l, v2, v1);
    ++applied;
    ++*n_t1;
  }
  for (const T2Cand& t : t2s) {
    if (lock[t.c] != t.id || lock[t.nb[0]] != t.id || lock[t.nb[1]] != t.id || lock[t.nb[2]] != t.id) continue;
    if (apply_t2(g, t) < 0) return -1;
    ++applied;
    ++*n_t2;
  }
  return applied;
}

// Division of cell c along (ux, uy) into c and newc, new vertices va (A) and
// vb (B); per-cell arrays copied to newc.  0 made, 1 refused, -1 broken.
int divide_cell(Net& g, int c, double ux, double uy, int newc, int va, int vb, double* theta, double* p0,
                double* v0, double* a0) {
  const int m = g.cc[c];
  if (m < 3) return 1;
  std::vector<int> v(m);
  for (int a = 0; a < m; ++a) v[a] = g.cv[c * kR + a];
  std::vector<double> qx(m), qy(m), sd(m);
  volatile double sx = 0.0, sy = 0.0;
  std::vector<double> px(m), py(m);
  for (int a = 0; a < m; ++a) {
    px[a] = mimg(g.hx[v[a]] - g.hx[v[0]], g.Lx);
    py[a] = mimg(g.hy[v[a]] - g.hy[v[0]], g.Ly);
  }
  for (int a = 1; a < m; ++a) {
    sx = sx + px[a];
    sy = sy + py[a];
  }
  const double mx = sx / (double)m, my = sy / (double)m;
  for (int a = 0; a < m; ++a) {
    qx[a] = px[a] - mx;
    qy[a] = py[a] - my;
    volatile double t1 = ux * qy[a];
    volatile double t2 = uy * qx[a];
    sd[a] = t1 - t2;
  }
  int a1 = -1, a2 = -1;
  double l1 = 0.0, l2 = 0.0, X1x = 0.0, X1y = 0.0, X2x = 0.0, X2y = 0.0;
  for (int a = 0; a < m; ++a) {
    const int b = (a + 1) % m;
    if ((sd[a] > 0.0) == (sd[b] > 0.0)) continue;
    volatile double den = sd[a] - sd[b];
    double t = sd[a] / den;
    if (t < 0.0625) t = 0.0625;
    if (t > 0.9375) t = 0.9375;
    volatile double dx = qx[b] - qx[a], dy = qy[b] - qy[a];
    volatile double tx = t * dx, ty = t * dy;
    volatile double Xx = qx[a] + tx, Xy = qy[a] + ty;
    volatile double lx = ux * Xx, ly = uy * Xy;
    const double lam = lx + ly;
    if (lam > 0.0 && (a1 < 0 || lam < l1)) { a1 = a; l1 = lam; X1x = Xx; X1y = Xy; }
    if (lam < 0.0 && (a2 < 0 || lam > l2)) { a2 = a; l2 = lam; X2x = Xx; X2y = Xy; }
  }
  if (a1 < 0 || a2 < 0) return 1;
  const int n1 = (a2 - a1 + m) % m + 2, n2 = (a1 - a2 + m) % m + 2;
  if (n1 > kR || n2 > kR) return 1;
  const int p1 = v[a1], p1n = v[(a1 + 1) % m], p2 = v[a2], p2n = v[(a2 + 1) % m];
  int x1 = -1, x2 = -1;
  for (int s = 0; s < 3; ++s) {
    const int y1 = g.vc[3 * p1 + s], y2 = g.vc[3 * p2 + s];
    if (y1 != c && (y1 == g.vc[3 * p1n] || y1 == g.vc[3 * p1n + 1] || y1 == g.vc[3 * p1n + 2])) x1 = y1;
    if (y2 != c && (y2 == g.vc[3 * p2n] || y2 == g.vc[3 * p2n + 1] || y2 == g.vc[3 * p2n + 2])) x2 = y2;
  }
  if (x1 < 0 || x2 < 0) return -1;
  if (g.cc[x1] + (x1 == x2 ? 2 : 1) > kR) return 1;
  if (x1 != x2 && g.cc[x2] + 1 > kR) return 1;
  // positions
  volatile double ax = mx + X1x, ay = my + X1y, bx = mx + X2x, by = my + X2y;
  const double x0 = g.hx[v[0]], y0 = g.hy[v[0]];
  // vertex neighbours along the cut edges
  const int s1 = slot_of(g.vn, p1, p1n), s1n = slot_of(g.vn, p1n, p1);
  const int s2 = slot_of(g.vn, p2, p2n), s2n = slot_of(g.vn, p2n, p2);
  if (s1 < 0 || s1n < 0 || s2 < 0 || s2n < 0) return -1;
  g.vn[3 * p1 + s1] = va;
  g.vn[3 * p1n + s1n] = va;
  g.vn[3 * p2 + s2] = vb;
  g.vn[3 * p2n + s2n] = vb;
  // the vertices of the new cell move from c to newc
  std::vector<int> d1, d2;
  d1.push_back(va);
  for (int a = (a1 + 1) % m;; a = (a + 1) % m) {
    d1.push_back(v[a]);
    if (a == a2) break;
  }
  d1.push_back(vb);
  d2.push_back(vb);
  for (int a = (a2 + 1) % m;; a = (a + 1) % m) {
    d2.push_back(v[a]);
    const int s = slot_of(g.vc, v[a], c);
    if (s < 0) return -1;
    g.vc[3 * v[a] + s] = newc;
    if (a == a1) break;
  }
  d2.push_back(va);
  for (int a = 0; a < kR; ++a) {
    g.cv[c * kR + a] = a < (int)d1.size() ? d1[a] : -1;
    g.cv[newc * kR + a] = a < (int)d2.size() ? d2[a] : -1;
  }
  g.cc[c] = (int)d1.size();
  g.cc[newc] = (int)d2.size();
  insert_after(g, x1, p1n, va);
  insert_after(g, x2, p2n, vb);
  g.vc[3 * va] = x1; g.vc[3 * va + 1] = c; g.vc[3 * va + 2] = newc;
  g.vn[3 * va] = p1n; g.vn[3 * va + 1] = vb; g.vn[3 * va + 2] = p1;
  g.vc[3 * vb] = x2; g.vc[3 * vb + 1] = newc; g.vc[3 * vb + 2] = c;
  g.vn[3 * vb] = p2n; g.vn[3 * vb + 1] = va; g.vn[3 * vb + 2] = p2;
  g.hx[va] = wrapL(x0 + ax, g.Lx);
  g.hy[va] = wrapL(y0 + ay, g.Ly);
  g.hx[vb] = wrapL(x0 + bx, g.Lx);
  g.hy[vb] = wrapL(y0 + by, g.Ly);
  theta[newc] = theta[c];
  p0[newc] = p0[c];
  v0[newc] = v0[c];
  a0[newc] = a0[c];
  return 0;
}

}  // namespace
}  // namespace cgo

using namespace cgo;

extern "C" {

// Initial vertex network: the Voronoi tessellation of cell seed positions.
// Outputs: V = 2n vertices (hx, hy), vc/vn [V*3], cc [n], cv [n*16].
int cgo_avm_build(int n, double Lx, double Ly, const double* x, const double* y, double* hx, double* hy,
                  int32_t* vc, int32_t* vn, int32_t* cc, int32_t* cv) {
  std::vector<int32_t> cnt(n), nbr((size_t)n * kR), off((size_t)n * kR * 2);
  int rc = cgo_triangulate(n, Lx, Ly, x, y, kR, cnt.data(), nbr.data(), off.data());
  if (rc) return rc;
  // vertex id of (cell, slot): owner = smallest cell of the triangle
  std::vector<int> base(n + 1, 0);
  for (int o = 0; o < n; ++o) {
    int owned = 0;
    for (int b = 0; b < cnt[o]; ++b) {
      int j = nbr[o * kR + b], k = nbr[o * kR + (b + 1) % cnt[o]];
      owned += (o < j && o < k);
    }
    base[o + 1] = base[o] + owned;
  }
  if (base[n] != 2 * n) return -20;
  auto owned_rank = [&](int o, int b) {
    int r = 0;
    for (int t = 0; t < b; ++t) {
      int j = nbr[o * kR + t], k = nbr[o * kR + (t + 1) % cnt[o]];
      r += (o < j && o < k);
    }
    return r;
  };
  // find slot of the triangle (c, u, w) in c's ring: ring[b] = u, ring[b+1] = w
  auto slot_pair = [&](int c, int u, int w) {
    for (int b = 0; b < cnt[c]; ++b)
      if (nbr[c * kR + b] == u && nbr[c * kR + (b + 1) % cnt[c]] == w) return b;
    return -1;
  };
  auto vid = [&](int c, int a) {  // vertex of triangle (c, ring[a], ring[a+1])
    int j = nbr[c * kR + a], k = nbr[c * kR + (a + 1) % cnt[c]];
    if (c < j && c < k) return base[c] + owned_rank(c, a);
    int o, b;
    if (j < k) { o = j; b = slot_pair(j, k, c); }   // seen from j: (j, k, c)
    else { o = k; b = slot_pair(k, c, j); }         // seen from k: (k, c, j)
    if (b < 0) return -1;
    return base[o] + owned_rank(o, b);
  };
  for (int c = 0; c < n; ++c) {
    cc[c] = cnt[c];
    for (int a = 0; a < kR; ++a) cv[c * kR + a] = a < cnt[c] ? vid(c, a) : -1;
    for (int a = 0; a < cnt[c]; ++a)
      if (cv[c * kR + a] < 0) return -21;
  }
  for (int o = 0; o < n; ++o) {
    int m = cnt[o];
    for (int b = 0; b < m; ++b) {
      int j = nbr[o * kR + b], k = nbr[o * kR + (b + 1) % m];
      if (!(o < j && o < k)) continue;
      int v = base[o] + owned_rank(o, b);
      vc[3 * v + 0] = o; vc[3 * v + 1] = j; vc[3 * v + 2] = k;
      vn[3 * v + 0] = cv[o * kR + (b + m - 1) % m];                // across edge (o, j)
      int p = slot_pair(j, k, o);                                  // (j, k, o) in j's ring
      int mj = cnt[j];
      vn[3 * v + 1] = cv[j * kR + (p + mj - 1) % mj];              // across edge (j, k)
      vn[3 * v + 2] = cv[o * kR + (b + 1) % m];                    // across edge (k, o)
      // position: circumcentre of (o, j, k) with the periodic offsets of the ring
      double ax = (x[j] - x[o]) + off[(o * kR + b) * 2] * Lx, ay = (y[j] - y[o]) + off[(o * kR + b) * 2 + 1] * Ly;
      int b1 = (b + 1) % m;
      double bx = (x[k] - x[o]) + off[(o * kR + b1) * 2] * Lx, by = (y[k] - y[o]) + off[(o * kR + b1) * 2 + 1] * Ly;
      double d = 2.0 * (ax * by - ay * bx);
      double la = ax * ax + ay * ay, lb = bx * bx + by * by;
      hx[v] = wrapL(x[o] + (by * la - ay * lb) / d, Lx);
      hy[v] = wrapL(y[o] + (ax * lb - bx * la) / d, Ly);
    }
  }
  return 0;
}

int cgo_avm_forces(int n, int V, double Lx, double Ly, double* hx, double* hy, int32_t* vc, int32_t* vn,
                   int32_t* cc, int32_t* cv, const double* p0, const double* a0, const double* mech, double* Fx,
                   double* Fy, double* A, double* P, double* E) {
  Net g{n, V, Lx, Ly, hx, hy, vc, vn, cc, cv};
  vertex_forces(g, p0, a0, mech[0], mech[1], Fx, Fy, A, P, E);
  return 0;
}

// Transition passes (T1, and T2 when t2_area > 0) until a pass proposes no
// candidate (at most cap passes with transitions); applied[0] = T1s,
// applied[1] = T2s made.  Returns -8 when candidates remain after cap.
int cgo_avm_t1(int n, int V, double Lx, double Ly, double* hx, double* hy, int32_t* vc, int32_t* vn, int32_t* cc,
               int32_t* cv, double thr, double newlen, double t2_area, int cap, int32_t* applied) {
  Net g{n, V, Lx, Ly, hx, hy, vc, vn, cc, cv};
  int tot1 = 0, tot2 = 0;
  for (int r = 0; r <= cap; ++r) {
    int rem = 0, a1 = 0, a2 = 0;
    int a = (r < cap) ? topo_pass(g, thr, newlen, t2_area, &rem, &a1, &a2) : 0;
    if (r == cap) {  // count what is left without applying
      Net h = g;
      std::vector<double> sx(hx, hx + V), sy(hy, hy + V);
      std::vector<int32_t> svc(vc, vc + 3 * V), svn(vn, vn + 3 * V), scc(cc, cc + n), scv(cv, cv + n * kR);
      h.hx = sx.data(); h.hy = sy.data(); h.vc = svc.data(); h.vn = svn.data(); h.cc = scc.data(); h.cv = scv.data();
      topo_pass(h, thr, newlen, t2_area, &rem, &a1, &a2);
      applied[0] = tot1;
      applied[1] = tot2;
      return rem ? -8 : 0;
    }
    if (a < 0) return -22;
    tot1 += a1;
    tot2 += a2;
    if (rem == 0) break;
  }
  applied[0] = tot1;
  applied[1] = tot2;
  return 0;
}

// One AVM step: vertex move (Eq. 4), director rotation, transition passes.
// par = {KA, KP, mu, Dr, dt, thr, newlen, t2_area}; p0, v0, a0 per cell.
int cgo_avm_step(int n, int V, double Lx, double Ly, double* hx, double* hy, double* theta, int32_t* vc, int32_t* vn,
                 int32_t* cc, int32_t* cv, const double* p0, const double* v0, const double* a0, const double* par,
                 uint64_t seed, int64_t step, int cap, int32_t* applied) {
  Net g{n, V, Lx, Ly, hx, hy, vc, vn, cc, cv};
  std::vector<double> Fx(V), Fy(V), A(n), P(n);
  vertex_forces(g, p0, a0, par[0], par[1], Fx.data(), Fy.data(), A.data(), P.data(), nullptr);
  const double mu = par[2], Dr = par[3], dt = par[4];
  std::vector<double> nx(n), ny(n);
  for (int c = 0; c < n; ++c) {
    nx[c] = v0[c] * std::cos(theta[c]);
    ny[c] = v0[c] * std::sin(theta[c]);
  }
  for (int v = 0; v < V; ++v) {
    if (vertex_free(g, v)) continue;  // removed by a T2: stays where it is
    // Eq. 4 with n = 3 cells per vertex (per-cell speeds v0_c)
    double ax = (nx[vc[3 * v]] + nx[vc[3 * v + 1]] + nx[vc[3 * v + 2]]) / 3.0;
    double ay = (ny[vc[3 * v]] + ny[vc[3 * v + 1]] + ny[vc[3 * v + 2]]) / 3.0;
    hx[v] = wrapL(hx[v] + dt * (mu * Fx[v] + ax), Lx);
    hy[v] = wrapL(hy[v] + dt * (mu * Fy[v] + ay), Ly);
  }
  const double s = std::sqrt(2.0 * Dr * dt);
  for (int c = 0; c < n; ++c) theta[c] = theta[c] + s * cgo_director_noise(seed, c, step);
  return cgo_avm_t1(n, V, Lx, Ly, hx, hy, vc, vn, cc, cv, par[5], par[6], par[7], cap, applied);
}

// Divisions of cells[k] along dirs[2k], dirs[2k+1], in order; each one made
// takes the lowest empty cell slot (cc = 0) and the two lowest free vertex
// slots (vc = -1) left.  made[k] = 1 when division k was made.  Returns -22
// on a broken network, -1 when the slots run out.
int cgo_avm_divide(int n, int V, double Lx, double Ly, double* hx, double* hy, int32_t* vc, int32_t* vn,
                   int32_t* cc, int32_t* cv, double* theta, double* p0, double* v0, double* a0, int count,
                   const int32_t* cells, const double* dirs, int32_t* made) {
  Net g{n, V, Lx, Ly, hx, hy, vc, vn, cc, cv};
  int fc = 0, fv = 0;  // search cursors: a call only fills slots
  for (int k = 0; k < count; ++k) {
    made[k] = 0;
    while (fc < n && cc[fc] != 0) ++fc;
    while (fv < V && vc[3 * fv] >= 0) ++fv;
    int fv2 = fv + 1;
    while (fv2 < V && vc[3 * fv2] >= 0) ++fv2;
    if (fc >= n || fv2 >= V) return -1;
    const int r = divide_cell(g, cells[k], dirs[2 * k], dirs[2 * k + 1], fc, fv, fv2, theta, p0, v0, a0);
    if (r < 0) return -22;
    if (r == 0) made[k] = 1;
  }
  return 0;
}

}  // extern "C"
