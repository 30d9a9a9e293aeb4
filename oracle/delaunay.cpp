// Oracle: Delaunay triangulation by Bowyer-Watson insertion. TEST
// INFRASTRUCTURE ONLY.
//
// The SPV model's cell shapes are the Voronoi cells of the cell positions,
// i.e. the duals of the Delaunay triangulation (paper Sec. 2.A and Fig. 1).
// This file builds that triangulation from scratch by inserting points one by
// one into a super-triangle: the triangles whose circumcircle contains the
// new point (the "cavity") are removed and the cavity is re-triangulated as a
// fan around the new point.  Every orientation and in-circle decision is exact
// (exact.cpp), so the result is the unique Delaunay triangulation of the
// symbolically perturbed point set.
#include "internal.h"
#include <algorithm>
#include <cstdio>
#include <limits>

namespace cgo {

namespace {

struct Tri {
  int v[3];   // CCW vertex indices; v[0] == -1 marks a dead slot
  int nb[3];  // triangle across the edge opposite v[k]; -1 if none
};

// Morton (Z-order) key of a point: only used to pick a spatially coherent
// insertion order so that point-location walks stay short.
uint64_t morton(uint32_t x, uint32_t y) {
  uint64_t r = 0;
  for (int b = 0; b < 32; ++b) {
    r |= (uint64_t)((x >> b) & 1u) << (2 * b);
    r |= (uint64_t)((y >> b) & 1u) << (2 * b + 1);
  }
  return r;
}

}  // namespace

int bowyer_watson_rings(const std::vector<Pt>& pts_in, const std::vector<char>& central,
                        std::vector<Ring>& rings_out, bool allow_open) {
  const int M = (int)pts_in.size();
  std::vector<Pt> P(pts_in);
  if (M == 0) return 0;

  int64_t minX = P[0].X, maxX = P[0].X, minY = P[0].Y, maxY = P[0].Y;
  for (const Pt& p : P) {
    minX = std::min(minX, p.X); maxX = std::max(maxX, p.X);
    minY = std::min(minY, p.Y); maxY = std::max(maxY, p.Y);
  }
  int64_t span = std::max(maxX - minX, maxY - minY) + 1;
  // Super-triangle with legs 16*span: contains the bounding box strictly.
  const int64_t kMax = std::numeric_limits<int64_t>::max();
  Pt sa{minX - 4 * span, minY - 4 * span, -1, 0, 0, kMax - 2};
  Pt sb{minX + 12 * span, minY - 4 * span, -1, 0, 0, kMax - 1};
  Pt sc{minX - 4 * span, minY + 12 * span, -1, 0, 0, kMax};
  P.push_back(sa); P.push_back(sb); P.push_back(sc);

  std::vector<Tri> T;
  T.reserve((size_t)2 * M + 64);
  std::vector<int> free_slots;
  T.push_back(Tri{{M, M + 1, M + 2}, {-1, -1, -1}});

  // insertion order
  std::vector<std::pair<uint64_t, int>> order(M);
  for (int i = 0; i < M; ++i) {
    uint32_t ux = (uint32_t)((P[i].X - minX) >> 24);
    uint32_t uy = (uint32_t)((P[i].Y - minY) >> 24);
    order[i] = {morton(ux, uy), i};
  }
  std::sort(order.begin(), order.end());

  std::vector<int> visit, inconf;
  std::vector<int> start_tri(M + 3, -1), end_tri(M + 3, -1);
  std::vector<int> cavity, stack;
  struct Edge { int a, b, out, old; };
  std::vector<Edge> boundary;
  int stamp = 0;
  int last = 0;
  uint32_t rng = 12345u;

  auto alloc = [&]() -> int {
    if (!free_slots.empty()) { int t = free_slots.back(); free_slots.pop_back(); return t; }
    T.push_back(Tri{{-1, -1, -1}, {-1, -1, -1}});
    return (int)T.size() - 1;
  };

  for (int oi = 0; oi < M; ++oi) {
    const int pi = order[oi].second;
    const Pt& p = P[pi];

    // --- point location: stochastic visibility walk, linear scan fallback
    int t = last;
    bool found = false;
    for (long iter = 0; iter < 4000000L; ++iter) {
      rng = rng * 1664525u + 1013904223u;
      int k0 = (int)((rng >> 16) % 3u);
      int next = -1;
      for (int m = 0; m < 3; ++m) {
        int k = (k0 + m) % 3;
        int a = T[t].v[(k + 1) % 3], b = T[t].v[(k + 2) % 3];
        if (orient2d_exact(P[a], P[b], p) < 0) { next = T[t].nb[k]; break; }
      }
      if (next < 0) { found = true; break; }
      t = next;
    }
    if (!found) {
      for (t = 0; t < (int)T.size(); ++t) {
        if (T[t].v[0] < 0) continue;
        bool in = true;
        for (int k = 0; k < 3 && in; ++k)
          in = orient2d_exact(P[T[t].v[(k + 1) % 3]], P[T[t].v[(k + 2) % 3]], p) >= 0;
        if (in) { found = true; break; }
      }
      if (!found) return -2;
    }
    for (int k = 0; k < 3; ++k) {
      const Pt& q = P[T[t].v[k]];
      if (q.X == p.X && q.Y == p.Y) return -1;  // duplicate point
    }

    // --- cavity: all triangles whose (perturbed) circumcircle contains p.
    // t contains p in its closed interior, so p is strictly inside its circle.
    ++stamp;
    if (visit.size() < T.size()) { visit.resize(T.size() * 2, 0); inconf.resize(T.size() * 2, 0); }
    cavity.clear(); stack.clear(); boundary.clear();
    visit[t] = stamp; inconf[t] = 1;
    stack.push_back(t);
    while (!stack.empty()) {
      int c = stack.back(); stack.pop_back();
      cavity.push_back(c);
      for (int k = 0; k < 3; ++k) {
        int nb = T[c].nb[k];
        if (nb < 0 || visit[nb] == stamp) continue;
        visit[nb] = stamp;
        const Tri& o = T[nb];
        int s = incircle_sos(P[o.v[0]], P[o.v[1]], P[o.v[2]], p);
        inconf[nb] = s > 0;
        if (s > 0) stack.push_back(nb);
      }
    }
    for (int c : cavity) {
      for (int k = 0; k < 3; ++k) {
        int nb = T[c].nb[k];
        if (nb >= 0 && visit[nb] == stamp && inconf[nb]) continue;
        boundary.push_back(Edge{T[c].v[(k + 1) % 3], T[c].v[(k + 2) % 3], nb, c});
      }
    }
    // --- re-triangulate the cavity as a fan around p.  Cavity slots are
    // released only after the outside neighbours have been re-pointed, so a
    // reused slot id can never be mistaken for one of the removed triangles.
    std::vector<int> created;
    created.reserve(boundary.size());
    for (const Edge& e : boundary) {
      int nt = alloc();
      T[nt] = Tri{{pi, e.a, e.b}, {e.out, -1, -1}};
      if (e.out >= 0) {
        for (int k = 0; k < 3; ++k)
          if (T[e.out].nb[k] == e.old) { T[e.out].nb[k] = nt; break; }
      }
      start_tri[e.a] = nt;
      end_tri[e.b] = nt;
      created.push_back(nt);
    }
    for (int nt : created) {
      int a = T[nt].v[1], b = T[nt].v[2];
      T[nt].nb[1] = start_tri[b];  // edge (b, p)
      T[nt].nb[2] = end_tri[a];    // edge (p, a)
    }
    for (int c : cavity) { T[c].v[0] = -1; free_slots.push_back(c); }
    last = created.empty() ? 0 : created[0];
    if (visit.size() < T.size()) { visit.resize(T.size() * 2, 0); inconf.resize(T.size() * 2, 0); }
  }

  // --- rings of central points: CCW cycle of (u -> w) over incident triangles
  rings_out.assign(M, Ring());
  std::vector<std::vector<std::pair<int, int>>> fan(M);
  for (const Tri& tr : T) {
    if (tr.v[0] < 0) continue;
    if (tr.v[0] >= M || tr.v[1] >= M || tr.v[2] >= M) continue;
    for (int k = 0; k < 3; ++k) {
      int c = tr.v[k];
      if (central[c]) fan[c].push_back({tr.v[(k + 1) % 3], tr.v[(k + 2) % 3]});
    }
  }
  for (int c = 0; c < M; ++c) {
    if (!central[c]) continue;
    auto& f = fan[c];
    if (allow_open) {
      // hull points of a plain point set have an open fan: leave their ring empty
      std::vector<int> us, ws;
      for (auto& e : f) { us.push_back(e.first); ws.push_back(e.second); }
      std::sort(us.begin(), us.end());
      std::sort(ws.begin(), ws.end());
      if (f.size() < 3 || us != ws) continue;
    }
    if (f.size() < 3) return -3;
    std::sort(f.begin(), f.end());
    // successor lookup by binary search on u
    std::vector<int> cyc;
    int u0 = f[0].first, u = u0;
    for (size_t step = 0; step <= f.size(); ++step) {
      cyc.push_back(u);
      auto it = std::lower_bound(f.begin(), f.end(), std::make_pair(u, std::numeric_limits<int>::min()));
      if (it == f.end() || it->first != u) return -3;
      u = it->second;
      if (u == u0) break;
    }
    if (u != u0 || cyc.size() != f.size()) return -3;
    // canonical start: smallest neighbour tag
    size_t best = 0;
    for (size_t m = 1; m < cyc.size(); ++m)
      if (P[cyc[m]].tag < P[cyc[best]].tag) best = m;
    Ring& r = rings_out[c];
    for (size_t m = 0; m < cyc.size(); ++m) {
      const Pt& q = P[cyc[(best + m) % cyc.size()]];
      r.tag.push_back(q.tag);
      r.ox.push_back(q.ox - P[c].ox);
      r.oy.push_back(q.oy - P[c].oy);
    }
    for (size_t m = 0; m < r.tag.size(); ++m)
      for (size_t m2 = m + 1; m2 < r.tag.size(); ++m2)
        if (r.tag[m] == r.tag[m2]) return -4;  // two images of one cell: box too small
  }
  return 0;
}

}  // namespace cgo
