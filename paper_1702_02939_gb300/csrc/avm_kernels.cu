// Active vertex model (AVM) kernels (Sussman, arXiv 1702.02939, Sec. 2.D,
// Eq. 4, Fig. 1).
//
// State: vertex positions (two buffers), per-vertex cells and neighbours
// (vc, vn: counter-clockwise, the edge v-vn[k] separates vc[k] and vc[k+1]),
// per-cell counter-clockwise vertex lists (cc, cv), directors theta.
// One step: polygon geometry per cell; vertex force and move per vertex
// (Eq. 4 with the activity averaged over the vertex's three cells); director
// rotation per cell; then T1 passes: edges shorter than the threshold propose
// a transition and take an atomic-min lock (edge id) on their four cells;
// an edge whose id holds all four locks rotates by 90 degrees about its
// midpoint and exchanges neighbours; passes repeat until none is proposed.
//
// Storage order: every vertex and cell slot carries a tag, its id in the
// network as built (the id the API speaks in).  Every rule that depends on
// ids takes tags: the T1 and T2 priorities, the end an edge is oriented from,
// the vertex a T2 keeps, the director noise counter and the slots divisions
// fill.  Results therefore do not depend on the storage order, which the
// Hilbert re-sort below changes (Sec. 2.B).
#include "cg_device.cuh"
#include "cg_kernels.h"

namespace cgk {

__device__ __forceinline__ double mimg_d(double d, double L) {
  if (d > 0.5 * L) d -= L;
  else if (d < -0.5 * L) d += L;
  return d;
}
// The same minimum image with the |d| > L/2 test on the integer pipe
// (non-negative doubles order like their bit patterns); the correction itself
// is rare.  Equal to mimg_d for every input.
__device__ __forceinline__ double mimg_a(double d, const Axis& a) {
  if (((unsigned long long)__double_as_longlong(d) & 0x7fffffffffffffffull) > a.half_bits)
    d = d > 0.0 ? d - a.L : d + a.L;
  return d;
}
__device__ __forceinline__ float mimg_f(float d, float L) {
  if (fabsf(d) > 0.5f * L) d = d > 0.0f ? d - L : d + L;
  return d;
}
__device__ __forceinline__ double wrap_d(double v, double L) {
  if (v >= 0.0 && v < L) return v;
  if (v >= L && v < 2.0 * L) return v - L;
  if (v < 0.0 && v >= -L) {
    const double r = v + L;
    return r >= L ? 0.0 : r;
  }
  double r = fmod(v, L);
  if (r < 0.0) r += L;
  return r >= L ? 0.0 : r;
}

// Reduction into [0, L) with the common case (already inside; +0 included)
// decided on the integer pipe.
__device__ __forceinline__ double wrap_a(double v, const Axis& a) {
  if ((unsigned long long)__double_as_longlong(v) < a.L_bits) return v;
  return wrap_d(v, a.L);
}

// ---------------------------------------------------------------------------
// Building the Voronoi network from a Delaunay triangulation (rings in user
// order).  Vertex ids: the triangles owned by each cell (its smallest cell),
// in ring order, numbered consecutively in increasing cell index.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool owns(const int* nbr, const int* cnt, int o, int b) {
  const int m = cnt[o];
  const int j = nbr[o * CG_RING + b], k = nbr[o * CG_RING + (b + 1) % m];
  return o < j && o < k;
}

__global__ void k_avm_count_owned(AvmBuildArgs g) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= g.n) return;
  int c = 0;
  for (int b = 0; b < g.cnt[o]; ++b) c += owns(g.nbr, g.cnt, o, b);
  g.owned[o] = c;
}

__device__ __forceinline__ int owned_rank(const AvmBuildArgs& g, int o, int b) {
  int r = 0;
  for (int t = 0; t < b; ++t) r += owns(g.nbr, g.cnt, o, t);
  return bin_begin(g.base_local, g.base_partial, o) + r;
}

__device__ __forceinline__ int slot_pair(const AvmBuildArgs& g, int c, int u, int w) {
  const int m = g.cnt[c];
  for (int b = 0; b < m; ++b)
    if (g.nbr[c * CG_RING + b] == u && g.nbr[c * CG_RING + (b + 1) % m] == w) return b;
  return -1;
}

__global__ void k_avm_cell_lists(AvmBuildArgs g) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.n) return;
  const int m = g.cnt[c];
  g.cc[c] = m;
  for (int a = 0; a < CG_RING; ++a) {
    int vid = -1;
    if (a < m) {
      const int j = g.nbr[c * CG_RING + a], k = g.nbr[c * CG_RING + (a + 1) % m];
      if (c < j && c < k) {
        vid = owned_rank(g, c, a);
      } else {
        int o, b;
        if (j < k) { o = j; b = slot_pair(g, j, k, c); }
        else { o = k; b = slot_pair(g, k, c, j); }
        vid = b < 0 ? -1 : owned_rank(g, o, b);
      }
      if (vid >= 2 * g.n) vid = -1;
      if (vid < 0) raise_status(g.ctl, kETOPO);
    }
    g.cv[c * CG_RING + a] = vid;
  }
}

__global__ void k_avm_vertices(AvmBuildArgs g) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= g.n) return;
  const int m = g.cnt[o];
  for (int b = 0; b < m; ++b) {
    if (!owns(g.nbr, g.cnt, o, b)) continue;
    const int j = g.nbr[o * CG_RING + b], k = g.nbr[o * CG_RING + (b + 1) % m];
    const int v = g.cv[o * CG_RING + b];
    if (v < 0) continue;
    g.vc[3 * v + 0] = o; g.vc[3 * v + 1] = j; g.vc[3 * v + 2] = k;
    g.vn[3 * v + 0] = g.cv[o * CG_RING + (b + m - 1) % m];  // across the edge o-j
    const int p = slot_pair(g, j, k, o);                     // (j, k, o) around j
    const int mj = g.cnt[j];
    if (p < 0) raise_status(g.ctl, kETOPO);
    g.vn[3 * v + 1] = p < 0 ? -1 : g.cv[j * CG_RING + (p + mj - 1) % mj];  // across j-k
    g.vn[3 * v + 2] = g.cv[o * CG_RING + (b + 1) % m];      // across k-o
    // circumcentre of (o, j, k), minimum-image offsets from o
    const double ax = mimg_d(g.x[j] - g.x[o], g.Lx), ay = mimg_d(g.y[j] - g.y[o], g.Ly);
    const double bx = mimg_d(g.x[k] - g.x[o], g.Lx), by = mimg_d(g.y[k] - g.y[o], g.Ly);
    const double d = 2.0 * (ax * by - ay * bx);
    const double la = ax * ax + ay * ay, lb = bx * bx + by * by;
    g.hx[v] = wrap_d(g.x[o] + (by * la - ay * lb) / d, g.Lx);
    g.hy[v] = wrap_d(g.y[o] + (ax * lb - bx * la) / d, g.Ly);
  }
}

void launch_avm_build(const AvmBuildArgs& a, cudaStream_t st) {
  const int blocks = (a.n + 127) / 128;
  k_avm_count_owned<<<blocks, 128, 0, st>>>(a);
  CellListArgs sc{};
  sc.n = a.n;
  sc.nbins = a.n;
  sc.ctl = a.ctl;
  sc.bin_count = a.owned;
  sc.bin_start = a.base_local;
  sc.scan_partials = a.base_partial;
  sc.only_if_flagged = 0;
  launch_scan(sc, st);
  k_avm_cell_lists<<<blocks, 128, 0, st>>>(a);
  k_avm_vertices<<<blocks, 128, 0, st>>>(a);
}

// ---------------------------------------------------------------------------
// Step kernels.
// ---------------------------------------------------------------------------
// Director terms of the next step (launch_avm_dir): the self-propulsion
// (v0/3) n(theta) of the current director (each of a cell's vertices takes a
// third, Eq. 4 with n = 3) and the director after the next step's rotation,
// theta + sqrt(2 D_r dt) xi (Philox, counter (cell, step) with the step
// counter of the next step, cell id = tag).  Cells removed by a T2 turn as
// well.
__global__ void k_avm_dir(AvmArgs g) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.n) return;
  const double th = g.theta[c];
  double sn, cs;
  dm_sincos(th, g.tab, sn, cs);
  const double v3 = g.v0[c] * (1.0 / 3.0);
  g.act[c] = make_double2(v3 * cs, v3 * sn);
  g.thn[c] = th + g.noise_amp * director_noise(g.seed, g.ctag[c], g.ctl->step, g.tab);
}

// Per cell: area and perimeter of the polygon and the force coefficients
// ka = 2 K_A (A - A0) and kp = 2 K_P (P - P0); when stepping, the director
// takes its rotated value thn (k_avm_dir computed it, with the activity act
// of the current director, before the step).
__global__ void k_avm_cells(AvmArgs g) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.n) return;
  const size_t V = (size_t)g.V;
  const int cur = g.ctl->cur;
  const double* hx = g.hx + cur * V;
  const double* hy = g.hy + cur * V;
  const int m = g.cc[c];
  if (g.move) g.theta[c] = g.thn[c];
  if (m == 0) {  // removed by a T2: no geometry, no force; the director still turns
    g.A[c] = 0.0;
    g.P[c] = 0.0;
    g.ka[c] = 0.0;
    g.kp[c] = 0.0;
    if (g.energy) g.energy[c] = 0.0;
    return;
  }
  if (m < 3 || m > CG_RING) {
    raise_status(g.ctl, kETOPO);
    return;
  }
  const int* row = g.cv + (size_t)c * CG_RING;
  for (int a = 0; a < m; ++a)
    if ((unsigned)row[a] >= (unsigned)g.V) {
      raise_status(g.ctl, kETOPO);
      return;
    }
  const int v0 = row[0];
  const double x0 = hx[v0], y0 = hy[v0];
  double px = 0.0, py = 0.0, area = 0.0, per = 0.0;
  for (int a = 1; a <= m; ++a) {
    double qx = 0.0, qy = 0.0;
    if (a < m) {
      const int v = row[a];
      qx = mimg_a(hx[v] - x0, g.ax);
      qy = mimg_a(hy[v] - y0, g.ay);
    }
    area = fma(-qx, py, fma(px, qy, area));
    const double l2 = (qx - px) * (qx - px) + (qy - py) * (qy - py);
    per = (__double_as_longlong(l2) > 0) ? fma(l2, fx_rsqrt(l2), per) : per;  // sqrt(l2)
    px = qx;
    py = qy;
  }
  const double A = 0.5 * area, P = per;
  g.A[c] = A;
  g.P[c] = P;
  const double dA = A - g.a0[c], dP = P - g.P0[c];
  g.ka[c] = g.KA * dA;  // half of dE/dA = 2 K_A (A - A0): dA/dh carries a 1/2
  g.kp[c] = 2.0 * g.KP * dP;
  if (g.energy) g.energy[c] = g.KA * dA * dA + g.KP * dP * dP;
}

// Per vertex: F_v = -sum_k [ka_k 1/2 perp(u_{k-1} - u_k) - kp_k (u^_k + u^_{k-1})]
// with u_k = h(n_k) - h(v); then, when stepping, the move of Eq. 4 into the
// other position buffer.  The last block switches buffers, advances the step
// counter and opens the step's T1 passes.
__global__ void k_avm_force_move(AvmArgs g) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t V = (size_t)g.V;
  const int cur = g.ctl->cur;
  bool ok = v < g.V;
  if (ok && g.vc[3 * v] < 0) {  // freed by a T2: stays where it is
    ok = false;
    g.Fx[v] = 0.0;
    g.Fy[v] = 0.0;
    if (g.move) {
      g.hx[(cur ^ 1) * V + v] = g.hx[cur * V + v];
      g.hy[(cur ^ 1) * V + v] = g.hy[cur * V + v];
    }
  }
  if (ok)
    for (int k = 0; k < 3; ++k)
      if ((unsigned)g.vn[3 * v + k] >= (unsigned)g.V || (unsigned)g.vc[3 * v + k] >= (unsigned)g.n) {
        raise_status(g.ctl, kETOPO);
        ok = false;
        break;
      }
  if (ok) {
    const double* hx = g.hx + cur * V;
    const double* hy = g.hy + cur * V;
    const double xv = hx[v], yv = hy[v];
    double ux[3], uy[3], il[3], kh[3], kp[3];
    double ax = 0.0, ay = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int w = g.vn[3 * v + k];
      ux[k] = mimg_a(hx[w] - xv, g.ax);
      uy[k] = mimg_a(hy[w] - yv, g.ay);
      il[k] = fx_rsqrt(ux[k] * ux[k] + uy[k] * uy[k]);
      const int c = g.vc[3 * v + k];
      kh[k] = g.ka[c];
      kp[k] = g.kp[c];
      if (g.move) {
        const double2 a = g.act[c];
        ax += a.x;
        ay += a.y;
      }
    }
    // dE_c/dh = kh perp(h_next - h_prev) + kp (t^_in - t^_out) summed over the
    // three cells and regrouped by edge: edge k (to vn[k], between cells k and
    // k+1) carries u_k (kh_k - kh_{k+1}) rotated and u^_k (kp_k + kp_{k+1});
    // F = -dE/dh, kh = K_A (A - A0) stored halved
    double fx = 0.0, fy = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int kn = (k + 1) % 3;
      const double dkh = kh[k] - kh[kn], skp = (kp[k] + kp[kn]) * il[k];
      fx = fma(uy[k], dkh, fma(ux[k], skp, fx));
      fy = fma(-ux[k], dkh, fma(uy[k], skp, fy));
    }
    g.Fx[v] = fx;
    g.Fy[v] = fy;
    if (g.move) {
      const int nxt = cur ^ 1;
      const double mx = xv + g.dt * (g.mu * fx + ax), my = yv + g.dt * (g.mu * fy + ay);
      if (!isfinite(mx) || !isfinite(my)) raise_status(g.ctl, kENONFINITE);
      const double wx = wrap_a(mx, g.ax), wy = wrap_a(my, g.ay);
      g.hx[nxt * V + v] = wx;
      g.hy[nxt * V + v] = wy;
      g.hf[v] = make_float2((float)wx, (float)wy);
    }
  }
  if (!g.move) return;  // uniform over the grid
  if (last_block(g.done) && threadIdx.x == 0) {
    Ctl* ctl = g.ctl;
    ctl->cur = cur ^ 1;
    ctl->step += 1;
    ctl->last_flagged = 0;  // T1 passes run in this step
    ctl->pad = 1;
  }
}

// Opens T1 passes on the current state without a move.
__global__ void k_avm_begin_t1(Ctl* ctl) {
  ctl->last_flagged = 0;
  ctl->count[1] = 0;
  ctl->pad = 1;
}

// ---------------------------------------------------------------------------
// T1 passes: the body of a conditional (while) graph node.  Candidate edges
// take an atomic minimum of a 64-bit key on their four cells; the high word
// 0xffffffff - pass number makes every key of this pass smaller than any
// left over from earlier passes, so the locks never need clearing.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long lock_key(int stamp, int e) {
  return ((unsigned long long)(0xffffffffu - (unsigned)stamp) << 32) | (unsigned)e;
}

__device__ __forceinline__ double len2_rn(double dx, double dy) {
  // products and sum rounded separately (no fused multiply-add)
  return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

// FP32 squared length of edge (v, w), v < w, from the float copies of the
// positions, in a fixed rounding order (the proposal's filter and the
// apply kernel's look-ahead see the same value).
__device__ __forceinline__ float t1_len2_f(const AvmArgs& g, float2 pv, float2 pw) {
  const float fx = mimg_f(pw.x - pv.x, g.Lxf), fy = mimg_f(pw.y - pv.y, g.Lyf);
  return __fadd_rn(__fmul_rn(fx, fx), __fmul_rn(fy, fy));
}

__device__ __forceinline__ int slot3(const int* a, int v, int val) {
  for (int s = 0; s < 3; ++s)
    if (a[3 * v + s] == val) return s;
  return -1;
}

// Cell other than c that has both vertices va and vb, or -1.
__device__ __forceinline__ int cell_across(const int* __restrict__ vc, int c, int va, int vb) {
  int r = -1;
#pragma unroll
  for (int s = 2; s >= 0; --s) {
    const int x = vc[3 * va + s];
    if (x != c && x >= 0 && (x == vc[3 * vb] || x == vc[3 * vb + 1] || x == vc[3 * vb + 2])) r = x;
  }
  return r;
}

// T2 proposal for the triangular cell c: twice its signed area (each product
// and the difference rounded separately, offsets from its first vertex)
// below twice the threshold; the cells across its three edges must be
// distinct with more than 3 vertices and the outer vertices distinct.  The
// candidate id is 3V + tag(c); its cells are c and the three across its edges.
__device__ void t2_propose(const AvmArgs& g, int c, int stamp) {
  const size_t V = (size_t)g.V;
  const int cur = g.ctl->cur;
  const double* hx = g.hx + cur * V;
  const double* hy = g.hy + cur * V;
  const int* row = g.cv + (size_t)c * CG_RING;
  int v[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    v[a] = row[a];
    if ((unsigned)v[a] >= (unsigned)g.V) {
      raise_status(g.ctl, kETOPO);
      return;
    }
  }
  const double px1 = mimg_a(hx[v[1]] - hx[v[0]], g.ax), py1 = mimg_a(hy[v[1]] - hy[v[0]], g.ay);
  const double px2 = mimg_a(hx[v[2]] - hx[v[0]], g.ax), py2 = mimg_a(hy[v[2]] - hy[v[0]], g.ay);
  const double d = __dsub_rn(__dmul_rn(px1, py2), __dmul_rn(px2, py1));
  if (!(d < g.t2_twice)) return;
  int nb[3], w[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int s = slot3(g.vc, v[a], c);
    nb[a] = cell_across(g.vc, c, v[a], v[(a + 1) % 3]);
    if (s < 0 || nb[a] < 0) {
      raise_status(g.ctl, kETOPO);
      return;
    }
    w[a] = g.vn[3 * v[a] + (s + 1) % 3];
  }
  bool ok = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    ok &= g.cc[nb[a]] > 3;
    ok &= nb[a] != nb[(a + 1) % 3] && w[a] != w[(a + 1) % 3];
    ok &= w[a] != v[0] && w[a] != v[1] && w[a] != v[2];
  }
  if (!ok) {  // a later transition may allow it
    g.ctl->t1_more = 1;
    return;
  }
  const int ek = 3 * g.V + g.ctag[c];  // priority: the id in tags
  const unsigned long long key = lock_key(stamp, ek);
  atomicMin(&g.lock[c], key);
  atomicMin(&g.lock[nb[0]], key);
  atomicMin(&g.lock[nb[1]], key);
  atomicMin(&g.lock[nb[2]], key);
  const int slot = atomicAdd(&g.ctl->count[1], 1);
  g.cand_e[slot] = 3 * g.V + c;
  g.cand_k[slot] = ek;
  g.cand[slot] = make_int4(c, nb[0], nb[1], nb[2]);
}

// One thread per vertex slot v, its edges (v, w) with slot w > v.  The
// squared length is first bounded in FP32 from the float copies of the
// positions; only edges within the error band of the threshold are decided in
// FP64 in the fixed rounding order (both bounds are symmetric in the two
// ends).  A short edge is then oriented from its end of smaller tag, v1 (the
// edge is slot a of v1's lists), and takes the id 3 tag(v1) + a.  Candidates
// go to a compact list.  A short edge that its cells' vertex counts keep from
// flipping marks the pass as possibly leaving work (another flip may change
// those counts).
__global__ void k_t1_propose(AvmArgs g) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  // stop the loop unless the closing kernel of this pass asks for another
  if (v == 0 && g.loop) cudaGraphSetConditional(g.loop, 0);
  const int stamp = g.ctl->round_count;
  if (g.t2_twice > 0.0 && v < g.n && g.cc[v] == 3) t2_propose(g, v, stamp);
  if (v >= g.V) return;
  const size_t V = (size_t)g.V;
  const float2 pv = g.hf[v];
  for (int s = 0; s < 3; ++s) {
    const int e = 3 * v + s;
    const int w = g.vn[e];
    if (w <= v) continue;
    if (w >= g.V) {
      raise_status(g.ctl, kETOPO);
      continue;
    }
    const float l2 = t1_len2_f(g, pv, g.hf[w]);
    if (l2 > g.t2hi) continue;
    if (!(l2 < g.t2lo)) {
      const int cur = g.ctl->cur;
      const double* hx = g.hx + cur * V;
      const double* hy = g.hy + cur * V;
      const double dx = mimg_a(hx[w] - hx[v], g.ax), dy = mimg_a(hy[w] - hy[v], g.ay);
      if (!(len2_rn(dx, dy) < g.thr2)) continue;
    }
    // orientation by tags: v1 the end of smaller tag, the edge slot a of v1
    // and slot b of v2; both ends' neighbour lists give the flip's four outer
    // vertices, recorded with the candidate so that the flip loads nothing
    // whose address waits on another load
    const int tv = g.vtag[v], tw = g.vtag[w];
    const int rv0 = g.vn[3 * v], rv1 = g.vn[3 * v + 1], rv2 = g.vn[3 * v + 2];
    const int rw0 = g.vn[3 * w], rw1 = g.vn[3 * w + 1], rw2 = g.vn[3 * w + 2];
    const int sw = rw0 == v ? 0 : rw1 == v ? 1 : rw2 == v ? 2 : -1;  // slot of v in w's list
    if (sw < 0) {
      raise_status(g.ctl, kETOPO);
      continue;
    }
    const bool vfirst = tv < tw;
    const int v1 = vfirst ? v : w, v2 = vfirst ? w : v;
    const int a = vfirst ? s : sw, b = vfirst ? sw : s;
    const int p0 = vfirst ? rv0 : rw0, p1 = vfirst ? rv1 : rw1, p2 = vfirst ? rv2 : rw2;  // v1's list
    const int q0 = vfirst ? rw0 : rv0, q1 = vfirst ? rw1 : rv1, q2 = vfirst ? rw2 : rv2;  // v2's list
    const int Aul = a == 0 ? p1 : a == 1 ? p2 : p0, All = a == 0 ? p2 : a == 1 ? p0 : p1;
    const int Alr = b == 0 ? q1 : b == 1 ? q2 : q0, Aur = b == 0 ? q2 : b == 1 ? q0 : q1;
    const int i = g.vc[3 * v1 + a], k = g.vc[3 * v1 + (a + 1) % 3], j = g.vc[3 * v1 + (a + 2) % 3];
    int l = -1;
    for (int t = 0; t < 3; ++t) {
      const int c = g.vc[3 * v2 + t];
      if (c != i && c != k) l = c;
    }
    if (l < 0) {
      raise_status(g.ctl, kETOPO);
      continue;
    }
    if (g.cc[i] <= 3 || g.cc[k] <= 3 || g.cc[j] >= CG_RING || g.cc[l] >= CG_RING) {
      g.ctl->t1_more = 1;
      continue;
    }
    const int ek = 3 * min(tv, tw) + a;  // priority: the id in tags
    const unsigned long long key = lock_key(stamp, ek);
    atomicMin(&g.lock[i], key);
    atomicMin(&g.lock[j], key);
    atomicMin(&g.lock[k], key);
    atomicMin(&g.lock[l], key);
    const int slot = atomicAdd(&g.ctl->count[1], 1);
    g.cand_e[slot] = 3 * v1 + a;
    g.cand_k[slot] = ek;
    g.cand[slot] = make_int4(i, j, k, l);
    g.cand_v[slot] = make_int4(v2, Aul, All, Alr);
    g.cand_w[slot] = Aur;
  }
}


__device__ void remove_from_cell(int* cc, int* cv, int c, int v) {
  const int m = cc[c];
  int* row = cv + (size_t)c * CG_RING;
  int w = 0;
  for (int a = 0; a < m; ++a)
    if (row[a] != v) row[w++] = row[a];
  for (int a = w; a < CG_RING; ++a) row[a] = -1;
  cc[c] = w;
}

__device__ void insert_in_cell(int* cc, int* cv, int c, int after, int v) {
  const int m = cc[c];
  int* row = cv + (size_t)c * CG_RING;
  int pos = -1;
  for (int a = 0; a < m; ++a)
    if (row[a] == after) pos = a;
  for (int a = m; a > pos + 1; --a) row[a] = row[a - 1];
  row[pos + 1] = v;
  cc[c] = m + 1;
}

// A cell's vertex list held in registers: four 16-byte loads, edits by
// compile-time-indexed selects, four 16-byte stores.  Slots past the count
// hold -1, as after the in-memory edits above.
struct Row {
  int r[CG_RING];
};
__device__ __forceinline__ Row load_row(const int* cv, int c) {
  Row w;
  const int4* p = reinterpret_cast<const int4*>(cv + (size_t)c * CG_RING);
#pragma unroll
  for (int q = 0; q < CG_RING / 4; ++q) {
    const int4 t = p[q];
    w.r[4 * q] = t.x; w.r[4 * q + 1] = t.y; w.r[4 * q + 2] = t.z; w.r[4 * q + 3] = t.w;
  }
  return w;
}
__device__ __forceinline__ void store_row(int* cv, int c, const Row& w) {
  int4* p = reinterpret_cast<int4*>(cv + (size_t)c * CG_RING);
#pragma unroll
  for (int q = 0; q < CG_RING / 4; ++q)
    p[q] = make_int4(w.r[4 * q], w.r[4 * q + 1], w.r[4 * q + 2], w.r[4 * q + 3]);
}
// Bit a set where entry a < m equals v: every compare at once, no chain.
__device__ __forceinline__ unsigned row_match(const Row& w, int m, int v) {
  unsigned hit = 0u;
#pragma unroll
  for (int a = 0; a < CG_RING; ++a) hit |= (a < m && w.r[a] == v) ? (1u << a) : 0u;
  return hit;
}
// Removes every occurrence of v among the first m entries; returns the count.
__device__ __forceinline__ int row_remove_all(Row& w, int m, int v) {
  Row o;
  int n = 0;
#pragma unroll
  for (int a = 0; a < CG_RING; ++a) o.r[a] = -1;
#pragma unroll
  for (int a = 0; a < CG_RING; ++a) {
    const bool keep = a < m && w.r[a] != v;
#pragma unroll
    for (int b = 0; b <= a; ++b)
      if (keep && n == b) o.r[b] = w.r[a];
    n += keep;
  }
  w = o;
  return n;
}
// The same for the usual case of at most one occurrence (a cell lists a
// vertex once): one shift selected per slot.
__device__ __forceinline__ int row_remove(Row& w, int m, int v) {
  const unsigned hit = row_match(w, m, v);
  if (__popc(hit) > 1) return row_remove_all(w, m, v);
  const int n = max(0, min(m, CG_RING)) - (hit ? 1 : 0);
  const int p = hit ? __ffs(hit) - 1 : CG_RING;
  Row o;
#pragma unroll
  for (int a = 0; a < CG_RING; ++a) {
    const int next = a + 1 < CG_RING ? w.r[a + 1] : -1;
    o.r[a] = a >= n ? -1 : a < p ? w.r[a] : next;
  }
  w = o;
  return n;
}
// Inserts v after the last occurrence of `after` among the first m entries
// (at the front if absent); returns the new count.
__device__ __forceinline__ int row_insert(Row& w, int m, int after, int v) {
  const unsigned hit = row_match(w, m, after);
  const int p = hit ? 31 - __clz(hit) : -1;
  Row o;
#pragma unroll
  for (int a = 0; a < CG_RING; ++a) {
    const int prev = a > 0 ? w.r[a - 1] : -1;
    o.r[a] = (a <= p) ? w.r[a] : (a == p + 1) ? v : (a <= m) ? prev : w.r[a];
  }
  w = o;
  return m + 1;
}

__device__ void apply_t1(const AvmArgs& g, int v1, int a, int4 cd, int4 nv, int Aur, unsigned long long key) {
  Ctl* ctl = g.ctl;
  const size_t V = (size_t)g.V;
  double* hx = g.hx + ctl->cur * V;
  double* hy = g.hy + ctl->cur * V;
  const int e = 3 * v1 + a;
  const int i = cd.x, j = cd.y, k = cd.z, l = cd.w;
  const int v2 = nv.x, Aul = nv.y, All = nv.z, Alr = nv.w;
  if ((unsigned)v2 >= (unsigned)g.V || (unsigned)Aul >= (unsigned)g.V || (unsigned)All >= (unsigned)g.V ||
      (unsigned)Alr >= (unsigned)g.V || (unsigned)Aur >= (unsigned)g.V) {
    raise_status(ctl, kETOPO);
    return;
  }
  // Every load of the flip at once (the proposal recorded the vertices it
  // touches, so no address waits on another load), before the lock check,
  // while other flips of the pass edit the network.  A flip that holds its
  // four locks sees none of this data change: a vertex has three cells, two
  // of them this flip's, so no other winner edits these lists or positions;
  // one that does not hold them discards it.
  const bool distinct = i != j && i != k && i != l && j != k && j != l && k != l;
  Row ri, rk, rj, rl;
  int mi = 0, mk = 0, mj = 0, ml = 0;
  if (distinct) {
    ri = load_row(g.cv, i); rk = load_row(g.cv, k); rj = load_row(g.cv, j); rl = load_row(g.cv, l);
    mi = g.cc[i]; mk = g.cc[k]; mj = g.cc[j]; ml = g.cc[l];
  }
  const int v2r = g.vn[e], Aul_r = g.vn[3 * v1 + (a == 2 ? 0 : a + 1)], All_r = g.vn[3 * v1 + (a == 0 ? 2 : a - 1)];
  int n2[3], c2[3], nu[3], nl[3];
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    n2[t] = g.vn[3 * v2 + t];
    c2[t] = g.vc[3 * v2 + t];
    nu[t] = g.vn[3 * Aul + t];
    nl[t] = g.vn[3 * Alr + t];
  }
  const double x1 = hx[v1], y1 = hy[v1], x2 = hx[v2], y2 = hy[v2];
  const float2 fAll = g.hf[All], fAlr = g.hf[Alr], fAul = g.hf[Aul], fAur = g.hf[Aur];
  if (g.lock[i] != key || g.lock[j] != key || g.lock[k] != key || g.lock[l] != key) {
    ctl->t1_more = 1;
    return;
  }
  // the network as the proposal saw it (always so for a lock holder); the
  // slot b of v1 in v2's lists picks by selects (no indexed local array)
  const int b = n2[0] == v1 ? 0 : n2[1] == v1 ? 1 : n2[2] == v1 ? 2 : -1;
  const int c2b = b == 0 ? c2[0] : b == 1 ? c2[1] : c2[2], c2b1 = b == 0 ? c2[1] : b == 1 ? c2[2] : c2[0];
  const int n2b1 = b == 0 ? n2[1] : b == 1 ? n2[2] : n2[0], n2b2 = b == 0 ? n2[2] : b == 1 ? n2[0] : n2[1];
  if (v2r != v2 || Aul_r != Aul || All_r != All || b < 0 || c2b != k || c2b1 != i || n2b1 != Alr || n2b2 != Aur) {
    raise_status(ctl, kETOPO);
    return;
  }
  const int su = nu[0] == v1 ? 0 : nu[1] == v1 ? 1 : nu[2] == v1 ? 2 : -1;  // v1 in Aul's list
  const int sl = nl[0] == v2 ? 0 : nl[1] == v2 ? 1 : nl[2] == v2 ? 2 : -1;  // v2 in Alr's list
  if (su < 0 || sl < 0) {
    raise_status(ctl, kETOPO);
    return;
  }
  // rotate the edge by 90 degrees about its midpoint, new length t1_len
  const double ex = mimg_a(x2 - x1, g.ax), ey = mimg_a(y2 - y1, g.ay);
  const double mx = x1 + 0.5 * ex, my = y1 + 0.5 * ey;
  // half the new length over the old one, from the refined inverse square
  // root (a short dependent chain; FP64 square root and division are long)
  const double h = fx_rsqrt(ex * ex + ey * ey) * (0.5 * g.t1_len);
  const double px = -ey * h, py = ex * h;
  const double nx1 = wrap_a(mx - px, g.ax), ny1 = wrap_a(my - py, g.ay);
  const double nx2 = wrap_a(mx + px, g.ax), ny2 = wrap_a(my + py, g.ay);
  hx[v1] = nx1; hy[v1] = ny1;
  hx[v2] = nx2; hy[v2] = ny2;
  const float2 f1 = make_float2((float)nx1, (float)ny1), f2 = make_float2((float)nx2, (float)ny2);
  g.hf[v1] = f1;
  g.hf[v2] = f2;
  // Look-ahead: the flip moved only v1 and v2, and no other flip of this pass
  // moves a vertex adjacent to them (it would need one of this flip's locked
  // cells), so the edges at v1 and v2 are the only ones whose length changed.
  // If none of them passes the proposal's FP32 bound, the next pass finds no
  // new candidate here.  (The bound is symmetric in the two ends: the float
  // difference and its minimum image change sign exactly.)
  {
    // the outer vertices' float positions as loaded, or v1's and v2's new
    // ones where a degenerate network names v1 or v2 among them
    auto now = [&](int u, float2 f) { return u == v1 ? f1 : u == v2 ? f2 : f; };
    const bool near = t1_len2_f(g, f1, f2) <= g.t2hi || t1_len2_f(g, f1, now(All, fAll)) <= g.t2hi ||
                      t1_len2_f(g, f1, now(Alr, fAlr)) <= g.t2hi || t1_len2_f(g, f2, now(Aul, fAul)) <= g.t2hi ||
                      t1_len2_f(g, f2, now(Aur, fAur)) <= g.t2hi;
    // (a degenerate network, with a cell on both sides of an edge, takes the
    // next pass regardless)
    if (near || !distinct) ctl->t1_more = 1;
  }
  // neighbour exchange (Fig. 1): v1 -> cells (j, i, l), v2 -> cells (k, j, l)
  g.vc[3 * v1 + 0] = j; g.vc[3 * v1 + 1] = i; g.vc[3 * v1 + 2] = l;
  g.vn[3 * v1 + 0] = All; g.vn[3 * v1 + 1] = Alr; g.vn[3 * v1 + 2] = v2;
  g.vc[3 * v2 + 0] = k; g.vc[3 * v2 + 1] = j; g.vc[3 * v2 + 2] = l;
  g.vn[3 * v2 + 0] = Aul; g.vn[3 * v2 + 1] = v1; g.vn[3 * v2 + 2] = Aur;
  g.vn[3 * Aul + su] = v2;
  g.vn[3 * Alr + sl] = v1;
  if (distinct) {
    g.cc[i] = row_remove(ri, mi, v2);
    g.cc[k] = row_remove(rk, mk, v1);
    g.cc[j] = row_insert(rj, mj, v1, v2);
    g.cc[l] = row_insert(rl, ml, v2, v1);
    store_row(g.cv, i, ri); store_row(g.cv, k, rk); store_row(g.cv, j, rj); store_row(g.cv, l, rl);
  } else {  // a degenerate network: the edits in order, in memory
    remove_from_cell(g.cc, g.cv, i, v2);
    remove_from_cell(g.cc, g.cv, k, v1);
    insert_in_cell(g.cc, g.cv, j, v1, v2);
    insert_in_cell(g.cc, g.cv, l, v2, v1);
  }
  // i or k left as a triangle may be removed by a T2 in the next pass
  if (g.t2_twice > 0.0 && (g.cc[i] == 3 || g.cc[k] == 3)) ctl->t1_more = 1;
  atomicAdd((unsigned long long*)&ctl->repaired_total, 1ull);
}

// Cell x's vertex list with v[0..2] replaced by vk and the repeat this makes
// dropped (x shares one edge with the removed triangle: one vertex fewer).
__device__ void merge_in_cell(int* cc, int* cv, int x, const int* v, int vk) {
  const int m = cc[x];
  int* row = cv + (size_t)x * CG_RING;
  int out = 0;
  for (int a = 0; a < m; ++a) {
    int e = row[a];
    if (e == v[0] || e == v[1] || e == v[2]) e = vk;
    if (out > 0 && e == vk && row[out - 1] == vk) continue;
    row[out++] = e;
  }
  if (out > 1 && row[0] == vk && row[out - 1] == vk) --out;
  for (int a = out; a < CG_RING; ++a) row[a] = -1;
  cc[x] = out;
}

// T2: the triangle c (cells across its edges cd.y, cd.z, cd.w) shrinks to
// its centroid.  The vertex of smallest tag among its three stays, joined to the
// three outer vertices in their order around the triangle; the other two are
// freed (vc, vn = -1) and the cell is emptied (cc = 0, cv = -1).
__device__ void apply_t2(const AvmArgs& g, int c, int4 cd) {
  Ctl* ctl = g.ctl;
  const size_t V = (size_t)g.V;
  double* hx = g.hx + ctl->cur * V;
  double* hy = g.hy + ctl->cur * V;
  int* row = g.cv + (size_t)c * CG_RING;
  int v[3], w[3], cp[3], cpp[3];
  const int nb[3] = {cd.y, cd.z, cd.w};
#pragma unroll
  for (int a = 0; a < 3; ++a) v[a] = row[a];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int s = slot3(g.vc, v[a], c);
    if (s < 0) {
      raise_status(ctl, kETOPO);
      return;
    }
    w[a] = g.vn[3 * v[a] + (s + 1) % 3];
    cp[a] = g.vc[3 * v[a] + (s + 1) % 3];
    cpp[a] = g.vc[3 * v[a] + (s + 2) % 3];
  }
  const int t0 = g.vtag[v[0]], t1 = g.vtag[v[1]], t2 = g.vtag[v[2]];
  const int vk = (t0 < t1) ? (t0 < t2 ? v[0] : v[2]) : (t1 < t2 ? v[1] : v[2]);
  // centroid relative to the first vertex of the list
  const double dx1 = mimg_a(hx[v[1]] - hx[v[0]], g.ax), dy1 = mimg_a(hy[v[1]] - hy[v[0]], g.ay);
  const double dx2 = mimg_a(hx[v[2]] - hx[v[0]], g.ax), dy2 = mimg_a(hy[v[2]] - hy[v[0]], g.ay);
  const double cx = wrap_a(hx[v[0]] + (dx1 + dx2) / 3.0, g.ax);
  const double cy = wrap_a(hy[v[0]] + (dy1 + dy2) / 3.0, g.ay);
  // outer edges around the kept vertex: from a = 0, each next one starts in
  // the cell where the previous one ends
  int ord[3] = {0, -1, -1};
#pragma unroll
  for (int q = 1; q < 3; ++q)
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (cp[a] == cpp[ord[q - 1]] && a != ord[0] && (q < 2 || a != ord[1])) ord[q] = a;
  if (ord[1] < 0 || ord[2] < 0 || cpp[ord[2]] != cp[ord[0]]) {
    raise_status(ctl, kETOPO);
    return;
  }
  int so[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    so[a] = slot3(g.vn, w[a], v[a]);
    if (so[a] < 0) {
      raise_status(ctl, kETOPO);
      return;
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) g.vn[3 * w[a] + so[a]] = vk;
#pragma unroll
  for (int a = 0; a < 3; ++a) merge_in_cell(g.cc, g.cv, nb[a], v, vk);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    g.vc[3 * vk + q] = cp[ord[q]];
    g.vn[3 * vk + q] = w[ord[q]];
  }
  hx[vk] = cx;
  hy[vk] = cy;
  g.hf[vk] = make_float2((float)cx, (float)cy);
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (v[a] != vk)
#pragma unroll
      for (int q = 0; q < 3; ++q) g.vc[3 * v[a] + q] = g.vn[3 * v[a] + q] = -1;
#pragma unroll
  for (int a = 0; a < CG_RING; ++a) row[a] = -1;
  g.cc[c] = 0;
  ctl->t1_more = 1;  // the merged vertex's edges and the neighbours' counts changed
  atomicAdd((unsigned long long*)&ctl->flagged_total, 1ull);
}

// Applies the listed candidates (T1 edges, T2 cells) that hold all four
// locks (passes 0 .. t1_cap-1; pass t1_cap only counts) and closes the pass:
// another pass runs while this one may have left work (a candidate that lost
// a lock, an edge at a moved vertex within the FP32 bound of the threshold,
// or a short edge its cells kept from flipping) and the cap is not reached;
// candidates at the counting pass raise the T1-cap status.  Without such
// work the next pass would propose nothing, so it is skipped.  A pass of at
// most one block's worth of candidates (the usual case once the tissue has
// relaxed) is applied by block 0 alone and closed after a block barrier; a
// larger one (the first steps of a fresh network) by every block, closed by
// the last block to finish.
constexpr int kApplyThreads = 128;
__global__ void k_t1_apply(AvmArgs g) {
  Ctl* ctl = g.ctl;
  // this thread's first candidate is loaded beside the pass's counters, before
  // their values are known (the list always has room for the index)
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  const bool room = t0 < 3 * g.V / 2 + g.n + 1;
  const int e0 = room ? g.cand_e[t0] : 0, k0 = room ? g.cand_k[t0] : 0, w0 = room ? g.cand_w[t0] : 0;
  const int4 cd0 = room ? g.cand[t0] : make_int4(0, 0, 0, 0), nv0 = room ? g.cand_v[t0] : make_int4(0, 0, 0, 0);
  const int pass = ctl->last_flagged;
  const int proposed = *(volatile int*)&ctl->count[1];
  // the same for every block (the count is cleared only by the closing
  // block, after every block that uses it has read it)
  const bool one_block = proposed <= (int)blockDim.x;
  if (one_block && blockIdx.x != 0) return;
  const int stride = one_block ? blockDim.x : gridDim.x * blockDim.x;
  if (pass < g.t1_cap) {
    const int stamp = ctl->round_count;
    for (int t = t0; t < proposed; t += stride) {
      const bool first = t == t0;
      const int e = first ? e0 : g.cand_e[t];
      const int4 cd = first ? cd0 : g.cand[t];
      const unsigned long long key = lock_key(stamp, first ? k0 : g.cand_k[t]);
      if (e < 3 * g.V) {
        apply_t1(g, e / 3, e % 3, cd, first ? nv0 : g.cand_v[t], first ? w0 : g.cand_w[t], key);  // checks the locks itself
        continue;
      }
      if (g.lock[cd.x] != key || g.lock[cd.y] != key || g.lock[cd.z] != key || g.lock[cd.w] != key) {
        ctl->t1_more = 1;
        continue;
      }
      apply_t2(g, e - 3 * g.V, cd);
    }
  }
  bool closing;
  if (one_block) {
    __syncthreads();  // every flip of the pass is done, its flags visible here
    closing = threadIdx.x == 0;
  } else {
    closing = last_block(g.done + 1) && threadIdx.x == 0;
  }
  if (closing) {
    ctl->count[1] = 0;
    ctl->round_count += 1;
    ctl->loop_total += 1;
    ctl->last_flagged = pass + 1;
    if (pass >= g.t1_cap && proposed > 0) atomicCAS(&ctl->status, 0, (int)kET1CAP);
    const int more = proposed > 0 && *(volatile int*)&ctl->t1_more && pass < g.t1_cap && ctl->status == 0;
    ctl->t1_more = 0;
    ctl->pad = more;  // read by the host when the passes run outside a graph
    if (more && g.loop) cudaGraphSetConditional(g.loop, 1);
  }
}

// Float copies of the current positions (after the network or the positions
// were replaced from outside).
__global__ void k_avm_shadow(AvmArgs g) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= g.V) return;
  const size_t off = (size_t)g.ctl->cur * g.V;
  g.hf[v] = make_float2((float)g.hx[off + v], (float)g.hy[off + v]);
}

// Index ranges of a network handed in from outside: vc in [0, n), vn in
// [0, V), 3 <= cc <= CG_RING, cv[a] in [0, V) for a < cc.
__global__ void k_avm_validate(AvmArgs g) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  if (t < g.V) {
    const bool freed = g.vc[3 * t] < 0;  // freed by a T2: all six entries -1
    for (int k = 0; k < 3; ++k)
      bad |= freed ? (g.vc[3 * t + k] != -1 || g.vn[3 * t + k] != -1)
                   : ((unsigned)g.vc[3 * t + k] >= (unsigned)g.n || (unsigned)g.vn[3 * t + k] >= (unsigned)g.V);
  }
  if (t < g.n) {
    const int m = g.cc[t];  // 0: removed by a T2
    if (m != 0 && (m < 3 || m > CG_RING)) bad = true;
    else
      for (int a = 0; a < m; ++a) bad |= (unsigned)g.cv[(size_t)t * CG_RING + a] >= (unsigned)g.V;
  }
  if (bad) raise_status(g.ctl, kEINVAL);
}

// Division of cell c along (ux, uy) into c and newc with new vertices va (A)
// and vb (B), the per-cell values copied to newc.  With p the minimum-image
// offsets of the vertices from the first one, m their mean (sum in list
// order, then / count), q = p - m and s = u x q, an edge is cut where s
// changes sign (s > 0 against s <= 0) at X = q_a + t (q_b - q_a),
// t = s_a / (s_a - s_b) clamped to [1/16, 15/16]; the cut with the smallest
// u.X > 0 gives A, the one with the largest u.X < 0 gives B.  Every product,
// sum and quotient is rounded on its own, so the host reference decides the
// same.  c keeps A, v_{a1+1} .. v_{a2}, B; newc gets B, v_{a2+1} .. v_{a1}, A.
// Returns 0 made, 1 refused (a missing cut, a daughter or a neighbour over 16
// vertices), -1 for an inconsistent network.
__device__ int divide_cell(const AvmArgs& g, int c, double ux, double uy, int newc, int va, int vb,
                           bool commit = true) {
  const size_t V = (size_t)g.V;
  double* hx = g.hx + g.ctl->cur * V;
  double* hy = g.hy + g.ctl->cur * V;
  const int m = g.cc[c];
  if (m < 3 || m > CG_RING) return 1;
  int v[CG_RING];
  double px[CG_RING], py[CG_RING], sd[CG_RING];
  for (int a = 0; a < m; ++a) v[a] = g.cv[(size_t)c * CG_RING + a];
  for (int a = 0; a < m; ++a) {
    px[a] = mimg_a(hx[v[a]] - hx[v[0]], g.ax);
    py[a] = mimg_a(hy[v[a]] - hy[v[0]], g.ay);
  }
  double sx = 0.0, sy = 0.0;
  for (int a = 1; a < m; ++a) {
    sx = __dadd_rn(sx, px[a]);
    sy = __dadd_rn(sy, py[a]);
  }
  const double mx = __ddiv_rn(sx, (double)m), my = __ddiv_rn(sy, (double)m);
  for (int a = 0; a < m; ++a) {
    px[a] = __dsub_rn(px[a], mx);  // q
    py[a] = __dsub_rn(py[a], my);
    sd[a] = __dsub_rn(__dmul_rn(ux, py[a]), __dmul_rn(uy, px[a]));
  }
  int a1 = -1, a2 = -1;
  double l1 = 0.0, l2 = 0.0, X1x = 0.0, X1y = 0.0, X2x = 0.0, X2y = 0.0;
  for (int a = 0; a < m; ++a) {
    const int b = (a + 1 == m) ? 0 : a + 1;
    if ((sd[a] > 0.0) == (sd[b] > 0.0)) continue;
    double t = __ddiv_rn(sd[a], __dsub_rn(sd[a], sd[b]));
    if (t < 0.0625) t = 0.0625;
    if (t > 0.9375) t = 0.9375;
    const double Xx = __dadd_rn(px[a], __dmul_rn(t, __dsub_rn(px[b], px[a])));
    const double Xy = __dadd_rn(py[a], __dmul_rn(t, __dsub_rn(py[b], py[a])));
    const double lam = __dadd_rn(__dmul_rn(ux, Xx), __dmul_rn(uy, Xy));
    if (lam > 0.0 && (a1 < 0 || lam < l1)) { a1 = a; l1 = lam; X1x = Xx; X1y = Xy; }
    if (lam < 0.0 && (a2 < 0 || lam > l2)) { a2 = a; l2 = lam; X2x = Xx; X2y = Xy; }
  }
  if (a1 < 0 || a2 < 0) return 1;
  const int n1 = (a2 - a1 + m) % m + 2, n2 = (a1 - a2 + m) % m + 2;
  if (n1 > CG_RING || n2 > CG_RING) return 1;
  const int p1 = v[a1], p1n = v[(a1 + 1) % m], p2 = v[a2], p2n = v[(a2 + 1) % m];
  int x1 = -1, x2 = -1;
  for (int s = 0; s < 3; ++s) {
    const int y1 = g.vc[3 * p1 + s], y2 = g.vc[3 * p2 + s];
    if (y1 != c && (y1 == g.vc[3 * p1n] || y1 == g.vc[3 * p1n + 1] || y1 == g.vc[3 * p1n + 2])) x1 = y1;
    if (y2 != c && (y2 == g.vc[3 * p2n] || y2 == g.vc[3 * p2n + 1] || y2 == g.vc[3 * p2n + 2])) x2 = y2;
  }
  if (x1 < 0 || x2 < 0) return -1;
  if (g.cc[x1] + (x1 == x2 ? 2 : 1) > CG_RING) return 1;
  if (x1 != x2 && g.cc[x2] + 1 > CG_RING) return 1;
  const double ax = __dadd_rn(mx, X1x), ay = __dadd_rn(my, X1y);
  const double bx = __dadd_rn(mx, X2x), by = __dadd_rn(my, X2y);
  const double x0 = hx[v[0]], y0 = hy[v[0]];
  const int s1 = slot3(g.vn, p1, p1n), s1n = slot3(g.vn, p1n, p1);
  const int s2 = slot3(g.vn, p2, p2n), s2n = slot3(g.vn, p2n, p2);
  if (s1 < 0 || s1n < 0 || s2 < 0 || s2n < 0) return -1;
  if (!commit) return 0;  // the division would be made (nothing written)
  g.vn[3 * p1 + s1] = va;
  g.vn[3 * p1n + s1n] = va;
  g.vn[3 * p2 + s2] = vb;
  g.vn[3 * p2n + s2n] = vb;
  int d1[CG_RING], d2[CG_RING], k1 = 0, k2 = 0;
  d1[k1++] = va;
  for (int a = (a1 + 1) % m;; a = (a + 1) % m) {
    d1[k1++] = v[a];
    if (a == a2) break;
  }
  d1[k1++] = vb;
  d2[k2++] = vb;
  for (int a = (a2 + 1) % m;; a = (a + 1) % m) {
    d2[k2++] = v[a];
    const int s = slot3(g.vc, v[a], c);
    if (s < 0) return -1;
    g.vc[3 * v[a] + s] = newc;
    if (a == a1) break;
  }
  d2[k2++] = va;
  for (int a = 0; a < CG_RING; ++a) {
    g.cv[(size_t)c * CG_RING + a] = a < k1 ? d1[a] : -1;
    g.cv[(size_t)newc * CG_RING + a] = a < k2 ? d2[a] : -1;
  }
  g.cc[c] = k1;
  g.cc[newc] = k2;
  insert_in_cell(g.cc, g.cv, x1, p1n, va);
  insert_in_cell(g.cc, g.cv, x2, p2n, vb);
  g.vc[3 * va] = x1; g.vc[3 * va + 1] = c; g.vc[3 * va + 2] = newc;
  g.vn[3 * va] = p1n; g.vn[3 * va + 1] = vb; g.vn[3 * va + 2] = p1;
  g.vc[3 * vb] = x2; g.vc[3 * vb + 1] = newc; g.vc[3 * vb + 2] = c;
  g.vn[3 * vb] = p2n; g.vn[3 * vb + 1] = va; g.vn[3 * vb + 2] = p2;
  const double hax = wrap_a(__dadd_rn(x0, ax), g.ax), hay = wrap_a(__dadd_rn(y0, ay), g.ay);
  const double hbx = wrap_a(__dadd_rn(x0, bx), g.ax), hby = wrap_a(__dadd_rn(y0, by), g.ay);
  hx[va] = hax; hy[va] = hay;
  hx[vb] = hbx; hy[vb] = hby;
  g.hf[va] = make_float2((float)hax, (float)hay);
  g.hf[vb] = make_float2((float)hbx, (float)hby);
  g.theta[newc] = g.theta[c];
  g.p0[newc] = g.p0[c];
  g.v0[newc] = g.v0[c];
  g.a0[newc] = g.a0[c];
  g.P0[newc] = g.P0[c];
  return 0;
}

// The divisions of a call, with the result of doing them one after the other
// in request order (each seeing the network the previous ones left), in
// rounds: the body of a conditional while node (launch_avm_divide_round).
// Division k reads and writes only the cells of its mother's 1-ring (the
// mother, the cells across its edges) and the vertices between them, plus
// fresh slots; divisions whose 1-rings are disjoint therefore commute.  Each
// round, the pending divisions of a window of kDivWindow take a 64-bit atomic
// minimum of (round stamp, request index) on every cell of their 1-ring (the
// stamp makes this round's keys smaller than any earlier one's, so the locks
// are never cleared within a call); the longest prefix of the window whose
// divisions all hold their locks is mutually disjoint and disjoint from every
// division after it.  Its divisions are tried without writing (made or not),
// one per block so that their FP64 work spreads over the SMs; each made one
// then takes its slots in request order (the next unused entries of cslots
// and of vslots, two each, after the made ones before it) and they are
// applied together.  Three kernels a round: locks, check and dry run,
// application (whose last block closes the round).  A division of a cell slot without a polygon (empty: an earlier
// division of the call may fill it) waits until it is the first pending one.
// The first pending division always holds its locks, so every round makes
// progress.  made[k] = 1 when division k was made.
constexpr int kDivLockThreads = 128;

__device__ __forceinline__ unsigned long long div_key(int round, int k) {
  return ((unsigned long long)(0xffffffffu - (unsigned)round) << 32) | (unsigned)k;
}

// Visits the cells of the 1-ring of c (c itself, then the cells of each of
// its vertices; repeats included).
template <class F>
__device__ __forceinline__ void for_ring_cells(const AvmArgs& g, int c, int m, F f) {
  f(c);
  for (int a = 0; a < m; ++a) {
    const int v = g.cv[(size_t)c * CG_RING + a];
    if ((unsigned)v < (unsigned)g.V)
      for (int q = 0; q < 3; ++q) {
        const int x = g.vc[3 * v + q];
        if ((unsigned)x < (unsigned)g.n) f(x);
      }
  }
}

// The free slots a call's divisions may take, in increasing tag order: empty
// cells (cc = 0) and free vertices (vc = -1), compacted on the device (flags,
// the counting-sort scan, a scatter); the cells the call names (tags) mapped
// to their slots.
__global__ void k_div_free_flags(AvmArgs g, const int* cslot, const int* vslot, int* fc, int* fv) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < g.n) fc[t] = g.cc[cslot[t]] == 0;
  if (t < g.V) fv[t] = g.vc[3 * vslot[t]] < 0;
}

__global__ void k_div_free_list(DivArgs d, const int* cslot, const int* vslot, const int* fc, const int* sc,
                                const int* scp, const int* fv, const int* sv, const int* svp) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = d.g.n, V = d.g.V, want = d.dc->count;
  if (t < n) {
    if (fc[t]) {
      const int p = bin_begin(sc, scp, t);
      if (p < want) d.cslots[p] = cslot[t];
    }
    const int k = t;  // the named cells, tags -> slots
    if (k < want) {
      const int c = d.cells[k];
      if ((unsigned)c < (unsigned)n) d.cells[k] = cslot[c];
    }
  }
  if (t < V && fv[t]) {
    const int p = bin_begin(sv, svp, t);
    if (p < 2 * want) d.vslots[p] = vslot[t];
  }
  if (t == 0) {
    d.dc->free_c = bin_begin(sc, scp, n);
    d.dc->free_v = bin_begin(sv, svp, V);
  }
}

// A call with fewer free slots than it may need makes no division and
// raises nothing (stop = 2; the host refuses the call).
__global__ void k_div_begin(DivArgs d) {
  DivCtl* dc = d.dc;
  dc->start = 0;
  dc->used = 0;
  dc->round = 0;
  dc->stop = (dc->free_c < dc->count || dc->free_v < 2 * dc->count) ? 2 : 0;
  dc->done = 0u;
}

__global__ void __launch_bounds__(kDivLockThreads) k_div_lock(DivArgs d) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  // stop the loop unless the closing kernel of this round asks for another
  if (t == 0 && d.loop) cudaGraphSetConditional(d.loop, 0);
  DivCtl* dc = d.dc;
  const int start = dc->start, wend = min(dc->count, start + kDivWindow);
  if (t == 0) dc->end = wend;
  const int k = start + t;
  if (k >= wend || dc->stop) return;
  const int c = d.cells[k];
  if ((unsigned)c >= (unsigned)d.g.n) return;
  const int m = d.g.cc[c];
  const unsigned long long key = div_key(dc->round, k);
  for_ring_cells(d.g, c, (m >= 3 && m <= CG_RING) ? m : 0, [&](int x) { atomicMin(&d.dlock[x], key); });
}

// One block per division of the window (lane 0 works, so that the divisions'
// FP64 work spreads over the SMs): whether it holds every lock of its 1-ring
// (the first non-holder ends the round's prefix) and, if it does, the dry run
// (made or not).  A holder beyond the prefix is tried too, harmlessly: it
// reads only its own 1-ring, which no division of the prefix touches.
__global__ void k_div_check_dry(DivArgs d) {
  if (threadIdx.x != 0) return;
  DivCtl* dc = d.dc;
  const int b = blockIdx.x, start = dc->start, wend = min(dc->count, start + kDivWindow);
  const int k = start + b;
  int flag = 0;
  if (k < wend && !dc->stop) {
    const int c = d.cells[k];
    bool ok = (unsigned)c < (unsigned)d.g.n;
    if (ok) {
      const int m = d.g.cc[c];
      const bool poly = m >= 3 && m <= CG_RING;
      // a mother without a polygon waits until it is the first pending division
      ok = poly || k == start;
      const unsigned long long key = div_key(dc->round, k);
      for_ring_cells(d.g, c, poly ? m : 0, [&](int x) { ok = ok && d.dlock[x] == key; });
    }
    if (!ok) {
      atomicMin(&dc->end, k);
    } else {
      const int r = divide_cell(d.g, c, d.dirs[2 * k], d.dirs[2 * k + 1], 0, 0, 0, false);
      if (r < 0) {
        raise_status(d.g.ctl, kETOPO);
        dc->stop = 1;
      }
      flag = (r == 0);
    }
  }
  d.flag[b] = flag;
}

// One block per division of the prefix [start, end): its slots (the made
// divisions before it in the prefix, counted by lane 0), the division
// applied, its outcome recorded.  The last block to finish closes the round:
// slots used, the next window's start, another round while divisions remain.
__global__ void k_div_commit(DivArgs d) {
  DivCtl* dc = d.dc;
  const int b = blockIdx.x, start = dc->start, end = dc->end;
  if (threadIdx.x == 0) {
    if (b == 0 && end == start && start < dc->count && !dc->stop) {
      // the first pending division can only fail by an invalid cell index
      raise_status(d.g.ctl, kEINVAL);
      dc->stop = 1;
    }
    const int k = start + b;
    if (k < end) {
      const int f = d.flag[b];
      d.made[k] = f;
      if (f && !dc->stop) {
        int p = dc->used;
        for (int t = 0; t < b; ++t) p += d.flag[t];
        if (divide_cell(d.g, d.cells[k], d.dirs[2 * k], d.dirs[2 * k + 1], d.cslots[p], d.vslots[2 * p],
                        d.vslots[2 * p + 1]) != 0) {
          raise_status(d.g.ctl, kETOPO);
          dc->stop = 1;
        }
      }
    }
  }
  if (last_block(&dc->done) && threadIdx.x == 0) {
    int made = 0;
    for (int t = 0; t < end - start; ++t) made += d.flag[t];
    dc->used += made;
    dc->start = end;
    dc->round += 1;
    const int more = end < dc->count && !dc->stop && d.g.ctl->status == 0;
    if (more && d.loop) cudaGraphSetConditional(d.loop, 1);
  }
}

// Preferred perimeters P0_c = p0_c sqrt(A0_c); A0_c must be finite and >= 0.
__global__ void k_avm_p0s(AvmArgs g) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.n) return;
  const double a0 = g.a0[c];
  if (!(a0 >= 0.0) || !isfinite(a0)) raise_status(g.ctl, kEINVAL);
  g.P0[c] = g.p0[c] * sqrt(a0);
}

__global__ void k_fill_d(int n, double v, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = v;
}
__global__ void k_fill_u64(int n, unsigned long long v, unsigned long long* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = v;
}

// ---------------------------------------------------------------------------
// Storage order: Hilbert re-sort of the vertex and cell slots (Sec. 2.B).
// A vertex's key is the Hilbert index of its position on a 2^hord_v grid, a
// cell's that of its first vertex on a 2^hord_c grid; freed vertices and
// empty cells take the last key.  A counting sort gives each slot its new
// place (within a key, in the order of the atomic ranks: the storage order is
// not deterministic, the results are); one kernel per kind moves every
// per-slot array and renames the entries.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned grid_coord(double x, double L, unsigned side) {
  const double u = x / L * (double)side;
  const unsigned g = u > 0.0 ? (unsigned)u : 0u;
  return g >= side ? side - 1 : g;
}

__global__ void k_avm_sort_keys(AvmSortArgs g) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int cur = g.ctl->cur;
  const double* hx = g.hx + (size_t)cur * g.V;
  const double* hy = g.hy + (size_t)cur * g.V;
  if (t < g.V) {
    const unsigned side = 1u << g.hord_v;
    int key = (int)(side * side);  // freed
    if (g.by_tag)
      key = g.vtag[t];
    else if (g.vc[3 * t] >= 0)
      key = (int)hilbert_index(g.hord_v, grid_coord(hx[t], g.Lx, side), grid_coord(hy[t], g.Ly, side));
    g.vkey[t] = key;
    g.vrank[t] = atomicAdd(&g.kcount_v[key], 1);
  }
  if (t < g.n) {
    const unsigned side = 1u << g.hord_c;
    int key = (int)(side * side);  // empty
    const int v0 = g.cv[(size_t)t * CG_RING];
    if (g.by_tag)
      key = g.ctag[t];
    else if (g.cc[t] > 0 && (unsigned)v0 < (unsigned)g.V)
      key = (int)hilbert_index(g.hord_c, grid_coord(hx[v0], g.Lx, side), grid_coord(hy[v0], g.Ly, side));
    g.ckey[t] = key;
    g.crank[t] = atomicAdd(&g.kcount_c[key], 1);
  }
}

__global__ void k_avm_sort_perm(AvmSortArgs g) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < g.V) g.vperm[t] = bin_begin(g.kstart_v, g.kpart_v, g.vkey[t]) + g.vrank[t];
  if (t < g.n) g.cperm[t] = bin_begin(g.kstart_c, g.kpart_c, g.ckey[t]) + g.crank[t];
}

__global__ void k_avm_sort_move(AvmSortArgs g) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t V = (size_t)g.V;
  const int cur = g.ctl->cur, alt = cur ^ 1;
  if (t < g.V) {
    const int j = g.vperm[t];
    g.hx_w[alt * V + j] = g.hx[cur * V + t];
    g.hy_w[alt * V + j] = g.hy[cur * V + t];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int c = g.vc[3 * t + k], w = g.vn[3 * t + k];
      g.vc_s[3 * j + k] = (unsigned)c < (unsigned)g.n ? g.cperm[c] : -1;
      g.vn_s[3 * j + k] = (unsigned)w < (unsigned)g.V ? g.vperm[w] : -1;
    }
    g.vtag_s[j] = g.vtag[t];
  }
  if (t < g.n) {
    const int j = g.cperm[t];
    const int m = g.cc[t];
    g.cc_s[j] = m;
    for (int a = 0; a < CG_RING; ++a) {
      const int v = g.cv[(size_t)t * CG_RING + a];
      g.cv_s[(size_t)j * CG_RING + a] = (a < m && (unsigned)v < (unsigned)g.V) ? g.vperm[v] : -1;
    }
    g.theta_s[j] = g.theta[t];
    g.p0_s[j] = g.p0[t];
    g.v0_s[j] = g.v0[t];
    g.a0_s[j] = g.a0[t];
    g.P0_s[j] = g.P0[t];
    g.ctag_s[j] = g.ctag[t];
  }
}

__global__ void k_avm_sort_finish(AvmSortArgs g) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < g.V) {
    g.vslot[g.vtag[t]] = t;
    g.kcount_v[g.vkey[t]] = 0;
  }
  if (t < g.n) {
    g.cslot[g.ctag[t]] = t;
    g.kcount_c[g.ckey[t]] = 0;
  }
  if (t == 0) g.ctl->cur ^= 1;
}

__global__ void k_iota2(int n, int* a, int* b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = b[i] = i;
}

// The network in tag order with its entries renamed to tags.
__global__ void k_avm_topology_by_tag(AvmArgs g, const int* vslot, const int* cslot, int* vc_out, int* vn_out,
                                      int* cc_out, int* cv_out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < g.V) {
    const int v = vslot[t];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int c = g.vc[3 * v + k], w = g.vn[3 * v + k];
      if (vc_out) vc_out[3 * t + k] = (unsigned)c < (unsigned)g.n ? g.ctag[c] : -1;
      if (vn_out) vn_out[3 * t + k] = (unsigned)w < (unsigned)g.V ? g.vtag[w] : -1;
    }
  }
  if (t < g.n) {
    const int c = cslot[t];
    const int m = g.cc[c];
    if (cc_out) cc_out[t] = m;
    if (cv_out)
      for (int a = 0; a < CG_RING; ++a) {
        const int v = g.cv[(size_t)c * CG_RING + a];
        cv_out[(size_t)t * CG_RING + a] = (a < m && (unsigned)v < (unsigned)g.V) ? g.vtag[v] : -1;
      }
  }
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
constexpr int kAvmThreads = 128;
static inline int blocks_of(int n) { return (n + kAvmThreads - 1) / kAvmThreads; }
// The FP64 step kernels in smaller blocks: 65536 cells make only ~3.4 blocks
// of 128 per SM, and the SMs given one block more set the kernel's time
// (measured best: 64 threads for the cells, 32 for the vertices).
constexpr int kAvmCellThreads = 64, kAvmVertexThreads = 32;
static inline int cell_blocks_of(int n) { return (n + kAvmCellThreads - 1) / kAvmCellThreads; }
static inline int vertex_blocks_of(int n) { return (n + kAvmVertexThreads - 1) / kAvmVertexThreads; }

void launch_avm_move(const AvmArgs& a, cudaStream_t st, int part) {
  AvmArgs m = a;
  m.move = 1;
  if (part != 2) k_avm_cells<<<cell_blocks_of(a.n), kAvmCellThreads, 0, st>>>(m);
  if (part != 1) k_avm_force_move<<<vertex_blocks_of(a.V), kAvmVertexThreads, 0, st>>>(m);
}
void launch_avm_dir(const AvmArgs& a, cudaStream_t st) {
  k_avm_dir<<<cell_blocks_of(a.n), kAvmCellThreads, 0, st>>>(a);
}
void launch_avm_begin_t1(Ctl* ctl, cudaStream_t st) { k_avm_begin_t1<<<1, 1, 0, st>>>(ctl); }
void launch_avm_t1_pass(const AvmArgs& a, cudaStream_t st) {
  k_t1_propose<<<blocks_of(a.V), kAvmThreads, 0, st>>>(a);
  k_t1_apply<<<a.apply_blocks, kApplyThreads, 0, st>>>(a);
}
void launch_avm_shadow(const AvmArgs& a, cudaStream_t st) {
  k_avm_shadow<<<blocks_of(a.V), kAvmThreads, 0, st>>>(a);
}
void launch_avm_forces(const AvmArgs& a, cudaStream_t st) {
  AvmArgs f = a;
  f.move = 0;
  k_avm_cells<<<cell_blocks_of(a.n), kAvmCellThreads, 0, st>>>(f);
  k_avm_force_move<<<vertex_blocks_of(a.V), kAvmVertexThreads, 0, st>>>(f);
}
void launch_avm_divide_slots(const DivArgs& d, const int* cslot, const int* vslot, int* fc, int* sc, int* scp,
                             int* fv, int* sv, int* svp, cudaStream_t st) {
  const int blocks = blocks_of(d.g.V);  // V = 2n covers the cells too
  k_div_free_flags<<<blocks, kAvmThreads, 0, st>>>(d.g, cslot, vslot, fc, fv);
  CellListArgs sc_args{};
  sc_args.ctl = d.g.ctl;
  sc_args.n = d.g.n;
  sc_args.nbins = d.g.n;
  sc_args.bin_count = fc;
  sc_args.bin_start = sc;
  sc_args.scan_partials = scp;
  launch_scan(sc_args, st);
  sc_args.n = d.g.V;
  sc_args.nbins = d.g.V;
  sc_args.bin_count = fv;
  sc_args.bin_start = sv;
  sc_args.scan_partials = svp;
  launch_scan(sc_args, st);
  k_div_free_list<<<blocks, kAvmThreads, 0, st>>>(d, cslot, vslot, fc, sc, scp, fv, sv, svp);
}
void launch_avm_divide_begin(const DivArgs& d, cudaStream_t st) {
  cudaMemsetAsync(d.dlock, 0xff, (size_t)d.g.n * sizeof(unsigned long long), st);
  cudaMemsetAsync(d.made, 0, (size_t)d.g.n * sizeof(int), st);
  k_div_begin<<<1, 1, 0, st>>>(d);
}
void launch_avm_divide_round(const DivArgs& d, cudaStream_t st) {
  k_div_lock<<<kDivWindow / kDivLockThreads, kDivLockThreads, 0, st>>>(d);
  k_div_check_dry<<<kDivWindow, 32, 0, st>>>(d);
  k_div_commit<<<kDivWindow, 32, 0, st>>>(d);
}
void launch_avm_sort(const AvmSortArgs& a, cudaStream_t st) {
  const int blocks = blocks_of(a.V);  // V = 2n covers the cells too
  k_avm_sort_keys<<<blocks, kAvmThreads, 0, st>>>(a);
  CellListArgs sc{};
  sc.ctl = a.ctl;
  sc.n = a.V;
  sc.nbins = a.by_tag ? a.V : (1 << (2 * a.hord_v)) + 1;
  sc.bin_count = a.kcount_v;
  sc.bin_start = a.kstart_v;
  sc.scan_partials = a.kpart_v;
  launch_scan(sc, st);
  sc.n = a.n;
  sc.nbins = a.by_tag ? a.n : (1 << (2 * a.hord_c)) + 1;
  sc.bin_count = a.kcount_c;
  sc.bin_start = a.kstart_c;
  sc.scan_partials = a.kpart_c;
  launch_scan(sc, st);
  k_avm_sort_perm<<<blocks, kAvmThreads, 0, st>>>(a);
  k_avm_sort_move<<<blocks, kAvmThreads, 0, st>>>(a);
  const size_t V = (size_t)a.V, n = (size_t)a.n;
  cudaMemcpyAsync(a.vc, a.vc_s, 3 * V * sizeof(int), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(a.vn, a.vn_s, 3 * V * sizeof(int), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(a.vtag, a.vtag_s, V * sizeof(int), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(a.cc, a.cc_s, n * sizeof(int), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(a.cv, a.cv_s, n * CG_RING * sizeof(int), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(a.ctag, a.ctag_s, n * sizeof(int), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(a.theta, a.theta_s, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(a.p0, a.p0_s, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(a.v0, a.v0_s, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(a.a0, a.a0_s, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(a.P0, a.P0_s, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  k_avm_sort_finish<<<blocks, kAvmThreads, 0, st>>>(a);
}
void launch_iota2(int n, int* tags, int* slots, cudaStream_t st) {
  if (n > 0) k_iota2<<<(n + 255) / 256, 256, 0, st>>>(n, tags, slots);
}
void launch_avm_topology_by_tag(const AvmArgs& a, const int* vslot, const int* cslot, int* vc_out, int* vn_out,
                                int* cc_out, int* cv_out, cudaStream_t st) {
  k_avm_topology_by_tag<<<blocks_of(a.V), kAvmThreads, 0, st>>>(a, vslot, cslot, vc_out, vn_out, cc_out, cv_out);
}
void launch_avm_p0s(const AvmArgs& a, cudaStream_t st) {
  k_avm_p0s<<<blocks_of(a.n), kAvmThreads, 0, st>>>(a);
}
void launch_avm_validate(const AvmArgs& a, cudaStream_t st) {
  k_avm_validate<<<blocks_of(a.V), kAvmThreads, 0, st>>>(a);
}
void launch_fill_d(int n, double v, double* out, cudaStream_t st) {
  if (n > 0) k_fill_d<<<(n + 255) / 256, 256, 0, st>>>(n, v, out);
}
void launch_fill_u64(int n, unsigned long long v, unsigned long long* out, cudaStream_t st) {
  if (n > 0) k_fill_u64<<<(n + 255) / 256, 256, 0, st>>>(n, v, out);
}

}  // namespace cgk
