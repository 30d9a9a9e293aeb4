// SPV step kernels: geometry + force sets, net force + update, Delaunay test.
//
// Sussman, arXiv 1702.02939:
//  * geometry of every cell from the circumcentres of its Delaunay triangles
//    (Sec. 2.C.1); areas, perimeters, E of Eq. 1
//  * "force sets" dE_c/dh per (cell, vertex) (Sec. 2.C.2, Eqs. A3-A5) and the
//    net force F_i = -sum_t (dh_t/dr_i)^T G_t (Eqs. A6-A7)
//  * displacement by Eq. 3 and director rotation (Sec. 2.C.3)
//  * empty-circumcircle test of the triangulation (Sec. 2.C.3)
//
// GB300 design notes: the path is bound by the FP64 pipe (about 1/74 of the
// FP32 rate), so FP64 is spent only on the physics.  The Jacobian dh/dr_i is
// used in its rank-one form J = w u^T / det (u = h - r_i, w = perp(r_k - r_j),
// det = (r_j - r_i) x (r_k - r_i)), which follows from differentiating the
// equidistance conditions |h - r_i| = |h - r_j| = |h - r_k| and equals the
// matrix of Eq. A16.  All predicates run on the FP32/integer pipes.
#include "cg_device.cuh"
#include "cg_kernels.h"
#include <algorithm>

namespace cgk {

// One thread per cell.  Writes A, P, force sets fs[a][i] = dE_i/dh_a, and the
// per-slot Jacobian factor s[a][i] = 2 u_a / det_a (the other factor, w_a / 2,
// is rebuilt exactly from the integer positions by k_force).
//
// The geometry runs in grid units (coordinates x 2^q): relative positions come
// exactly from the int64 grid coordinates, and the powers of two cancel in the
// force (u/det scales as 2^q, w as 2^-q) or fold into one factor per cell
// (A x 2^-2q, P x 2^-q, dA/dh x 2^-q).  The circumcentres are kept doubled,
// g_a = 2 h_a = num / det: every use is homogeneous in h, so the factor 2
// (exact) folds into the per-cell constants (A x 1/4, P x 1/2, dA/dh x 1/2,
// s x 2 against w / 2) and the results equal those of h itself bit for bit.
// Integer-to-double conversions run on the integer pipes (i2d_int).
//
// Per ring slot the kernel keeps the circumcentre and the unit vector of the
// edge ending there for the force-set pass: the first kGeomSh slots in shared
// memory (10 KB per one-warp block, so that 20 blocks fit on an SM), the
// slots of longer rings (rare) in local memory.
__global__ void __launch_bounds__(kGeomThreads, kGeomMinBlocks) k_geom(GeomArgs g) {
  __shared__ double sh_hx[kGeomSh][kGeomThreads];
  __shared__ double sh_hy[kGeomSh][kGeomThreads];
  __shared__ double sh_ex[kGeomSh][kGeomThreads];  // unit vector of the edge ending at vertex a
  __shared__ double sh_ey[kGeomSh][kGeomThreads];
  constexpr int kLo = (CG_RING > kGeomSh) ? CG_RING - kGeomSh : 1;
  double lo_hx[kLo], lo_hy[kLo], lo_ex[kLo], lo_ey[kLo];
  const int t = threadIdx.x;
  auto put = [&](double (&sh)[kGeomSh][kGeomThreads], double* lo, int a, double v) {
    if (a < kGeomSh) sh[a][t] = v;
    else lo[a - kGeomSh] = v;
  };
  auto get = [&](const double (&sh)[kGeomSh][kGeomThreads], const double* lo, int a) -> double {
    return (a < kGeomSh) ? sh[a][t] : lo[a - kGeomSh];
  };
  const size_t N = (size_t)g.n;
  const int cur = g.ctl->cur;
  const long long* __restrict__ X = g.X + (size_t)cur * N;
  const long long* __restrict__ Y = g.Y + (size_t)cur * N;
  const int total = g.list ? *g.list_count : g.n;
  for (int item = blockIdx.x * kGeomThreads + t; item < total; item += gridDim.x * kGeomThreads) {
    const int i = g.list ? g.list[item] : (g.order ? g.order[item] : item);
    if (g.list_bits) atomicAnd(&g.list_bits[i >> 5], ~(1u << (i & 31)));
    const Rep R = g.reps[g.rep[i]];
    const long long Xi = X[i], Yi = Y[i];
    const int m = g.cnt[i];
    if (m < 3 || m > CG_RING) {
      if (!g.tolerant) raise_status(g.ctl, kETOPO);
      continue;
    }
    const int* ring = g.nbr + (size_t)i * CG_RING;
    // a ring being rewritten concurrently may hold -1 entries: read the cell
    // itself there (the result is discarded and computed again)
    auto nb = [&](int a) {
      const int j = ring[a];
      return ((unsigned)j < (unsigned)g.n) ? j : i;
    };

    // squared lengths and the triangle determinants exactly in 128-bit
    // integers from the grid offsets; the doubled circumcentre g = num / det
    // with num = (b_y |a|^2 - a_y |b|^2, a_x |b|^2 - b_x |a|^2) in 128-bit
    // integers too, from |a|^2 and |b|^2 cut to 62 significant bits by a
    // shift common to the triangle (at least as accurate as FP64 products
    // of the rounded squares), each rounded to double once
    const int j0 = nb(0);
    const long long D0X = min_image_i(X[j0] - Xi, R.LX), D0Y = min_image_i(Y[j0] - Yi, R.LY);
    const unsigned __int128 L0 = (unsigned __int128)((__int128)D0X * D0X + (__int128)D0Y * D0Y);
    unsigned __int128 LA = L0;
    long long AX = D0X, AY = D0Y;
    double hpx = 0.0, hpy = 0.0, h0x = 0.0, h0y = 0.0;
    double area = 0.0, per = 0.0;
    for (int a = 0; a < m; ++a) {
      long long BX, BY;
      unsigned __int128 LB;
      if (a + 1 < m) {
        const int j = nb(a + 1);
        BX = min_image_i(X[j] - Xi, R.LX);
        BY = min_image_i(Y[j] - Yi, R.LY);
        LB = (unsigned __int128)((__int128)BX * BX + (__int128)BY * BY);
      } else {
        BX = D0X; BY = D0Y; LB = L0;
      }
      // (r_j - r_i) x (r_k - r_i)
      const double det = i128_to_double((__int128)AX * BY - (__int128)AY * BX);
      const double r = fx_rcp(det);
      // |offsets| < 2^49 and the cut squares < 2^62: the numerators fit in 113 bits
      const int S = max(u128_bits(LA > LB ? LA : LB) - 62, 0);
      const long long la = (long long)(LA >> S), lb = (long long)(LB >> S);
      const double hx = i128_to_double((__int128)BY * la - (__int128)AY * lb, S) * r;
      const double hy = i128_to_double((__int128)AX * lb - (__int128)BX * la, S) * r;
      g.s[a * N + i] = make_double2(hx * r, hy * r);
      put(sh_hx, lo_hx, a, hx);
      put(sh_hy, lo_hy, a, hy);
      if (a == 0) {
        h0x = hx; h0y = hy;
      } else {
        area = fma(-hx, hpy, fma(hpx, hy, area));  // shoelace term, two FMAs
        const double ex = hx - hpx, ey = hy - hpy;
        const double l2 = ex * ex + ey * ey;
        const double il = (__double_as_longlong(l2) > 0) ? fx_rsqrt(l2) : 0.0;  // zero-length edge: no direction
        per += l2 * il;
        put(sh_ex, lo_ex, a, ex * il);
        put(sh_ey, lo_ey, a, ey * il);
      }
      hpx = hx; hpy = hy;
      LA = LB;
      AX = BX; AY = BY;
    }
    {  // closing edge h_{m-1} -> h_0 is the incoming edge of vertex 0
      area = fma(-h0x, hpy, fma(hpx, h0y, area));
      const double ex = h0x - hpx, ey = h0y - hpy;
      const double l2 = ex * ex + ey * ey;
      const double il = (__double_as_longlong(l2) > 0) ? fx_rsqrt(l2) : 0.0;  // zero-length edge: no direction
      per += l2 * il;
      sh_ex[0][t] = ex * il;
      sh_ey[0][t] = ey * il;
    }
    const double sc = R.inv_scale;
    const double A = 0.125 * area * sc * sc, P = 0.5 * per * sc;
    g.A[i] = A;
    g.P[i] = P;
    const double dA = A - g.A0, dP = P - g.p0[i] * g.sqrtA0;
    if (g.energy_out) g.energy_out[i] = g.KA * dA * dA + g.KP * dP * dP;
    // dA/dh = 1/2 perp(h_next - h_prev) (the 1/2, the doubling of g and the
    // grid scale fold into ka); dP/dh = e_in - e_out (unit edge vectors)
    const double ka = g.KA * dA * (0.5 * sc), kp = 2.0 * g.KP * dP;
    for (int a = 0; a < m; ++a) {
      const int ap = (a == 0) ? m - 1 : a - 1;
      const int an = (a + 1 == m) ? 0 : a + 1;
      const double gx = get(sh_hy, lo_hy, an) - get(sh_hy, lo_hy, ap);
      const double gy = get(sh_hx, lo_hx, ap) - get(sh_hx, lo_hx, an);
      const double dPx = get(sh_ex, lo_ex, a) - get(sh_ex, lo_ex, an);
      const double dPy = get(sh_ey, lo_ey, a) - get(sh_ey, lo_ey, an);
      g.fs[a * N + i] = make_double2(fma(ka, gx, kp * dPx), fma(ka, gy, kp * dPy));
    }
  }
}

// Net force on cell i: G_t = sum over the triangle's three cells of their
// force sets, F_i = -sum_t s_t (w_t . G_t), with s_t = 2 u_t / det_t from
// k_geom and w_t / 2 = perp(r_k - r_j) / 2 rebuilt exactly from the integer
// grid offsets (an exact difference, converted on the integer pipes).  False
// (status raised) for a malformed ring.
__device__ __forceinline__ bool net_force(const ForceArgs& g, int i, double& fx_out, double& fy_out) {
  const size_t N = (size_t)g.n;
  const int m = g.cnt[i];
  if (m < 3 || m > CG_RING) {
    if (!g.tolerant) raise_status(g.ctl, kETOPO);
    return false;
  }
  const int cur = g.ctl->cur;
  const long long* __restrict__ X = g.X + (size_t)cur * N;
  const long long* __restrict__ Y = g.Y + (size_t)cur * N;
  const Rep R = g.reps[g.rep[i]];
  const long long Xi = X[i], Yi = Y[i];
  const int* ring = g.nbr + (size_t)i * CG_RING;
  bool bad = false;
  // a ring being rewritten meanwhile (tolerant pass) may hold -1 entries:
  // the cell itself is read there and the result marked bad
  auto nb = [&](int a) {
    const int j = ring[a];
    const bool ok = (unsigned)j < (unsigned)g.n;
    bad |= !ok;
    return ok ? j : i;
  };
  int jfirst = nb(0);
  int pfirst = ring_pos(g.nbr, g.cnt, jfirst, i);
  int j = jfirst, pj = pfirst;
  const long long fX = min_image_i(X[jfirst] - Xi, R.LX), fY = min_image_i(Y[jfirst] - Yi, R.LY);
  long long aX = fX, aY = fY;
  double fx = 0.0, fy = 0.0;
  bad |= pfirst < 0;
  for (int a = 0; a < m; ++a) {
    int k, pk;
    long long bX, bY;
    if (a + 1 < m) {
      k = nb(a + 1);
      pk = ring_pos(g.nbr, g.cnt, k, i);
      bad |= pk < 0;
      bX = min_image_i(X[k] - Xi, R.LX);
      bY = min_image_i(Y[k] - Yi, R.LY);
    } else {
      k = jfirst;
      pk = pfirst;
      bX = fX;
      bY = fY;
    }
    // triangle (i, j, k) is slot pj-1 around j and slot pk around k
    const int mj = g.cnt[j];
    const int bj = (pj <= 0) ? (mj > 0 ? mj - 1 : 0) : pj - 1;
    const double2 f0 = g.fs[a * N + i];
    const double2 f1 = g.fs[(size_t)bj * N + j];
    const double2 f2 = g.fs[(size_t)(pk < 0 ? 0 : pk) * N + k];
    const double Gx = f0.x + f1.x + f2.x, Gy = f0.y + f1.y + f2.y;
    const double2 s = g.s[a * N + i];
    const double wx = i2d_int(bY - aY, -1), wy = i2d_int(aX - bX, -1);
    const double c = wx * Gx + wy * Gy;
    fx -= s.x * c;
    fy -= s.y * c;
    j = k;
    pj = pk;
    aX = bX;
    aY = bY;
  }
  if (bad) {
    if (g.tolerant) return false;
    raise_status(g.ctl, kETOPO);
  }
  fx_out = fx;
  fy_out = fy;
  return true;
}


// Cell i's net force (integrate 0 or 1) and update of Eq. 3 (integrate 1),
// or the update alone from the stored forces of the current positions
// (integrate 2: after a change of v0).
__device__ __forceinline__ void force_cell(const ForceArgs& g, int i) {
  const size_t N = (size_t)g.n;
  double fx, fy;
  if (g.integrate == 2) {
    fx = g.Fx[i];
    fy = g.Fy[i];
  } else {
    if (!net_force(g, i, fx, fy)) {
      if (g.tolerant) claim_fix(g.fix_bits, g.fix_list, &g.ctl->force_count, i);
      return;
    }
    g.Fx[i] = fx;
    g.Fy[i] = fy;
    if (!g.integrate) return;
  }

  // Eq. 3: r <- r + dt (mu F + v0 n(theta)), rounded to the grid and wrapped
  // into the other position buffer; the director rotation
  // theta <- theta + sqrt(2 D_r dt) xi follows at the start of the next step
  // (k_dir), so the state between steps is (r, theta) of one time.
  const int cur = g.ctl->cur;
  const Rep R = g.reps[g.rep[i]];
  const double xi = g.x[(size_t)cur * N + i], yi = g.y[(size_t)cur * N + i];
  const double2 nd = g.nrm[i];  // (cos theta, sin theta), from k_dir
  double v0;
  if (g.v0_user) {  // integrate 2 with new speeds: take them over first
    v0 = g.v0_user[g.tag[i]];
    if (!isfinite(v0)) raise_status(g.ctl, kEINVAL);
    g.v0[i] = v0;
  } else {
    v0 = g.v0[i];
  }
  const double vx = g.mu * fx + v0 * nd.x, vy = g.mu * fy + v0 * nd.y;
  const double xn = fma(g.dt, vx, xi), yn = fma(g.dt, vy, yi);
  long long X, Y;
  if (isfinite(xn) && isfinite(yn)) {
    if (!R.framed) {
      X = wrap_to_grid(xn, R.Lx, R.scale, R.LX);
      Y = wrap_to_grid(yn, R.Ly, R.scale, R.LY);
    } else {
      X = move_framed(xi, g.dt, vx, R.x0, R.Lxg, R.scale, R.X0, R.LXg, R.LX);
      Y = move_framed(yi, g.dt, vy, R.y0, R.Lyg, R.scale, R.Y0, R.LYg, R.LY);
    }
  } else {
    if (g.tolerant) {  // decided again, strictly, after the repair rounds
      claim_fix(g.fix_bits, g.fix_list, &g.ctl->force_count, i);
      return;
    }
    raise_status(g.ctl, kENONFINITE);
    X = (long long)rint(xi * R.scale);
    Y = (long long)rint(yi * R.scale);
  }
  const int nxt = cur ^ 1;
  g.x[(size_t)nxt * N + i] = i2d_int(X, -R.q);
  g.y[(size_t)nxt * N + i] = i2d_int(Y, -R.q);
  g.X[(size_t)nxt * N + i] = X;
  g.Y[(size_t)nxt * N + i] = Y;
}

// One thread per cell: the net force (integrate 0 or 1) and the update of
// Eq. 3 (integrate 1), or the update alone from the stored forces of the
// current positions (integrate 2: after a change of v0); with a list, the
// cells of the list (grid-stride), their list bits cleared.
__global__ void __launch_bounds__(kForceThreads) k_force(ForceArgs g) {
  const int total = g.list ? *g.list_count : g.n;
  for (int item = blockIdx.x * kForceThreads + threadIdx.x; item < total; item += gridDim.x * kForceThreads) {
    const int i = g.list ? g.list[item] : (g.order ? g.order[item] : item);
    if (g.list_bits) atomicAnd(&g.list_bits[i >> 5], ~(1u << (i & 31)));
    force_cell(g, i);
  }
}

// The fix-up list of the force pass: each rewritten ring's cell and the
// cells of its new ring (their force sets or ring positions changed).
__global__ void k_force_fix_list(ForceFixArgs g) {
  const int total = *g.dirty_count;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int d = g.dirty_list[t];
    if ((unsigned)d >= (unsigned)g.n) continue;
    claim_fix(g.fix_bits, g.fix_list, &g.ctl->force_count, d);
    const int m = min(g.cnt[d], CG_RING);
    for (int a = 0; a < m; ++a) {
      const int j = g.nbr[(size_t)d * CG_RING + a];
      if ((unsigned)j < (unsigned)g.n) claim_fix(g.fix_bits, g.fix_list, &g.ctl->force_count, j);
    }
  }
}

// Director terms of a step: with `advance`, first the rotation of the
// previous step theta <- theta + sqrt(2 D_r dt) xi; then n(theta) and the
// noise xi of this step (Philox counter (tag, step)), grid-stride over cells.
// In the step graph it runs beside the circumcircle test, the cell list and
// the repair rounds, which leave the FP64 pipe idle.
__global__ void k_dir(DirArgs g) {
  const long long step = g.ctl->step;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += gridDim.x * blockDim.x) {
    double th = g.theta[i];
    if (g.advance) {
      th = th + g.noise_amp * g.xi[i];
      g.theta[i] = th;
    }
    double sn, cs;
    dm_sincos(th, g.tab, sn, cs);
    g.nrm[i] = make_double2(cs, sn);
    g.xi[i] = director_noise(g.seed, g.tag[i], step, g.tab);
  }
}
void launch_dir(const DirArgs& a, cudaStream_t st, int blocks) {
  if (a.n <= 0) return;
  const int full = (a.n + 127) / 128;
  k_dir<<<(blocks > 0 && blocks < full) ? blocks : full, 128, 0, st>>>(a);
}

// Table of dir_math.cuh: (sin, cos)(j pi/128) from CUDA's sinpi/cospi (exact
// at multiples of pi/2), then per logarithm interval j the reciprocal of its
// centre and minus its logarithm (exactly 1 and 0 for the interval around 1).
__global__ void k_init_dir_tables(double2* tab) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < 256) {
    tab[j] = make_double2(sinpi(j / 128.0), cospi(j / 128.0));
  } else if (j >= kDirTabQ && j < kDirTabQ + 256) {
    // the same values in Q1.62 (exact: every nonzero entry is above 2^-10)
    const double sn = sinpi((j - kDirTabQ) / 128.0), cs = cospi((j - kDirTabQ) / 128.0);
    reinterpret_cast<longlong2*>(tab)[j] = make_longlong2(__double2ll_rn(sn * 0x1p62), __double2ll_rn(cs * 0x1p62));
  } else if (j < kDirTabQ) {
    const int i = j - 256;
    const double inv =
        (i == kLogOne) ? 1.0 : 1.0 / __longlong_as_double(kLogOff + ((long long)i << 44) + (1LL << 43));
    tab[j] = make_double2(inv, -log(inv));
  }
}
void launch_init_dir_tables(double2* tab, cudaStream_t st) { k_init_dir_tables<<<kDirTabEntries / 128, 128, 0, st>>>(tab); }

__global__ void k_dir_terms(int n, const double* __restrict__ theta, const int* __restrict__ tag,
                            unsigned long long seed, long long step, const double2* __restrict__ tab,
                            double* cs, double* sn, double* xi) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s, c;
    dm_sincos(theta[i], tab, s, c);
    cs[i] = c;
    sn[i] = s;
    xi[i] = director_noise(seed, tag[i], step, tab);
  }
}
void launch_dir_terms(int n, const double* theta, const int* tag, unsigned long long seed, long long step,
                      const double2* tab, double* cs, double* sn, double* xi, cudaStream_t st) {
  if (n <= 0) return;
  const int blocks = (int)std::min<long long>((n + 127) / 128, 152LL * 16);
  k_dir_terms<<<blocks, 128, 0, st>>>(n, theta, tag, seed, step, tab, cs, sn, xi);
}

// Start of the topology phase of a step: the new positions become current,
// the step counter advances and the flagged list is emptied.
__global__ void k_begin_topology(Ctl* ctl, int flip) {
  if (flip) {
    ctl->cur ^= 1;
    ctl->step += 1;
  }
  ctl->count[0] = 0;
  ctl->count[1] = 0;
  ctl->round_count = 0;
  ctl->dirty_count = 0;
  ctl->force_count = 0;
}

__device__ __forceinline__ void flag_cell(unsigned* flags, int* list, int* count, int c) {
  const unsigned bit = 1u << (c & 31);
  const unsigned old = atomicOr(&flags[c >> 5], bit);
  if (!(old & bit)) list[atomicAdd(count, 1)] = c;
}

// One thread per cell: every edge (i, j_a) with i < j_a must be locally
// Delaunay (the far vertex j_{a+1} outside the circle through i, j_{a-1}, j_a)
// and every triangle owned by i (i its smallest index) positively oriented.
// Failing quadruples/triangles flag all their cells.
__device__ __forceinline__ void test_cell(const TestArgs& g, int i, const long long* __restrict__ X,
                                          const long long* __restrict__ Y) {
  const Rep R = g.reps[g.rep[i]];
  const float sc = (float)R.inv_scale;
  const long long Xi = X[i], Yi = Y[i];
  const int m = g.cnt[i];
  if (m < 3 || m > CG_RING) {
    raise_status(g.ctl, kETOPO);
    return;
  }
  const int* ring = g.nbr + (size_t)i * CG_RING;
  // sliding window over (j_{a-1}, j_a, j_{a+1}): grid offsets (exact) and
  // their float values, each converted once
  int jp = ring[m - 1], ja = ring[0];
  long long pX = min_image_i(X[jp] - Xi, R.LX), pY = min_image_i(Y[jp] - Yi, R.LY);
  long long aX = min_image_i(X[ja] - Xi, R.LX), aY = min_image_i(Y[ja] - Yi, R.LY);
  float fpx = i2f_scaled(pX, sc), fpy = i2f_scaled(pY, sc);
  float fax = i2f_scaled(aX, sc), fay = i2f_scaled(aY, sc);
  const long long fX = aX, fY = aY;
  const float ffx = fax, ffy = fay;
  const int jfirst = ja;
  for (int a = 0; a < m; ++a) {
    int jn;
    long long nX, nY;
    float fnx, fny;
    if (a + 1 < m) {
      jn = ring[a + 1];
      nX = min_image_i(X[jn] - Xi, R.LX);
      nY = min_image_i(Y[jn] - Yi, R.LY);
      fnx = i2f_scaled(nX, sc);
      fny = i2f_scaled(nY, sc);
    } else {
      jn = jfirst; nX = fX; nY = fY; fnx = ffx; fny = ffy;
    }
    if (i < ja) {
      // triangle (i, j_{a-1}, j_a) CCW; j_{a+1} must be outside its circle
      int s = incircle0_sign(fpx, fpy, fax, fay, fnx, fny, pX, pY, aX, aY, nX, nY, g.tag, i, jp, ja, jn, sc);
      if (s > 0) {
        flag_cell(g.flags, g.list, &g.ctl->count[0], i);
        flag_cell(g.flags, g.list, &g.ctl->count[0], jp);
        flag_cell(g.flags, g.list, &g.ctl->count[0], ja);
        flag_cell(g.flags, g.list, &g.ctl->count[0], jn);
      }
    }
    if (i < ja && i < jn) {
      if (orient0_sign(fax, fay, fnx, fny, aX, aY, nX, nY) <= 0) {
        flag_cell(g.flags, g.list, &g.ctl->count[0], i);
        flag_cell(g.flags, g.list, &g.ctl->count[0], ja);
        flag_cell(g.flags, g.list, &g.ctl->count[0], jn);
      }
    }
    jp = ja; pX = aX; pY = aY; fpx = fax; fpy = fay;
    ja = jn; aX = nX; aY = nY; fax = fnx; fay = fny;
  }
}

// Grid-stride over cells (a smaller grid leaves room on every SM for the
// FP64 branch that runs beside the test).
__global__ void __launch_bounds__(kTestThreads) k_test(TestArgs g) {
  const size_t N = (size_t)g.n;
  const int cur = g.ctl->cur;
  const long long* __restrict__ X = g.X + (size_t)cur * N;
  const long long* __restrict__ Y = g.Y + (size_t)cur * N;
  for (int item = blockIdx.x * kTestThreads + threadIdx.x; item < g.n; item += gridDim.x * kTestThreads)
    test_cell(g, g.order ? g.order[item] : item, X, Y);
}

// Ring-size grouping of each chunk of kOrderChunk cells (see launch_order):
// a counting sort by min(cnt, CG_RING) in shared memory.  Ranks within a
// size come from shared atomics (their order does not matter: every cell's
// results are computed independently of which thread computes them).
__global__ void __launch_bounds__(256) k_order(int n, const int* __restrict__ cnt, int* __restrict__ order) {
  __shared__ int hist[CG_RING + 1], base[CG_RING + 1];
  const int c0 = blockIdx.x * kOrderChunk;
  const int len = min(kOrderChunk, n - c0);
  if (threadIdx.x <= CG_RING) hist[threadIdx.x] = 0;
  __syncthreads();
  int msz[kOrderChunk / 256];
#pragma unroll
  for (int k = 0; k < kOrderChunk / 256; ++k) {
    const int c = k * 256 + threadIdx.x;
    int m = -1;
    if (c < len) {
      m = cnt[c0 + c];
      m = m < 0 ? 0 : (m > CG_RING ? CG_RING : m);
      atomicAdd(&hist[m], 1);
    }
    msz[k] = m;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int b = 0; b <= CG_RING; ++b) {
      base[b] = acc;
      acc += hist[b];
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kOrderChunk / 256; ++k) {
    const int c = k * 256 + threadIdx.x;
    if (msz[k] >= 0) order[c0 + atomicAdd(&base[msz[k]], 1)] = c0 + c;
  }
}

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------
void launch_order(int n, const int* cnt, int* order, cudaStream_t st) {
  if (n <= 0) return;
  k_order<<<(n + kOrderChunk - 1) / kOrderChunk, 256, 0, st>>>(n, cnt, order);
}
void launch_geom(const GeomArgs& a, cudaStream_t st, int blocks) {
  if (a.n <= 0) return;
  const int full = (a.n + kGeomThreads - 1) / kGeomThreads;
  k_geom<<<(blocks > 0 && blocks < full) ? blocks : full, kGeomThreads, 0, st>>>(a);
}
void launch_force(const ForceArgs& a, cudaStream_t st, int blocks) {
  if (a.n <= 0) return;
  const int full = (a.n + kForceThreads - 1) / kForceThreads;
  k_force<<<(blocks > 0 && blocks < full) ? blocks : full, kForceThreads, 0, st>>>(a);
}
void launch_force_fix_list(const ForceFixArgs& a, int blocks, cudaStream_t st) {
  if (a.n > 0) k_force_fix_list<<<blocks, 128, 0, st>>>(a);
}
void launch_begin_topology(Ctl* ctl, int flip, cudaStream_t st) { k_begin_topology<<<1, 1, 0, st>>>(ctl, flip); }
void launch_test(const TestArgs& a, cudaStream_t st, int blocks) {
  if (a.n <= 0) return;
  const int full = (a.n + kTestThreads - 1) / kTestThreads;
  k_test<<<(blocks > 0 && blocks < full) ? blocks : full, kTestThreads, 0, st>>>(a);
}

}  // namespace cgk
