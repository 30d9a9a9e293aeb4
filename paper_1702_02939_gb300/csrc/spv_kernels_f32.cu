// SPV step kernels in single precision: geometry + force sets, net force +
// move, and the director terms, with every floating-point operation of the
// physics in FP32 (Sussman, arXiv 1702.02939: the code builds in single or
// double precision and times both, Sec. 3 and Fig. 2).
//
// What stays exact: positions live on the dyadic grid as int64 (the move is
// accumulated and rounded to the grid in FP64), and the circumcircle test and
// repair decide every predicate exactly in integer arithmetic, so the
// triangulation of a given state is the same as in double precision.  What
// changes: A, P, the forces, n(theta) and the noise carry FP32 rounding
// (relative 2^-24 per operation).  On GB300 the FP32 pipe issues about 74
// times as many operations per clock as the FP64 pipe.
//
// Same formulas and layouts as the FP64 kernels (spv_kernels.cu), in real
// units: the per-slot arrays fs, s, w hold float2 values in the first half of
// their double2 buffers.
#include "cg_device.cuh"
#include "cg_kernels.h"

namespace cgk {

namespace {

__device__ __forceinline__ float2* as_f2(double2* p) { return reinterpret_cast<float2*>(p); }
__device__ __forceinline__ const float2* as_f2(const double2* p) { return reinterpret_cast<const float2*>(p); }

// Relative position of cell j seen from cell i: exact grid difference
// (minimum image) and its float value in real units (relative error
// <= 2u + u^2).
__device__ __forceinline__ void rel_f(const Rep& R, const long long* X, const long long* Y, long long Xi,
                                      long long Yi, int j, float sc, long long& gx, long long& gy, float& dx,
                                      float& dy) {
  gx = min_image_i(X[j] - Xi, R.LX);
  gy = min_image_i(Y[j] - Yi, R.LY);
  dx = i2f_scaled(gx, sc);
  dy = i2f_scaled(gy, sc);
}

// (a x b) in real units from the exact grid coordinates: the 128-bit
// determinant, then to float.  A float determinant of the rounded relative
// positions can vanish for two nearly coincident neighbours; this one is the
// exact value rounded once (positive for every triangle of the triangulation).
__device__ __forceinline__ float det_f(long long ax, long long ay, long long bx, long long by, float sc) {
  const __int128 d = (__int128)ax * by - (__int128)ay * bx;
  const bool neg = d < 0;
  const unsigned __int128 m = neg ? (unsigned __int128)(-d) : (unsigned __int128)d;
  const unsigned long long hi = (unsigned long long)(m >> 64), lo = (unsigned long long)m;
  // hi * 2^64 + lo with hi < 2^63; the low half enters as 2 (lo >> 1) (its last
  // bit is below the float resolution); relative error ~3u
  const float f = i2f_scaled((long long)hi, 0x1p64f * sc * sc) + i2f_scaled((long long)(lo >> 1), 2.0f * sc * sc);
  return neg ? -f : f;
}

}  // namespace

// One thread per cell (grid-stride; optional list of cells; tolerant mode for
// the pass beside the repair rounds), as k_geom.
__global__ void __launch_bounds__(kGeomThreads) k_geom_f32(GeomArgs g) {
  __shared__ float sh_hx[CG_RING][kGeomThreads];
  __shared__ float sh_hy[CG_RING][kGeomThreads];
  __shared__ float sh_ex[CG_RING][kGeomThreads];  // unit vector of the edge ending at vertex a
  __shared__ float sh_ey[CG_RING][kGeomThreads];
  const int t = threadIdx.x;
  const size_t N = (size_t)g.n;
  const int cur = g.ctl->cur;
  const long long* __restrict__ X = g.X + (size_t)cur * N;
  const long long* __restrict__ Y = g.Y + (size_t)cur * N;
  float2* fs = as_f2(g.fs);
  float2* sv = as_f2(g.s);
  float2* wv = as_f2(g.w);
  const int total = g.list ? *g.list_count : g.n;
  for (int item = blockIdx.x * kGeomThreads + t; item < total; item += gridDim.x * kGeomThreads) {
    const int i = g.list ? g.list[item] : (g.order ? g.order[item] : item);
    if (g.list_bits) atomicAnd(&g.list_bits[i >> 5], ~(1u << (i & 31)));
    const Rep R = g.reps[g.rep[i]];
    const float sc = (float)R.inv_scale;
    const long long Xi = X[i], Yi = Y[i];
    const int m = g.cnt[i];
    if (m < 3 || m > CG_RING) {
      if (!g.tolerant) raise_status(g.ctl, kETOPO);
      continue;
    }
    const int* ring = g.nbr + (size_t)i * CG_RING;
    auto nb = [&](int a) {
      const int j = ring[a];
      return ((unsigned)j < (unsigned)g.n) ? j : i;
    };
    long long g0x, g0y;
    float d0x, d0y;
    rel_f(R, X, Y, Xi, Yi, nb(0), sc, g0x, g0y, d0x, d0y);
    const float l0 = d0x * d0x + d0y * d0y;
    float ax = d0x, ay = d0y, la = l0;
    long long gax = g0x, gay = g0y;
    float hpx = 0.f, hpy = 0.f, h0x = 0.f, h0y = 0.f;
    float area = 0.f, per = 0.f;
    for (int a = 0; a < m; ++a) {
      float bx, by, lb;
      long long gbx, gby;
      if (a + 1 < m) {
        rel_f(R, X, Y, Xi, Yi, nb(a + 1), sc, gbx, gby, bx, by);
        lb = bx * bx + by * by;
      } else {
        bx = d0x; by = d0y; lb = l0;
        gbx = g0x; gby = g0y;
      }
      const float det = det_f(gax, gay, gbx, gby, sc);  // (r_j - r_i) x (r_k - r_i)
      const float r = 1.0f / det;
      const float hr = 0.5f * r;
      const float hx = (by * la - ay * lb) * hr;  // circumcentre relative to r_i
      const float hy = (ax * lb - bx * la) * hr;
      sv[a * N + i] = make_float2(hx * r, hy * r);
      wv[a * N + i] = make_float2(by - ay, ax - bx);
      sh_hx[a][t] = hx;
      sh_hy[a][t] = hy;
      if (a == 0) {
        h0x = hx; h0y = hy;
      } else {
        area += hpx * hy - hx * hpy;
        const float ex = hx - hpx, ey = hy - hpy;
        const float l2 = ex * ex + ey * ey;
        const float il = l2 > 0.f ? rsqrtf(l2) : 0.f;  // a zero-length edge has no direction
        per += l2 * il;
        sh_ex[a][t] = ex * il;
        sh_ey[a][t] = ey * il;
      }
      hpx = hx; hpy = hy;
      ax = bx; ay = by; la = lb;
      gax = gbx; gay = gby;
    }
    {  // closing edge h_{m-1} -> h_0 is the incoming edge of vertex 0
      area += hpx * h0y - h0x * hpy;
      const float ex = h0x - hpx, ey = h0y - hpy;
      const float l2 = ex * ex + ey * ey;
      const float il = l2 > 0.f ? rsqrtf(l2) : 0.f;
      per += l2 * il;
      sh_ex[0][t] = ex * il;
      sh_ey[0][t] = ey * il;
    }
    const float A = 0.5f * area, P = per;
    g.A[i] = A;
    g.P[i] = P;
    const float dA = A - (float)g.A0, dP = P - (float)(g.p0[i] * g.sqrtA0);
    if (g.energy_out) g.energy_out[i] = (double)((float)g.KA * dA * dA + (float)g.KP * dP * dP);
    // dA/dh = 1/2 perp(h_next - h_prev); dP/dh = e_in - e_out
    const float ka = (float)g.KA * dA, kp = 2.0f * (float)g.KP * dP;
    for (int a = 0; a < m; ++a) {
      const int ap = (a == 0) ? m - 1 : a - 1;
      const int an = (a + 1 == m) ? 0 : a + 1;
      const float gx = sh_hy[an][t] - sh_hy[ap][t], gy = sh_hx[ap][t] - sh_hx[an][t];
      const float dPx = sh_ex[a][t] - sh_ex[an][t], dPy = sh_ey[a][t] - sh_ey[an][t];
      fs[a * N + i] = make_float2(fmaf(ka, gx, kp * dPx), fmaf(ka, gy, kp * dPy));
    }
  }
}

// Net force on cell i in FP32 from the float force sets (false for a
// malformed ring: status raised, or, in the tolerant pass beside the repair
// rounds, nothing raised and the cell left to the fix-up).
__device__ __forceinline__ bool net_force_f32(const ForceArgs& g, int i, float& fx_out, float& fy_out) {
  const size_t N = (size_t)g.n;
  const float2* fs = as_f2(g.fs);
  const float2* sv = as_f2(g.s);
  const float2* wv = as_f2(g.w);
  const int m = g.cnt[i];
  if (m < 3 || m > CG_RING) {
    if (!g.tolerant) raise_status(g.ctl, kETOPO);
    return false;
  }
  const int* ring = g.nbr + (size_t)i * CG_RING;
  bool bad = false;
  auto nb = [&](int a) {  // a ring being rewritten may hold -1 entries
    const int j = ring[a];
    const bool ok = (unsigned)j < (unsigned)g.n;
    bad |= !ok;
    return ok ? j : i;
  };
  int jfirst = nb(0);
  int pfirst = ring_pos(g.nbr, g.cnt, jfirst, i);
  int j = jfirst, pj = pfirst;
  float fx = 0.f, fy = 0.f;
  bad |= pfirst < 0;
  for (int a = 0; a < m; ++a) {
    int k, pk;
    if (a + 1 < m) {
      k = nb(a + 1);
      pk = ring_pos(g.nbr, g.cnt, k, i);
      bad |= pk < 0;
    } else {
      k = jfirst;
      pk = pfirst;
    }
    const int mj = g.cnt[j];
    const int bj = (pj <= 0) ? (mj > 0 ? mj - 1 : 0) : pj - 1;
    const float2 f0 = fs[a * N + i];
    const float2 f1 = fs[(size_t)bj * N + j];
    const float2 f2 = fs[(size_t)(pk < 0 ? 0 : pk) * N + k];
    const float Gx = f0.x + f1.x + f2.x, Gy = f0.y + f1.y + f2.y;
    const float2 s = sv[a * N + i], w = wv[a * N + i];
    const float c = w.x * Gx + w.y * Gy;
    fx -= s.x * c;
    fy -= s.y * c;
    j = k;
    pj = pk;
  }
  if (bad) {
    if (g.tolerant) return false;
    raise_status(g.ctl, kETOPO);
  }
  fx_out = fx;
  fy_out = fy;
  return true;
}

// Cell i's net force and, as in k_force, the move of Eq. 3 accumulated in
// FP64 and rounded to the grid (integrate 2: the move alone from the stored
// forces, which hold the FP32 values exactly).
__device__ __forceinline__ void force_cell_f32(const ForceArgs& g, int i) {
  const size_t N = (size_t)g.n;
  float fx, fy;
  if (g.integrate == 2) {
    fx = (float)g.Fx[i];
    fy = (float)g.Fy[i];
  } else {
    if (!net_force_f32(g, i, fx, fy)) {
      if (g.tolerant) claim_fix(g.fix_bits, g.fix_list, &g.ctl->force_count, i);
      return;
    }
    g.Fx[i] = fx;
    g.Fy[i] = fy;
    if (!g.integrate) return;
  }

  const int cur = g.ctl->cur;
  const Rep R = g.reps[g.rep[i]];
  const double xi = g.x[(size_t)cur * N + i], yi = g.y[(size_t)cur * N + i];
  const double2 nd = g.nrm[i];  // (cos theta, sin theta), from k_dir_f32
  double v0;
  if (g.v0_user) {  // integrate 2 with new speeds: take them over first
    v0 = g.v0_user[g.tag[i]];
    if (!isfinite(v0)) raise_status(g.ctl, kEINVAL);
    g.v0[i] = v0;
  } else {
    v0 = g.v0[i];
  }
  const double vx = g.mu * (double)fx + v0 * nd.x, vy = g.mu * (double)fy + v0 * nd.y;
  const double xn = fma(g.dt, vx, xi), yn = fma(g.dt, vy, yi);
  long long Xn, Yn;
  if (isfinite(xn) && isfinite(yn)) {
    if (!R.framed) {
      Xn = wrap_to_grid(xn, R.Lx, R.scale, R.LX);
      Yn = wrap_to_grid(yn, R.Ly, R.scale, R.LY);
    } else {
      Xn = move_framed(xi, g.dt, vx, R.x0, R.Lxg, R.scale, R.X0, R.LXg, R.LX);
      Yn = move_framed(yi, g.dt, vy, R.y0, R.Lyg, R.scale, R.Y0, R.LYg, R.LY);
    }
  } else {
    if (g.tolerant) {  // decided again, strictly, after the repair rounds
      claim_fix(g.fix_bits, g.fix_list, &g.ctl->force_count, i);
      return;
    }
    raise_status(g.ctl, kENONFINITE);
    Xn = (long long)rint(xi * R.scale);
    Yn = (long long)rint(yi * R.scale);
  }
  const int nxt = cur ^ 1;
  g.x[(size_t)nxt * N + i] = i2d_exact(Xn) * R.inv_scale;
  g.y[(size_t)nxt * N + i] = i2d_exact(Yn) * R.inv_scale;
  g.X[(size_t)nxt * N + i] = Xn;
  g.Y[(size_t)nxt * N + i] = Yn;
}

// One thread per cell, or grid-stride over a list (bits cleared), as k_force.
__global__ void __launch_bounds__(kForceThreads) k_force_f32(ForceArgs g) {
  const int total = g.list ? *g.list_count : g.n;
  for (int item = blockIdx.x * kForceThreads + threadIdx.x; item < total; item += gridDim.x * kForceThreads) {
    const int i = g.list ? g.list[item] : (g.order ? g.order[item] : item);
    if (g.list_bits) atomicAnd(&g.list_bits[i >> 5], ~(1u << (i & 31)));
    force_cell_f32(g, i);
  }
}

// Director terms in FP32: n(theta) of the float director, and the noise from
// the same Philox words as director_noise, with 24-bit uniforms
// u = (top 24 bits + 1) 2^-24 and xi = sqrt(-2 ln u1) cos(2 pi u2).
__global__ void k_dir_f32(DirArgs g) {
  const long long step = g.ctl->step;
  const uint2 key = make_uint2((unsigned)g.seed, (unsigned)(g.seed >> 32));
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += gridDim.x * blockDim.x) {
    double th = g.theta[i];
    if (g.advance) {
      th = th + g.noise_amp * g.xi[i];
      g.theta[i] = th;
    }
    float sn, cs;
    sincosf((float)th, &sn, &cs);
    g.nrm[i] = make_double2(cs, sn);
    const uint4 r = philox_10(make_uint4((unsigned)g.tag[i], (unsigned)(unsigned long long)step,
                                         (unsigned)((unsigned long long)step >> 32), 0u),
                              key);
    const float u1 = (float)((r.x >> 8) + 1u) * 0x1p-24f;
    const float u2 = (float)((r.z >> 8) + 1u) * 0x1p-24f;
    g.xi[i] = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
  }
}

void launch_geom_f32(const GeomArgs& a, cudaStream_t st, int blocks) {
  if (a.n <= 0) return;
  const int full = (a.n + kGeomThreads - 1) / kGeomThreads;
  k_geom_f32<<<(blocks > 0 && blocks < full) ? blocks : full, kGeomThreads, 0, st>>>(a);
}
void launch_force_f32(const ForceArgs& a, cudaStream_t st, int blocks) {
  if (a.n <= 0) return;
  const int full = (a.n + kForceThreads - 1) / kForceThreads;
  k_force_f32<<<(blocks > 0 && blocks < full) ? blocks : full, kForceThreads, 0, st>>>(a);
}
void launch_dir_f32(const DirArgs& a, cudaStream_t st, int blocks) {
  if (a.n <= 0) return;
  const int full = (a.n + 127) / 128;
  k_dir_f32<<<(blocks > 0 && blocks < full) ? blocks : full, 128, 0, st>>>(a);
}

}  // namespace cgk
