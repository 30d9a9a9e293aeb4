// Backward pass of the SPV step: Hessian-vector products and parameter
// cotangents (Sussman, arXiv 1702.02939, Eq. 3 with forces of Eqs. A6-A16).
//
// With the director noise replayed from the seed, the step map is
//   r' = r + dt (mu F(r) + v0 n(theta)),  F = -grad E,
// whose transposed Jacobian is I - dt mu H(r), H the symmetric Hessian of E.
// Reverse accumulation therefore needs H g for the running cotangent g; it is
// computed here as the forward-mode derivative of -F along g on the frozen
// topology of the step.  The tangent of every geometric quantity follows from
// the definitions:
//   circumcentre u of (0, a, b):  u.a = |a|^2/2, u.b = |b|^2/2
//       => [a; b] udot = [(a-u).adot; (b-u).bdot]
//   A = 1/2 sum u_a x u_{a+1},  P = sum |e_a|, e_a = u_a - u_{a-1}
//   edot-hat = (edot - e^ (e^.edot)) / |e|
//   force sets fs = ka/2 perp(u_next - u_prev) + kp (e^_a - e^_next)
//   net force  F_i = -sum_a s_a (w_a . G_a), s = u/det, w = perp(b - a).
// Parameter cotangents use the same tangents of A and P along g:
//   dL/dp0_i += dt mu 2 K_P sqrt(A0) Pdot_i
//   dL/dK_A  += -dt mu sum_c 2 (A_c - A0) Adot_c
//   dL/dK_P  += -dt mu sum_c 2 (P_c - P0_c) Pdot_c
//   dL/dv0_i += dt g_i . n(theta_i)
#include "cg_device.cuh"
#include "cg_kernels.h"

namespace cgk {

constexpr int kJvpThreads = 32;

__device__ __forceinline__ double i2d_exact_a(long long v) {
  return __longlong_as_double(0x4338000000000000LL + v) - 0x1.8p52;
}

__global__ void __launch_bounds__(kJvpThreads) k_geom_jvp(JvpArgs g) {
  __shared__ double s_ux[CG_RING][kJvpThreads], s_uy[CG_RING][kJvpThreads];
  __shared__ double s_vx[CG_RING][kJvpThreads], s_vy[CG_RING][kJvpThreads];  // udot
  __shared__ double s_ex[CG_RING][kJvpThreads], s_ey[CG_RING][kJvpThreads];  // unit edge ending at a
  __shared__ double s_fx[CG_RING][kJvpThreads], s_fy[CG_RING][kJvpThreads];  // its tangent
  const int t = threadIdx.x;
  const int i = blockIdx.x * kJvpThreads + t;
  if (i >= g.n) return;
  const size_t N = (size_t)g.n;
  const int cur = g.ctl->cur;
  const long long* __restrict__ X = g.X + (size_t)cur * N;
  const long long* __restrict__ Y = g.Y + (size_t)cur * N;
  const Rep R = g.reps[g.rep[i]];
  const double sc = R.inv_scale;
  const long long Xi = X[i], Yi = Y[i];
  const int m = g.cnt[i];
  if (m < 3 || m > CG_RING) {
    raise_status(g.ctl, kETOPO);
    return;
  }
  const int* ring = g.nbr + (size_t)i * CG_RING;
  const double2 vi = g.v[i];

  const int j0 = ring[0];
  const double d0x = i2d_exact_a(min_image_i(X[j0] - Xi, R.LX)) * sc;
  const double d0y = i2d_exact_a(min_image_i(Y[j0] - Yi, R.LY)) * sc;
  const double2 v0 = g.v[j0];
  const double t0x = v0.x - vi.x, t0y = v0.y - vi.y;
  double ax = d0x, ay = d0y, adx = t0x, ady = t0y;
  for (int a = 0; a < m; ++a) {
    double bx, by, bdx, bdy;
    if (a + 1 < m) {
      const int j = ring[a + 1];
      bx = i2d_exact_a(min_image_i(X[j] - Xi, R.LX)) * sc;
      by = i2d_exact_a(min_image_i(Y[j] - Yi, R.LY)) * sc;
      const double2 vj = g.v[j];
      bdx = vj.x - vi.x;
      bdy = vj.y - vi.y;
    } else {
      bx = d0x; by = d0y; bdx = t0x; bdy = t0y;
    }
    const double la = ax * ax + ay * ay, lb = bx * bx + by * by;
    const double det = ax * by - ay * bx;
    const double r = 1.0 / det;
    const double ux = 0.5 * (by * la - ay * lb) * r;
    const double uy = 0.5 * (ax * lb - bx * la) * r;
    const double ra = (ax - ux) * adx + (ay - uy) * ady;
    const double rb = (bx - ux) * bdx + (by - uy) * bdy;
    const double udx = (by * ra - ay * rb) * r;
    const double udy = (ax * rb - bx * ra) * r;
    const double detd = adx * by + ax * bdy - ady * bx - ay * bdx;
    g.s[a * N + i] = make_double2(ux * r, uy * r);
    g.sd[a * N + i] = make_double2(udx * r - ux * detd * r * r, udy * r - uy * detd * r * r);
    g.w[a * N + i] = make_double2(by - ay, ax - bx);
    g.wd[a * N + i] = make_double2(bdy - ady, adx - bdx);
    s_ux[a][t] = ux; s_uy[a][t] = uy;
    s_vx[a][t] = udx; s_vy[a][t] = udy;
    ax = bx; ay = by; adx = bdx; ady = bdy;
  }
  double A = 0.0, Ad = 0.0, P = 0.0, Pd = 0.0;
  for (int a = 0; a < m; ++a) {
    const int ap = (a == 0) ? m - 1 : a - 1;
    const double px = s_ux[ap][t], py = s_uy[ap][t], pdx = s_vx[ap][t], pdy = s_vy[ap][t];
    const double hx = s_ux[a][t], hy = s_uy[a][t], hdx = s_vx[a][t], hdy = s_vy[a][t];
    A += px * hy - hx * py;
    Ad += pdx * hy + px * hdy - hdx * py - hx * pdy;
    const double ex = hx - px, ey = hy - py, edx = hdx - pdx, edy = hdy - pdy;
    const double len = sqrt(ex * ex + ey * ey);
    const double il = 1.0 / len;
    const double nx = ex * il, ny = ey * il;
    const double dl = nx * edx + ny * edy;
    P += len;
    Pd += dl;
    s_ex[a][t] = nx; s_ey[a][t] = ny;
    s_fx[a][t] = (edx - nx * dl) * il;
    s_fy[a][t] = (edy - ny * dl) * il;
  }
  A *= 0.5;
  Ad *= 0.5;
  const double P0 = g.p0[i] * g.sqrtA0;
  double ka, kp, kad, kpd;
  if (g.coefA) {
    ka = g.coefA[i]; kp = g.coefP[i]; kad = 0.0; kpd = 0.0;
  } else {
    ka = 2.0 * g.KA * (A - g.A0); kp = 2.0 * g.KP * (P - P0);
    kad = 2.0 * g.KA * Ad; kpd = 2.0 * g.KP * Pd;
  }
  if (g.A) g.A[i] = A;
  if (g.P) g.P[i] = P;
  if (g.Adot) g.Adot[i] = Ad;
  if (g.Pdot) g.Pdot[i] = Pd;
  if (g.gp0) {  // parameter cotangents along v = g_{t+1}
    g.gp0[i] += g.dtmu * 2.0 * g.KP * g.sqrtA0 * Pd;
    g.gKA[i] += -g.dtmu * 2.0 * (A - g.A0) * Ad;
    g.gKP[i] += -g.dtmu * 2.0 * (P - P0) * Pd;
    double sn, cs;
    sincos(g.theta[i], &sn, &cs);
    g.gv0[i] += g.dt * (vi.x * cs + vi.y * sn);
  }
  for (int a = 0; a < m; ++a) {
    const int ap = (a == 0) ? m - 1 : a - 1;
    const int an = (a + 1 == m) ? 0 : a + 1;
    const double gx = 0.5 * (s_uy[an][t] - s_uy[ap][t]), gy = 0.5 * (s_ux[ap][t] - s_ux[an][t]);
    const double gdx = 0.5 * (s_vy[an][t] - s_vy[ap][t]), gdy = 0.5 * (s_vx[ap][t] - s_vx[an][t]);
    const double qx = s_ex[a][t] - s_ex[an][t], qy = s_ey[a][t] - s_ey[an][t];
    const double qdx = s_fx[a][t] - s_fx[an][t], qdy = s_fy[a][t] - s_fy[an][t];
    g.fs[a * N + i] = make_double2(ka * gx + kp * qx, ka * gy + kp * qy);
    g.fsd[a * N + i] = make_double2(kad * gx + ka * gdx + kpd * qx + kp * qdx, kad * gy + ka * gdy + kpd * qy + kp * qdy);
  }
}

__device__ __forceinline__ int ring_pos_a(const int* __restrict__ nbr, const int* __restrict__ cnt, int j, int i) {
  const int* row = nbr + (size_t)j * CG_RING;
  const int mj = cnt[j];
  for (int b = 0; b < mj; ++b)
    if (row[b] == i) return b;
  return -1;
}

// H g = -Fdot and the cotangent update g <- g - dt mu H g (in place: this
// kernel reads only per-slot data written by k_geom_jvp).
__global__ void k_force_jvp(JvpArgs g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const size_t N = (size_t)g.n;
  const int m = g.cnt[i];
  if (m < 3 || m > CG_RING) return;
  const int* ring = g.nbr + (size_t)i * CG_RING;
  const int jfirst = ring[0];
  const int pfirst = ring_pos_a(g.nbr, g.cnt, jfirst, i);
  int j = jfirst, pj = pfirst;
  bool bad = pfirst < 0;
  double Fdx = 0.0, Fdy = 0.0, Fx = 0.0, Fy = 0.0;
  for (int a = 0; a < m; ++a) {
    int k, pk;
    if (a + 1 < m) {
      k = ring[a + 1];
      pk = ring_pos_a(g.nbr, g.cnt, k, i);
      bad |= pk < 0;
    } else {
      k = jfirst;
      pk = pfirst;
    }
    const int mj = g.cnt[j];
    const int bj = (pj <= 0) ? (mj > 0 ? mj - 1 : 0) : pj - 1;
    const int bk = pk < 0 ? 0 : pk;
    const double2 f0 = g.fs[a * N + i], f1 = g.fs[(size_t)bj * N + j], f2 = g.fs[(size_t)bk * N + k];
    const double2 e0 = g.fsd[a * N + i], e1 = g.fsd[(size_t)bj * N + j], e2 = g.fsd[(size_t)bk * N + k];
    const double Gx = f0.x + f1.x + f2.x, Gy = f0.y + f1.y + f2.y;
    const double Gdx = e0.x + e1.x + e2.x, Gdy = e0.y + e1.y + e2.y;
    const double2 s = g.s[a * N + i], sd = g.sd[a * N + i];
    const double2 w = g.w[a * N + i], wd = g.wd[a * N + i];
    const double c = w.x * Gx + w.y * Gy;
    const double cd = wd.x * Gx + wd.y * Gy + w.x * Gdx + w.y * Gdy;
    Fx -= s.x * c;
    Fy -= s.y * c;
    Fdx -= sd.x * c + s.x * cd;
    Fdy -= sd.y * c + s.y * cd;
    j = k;
    pj = pk;
  }
  if (bad) raise_status(g.ctl, kETOPO);
  if (g.F) g.F[i] = make_double2(Fx, Fy);
  if (g.Hv) g.Hv[i] = make_double2(-Fdx, -Fdy);
  if (g.update) {
    double2 gi = g.v[i];
    gi.x += g.dtmu * Fdx;  // g - dt mu H g, H g = -Fdot
    gi.y += g.dtmu * Fdy;
    g.v[i] = gi;
  }
}

// g = (gx, gy) - F_coef : cotangent of the final positions, where F_coef is the
// "force" of the loss coefficients (minus the gradient of sum cA A + cP P).
__global__ void k_combine_final(int n, const double* gx, const double* gy, const double2* F, double2* g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) g[i] = make_double2(gx[i] - F[i].x, gy[i] - F[i].y);
}

__global__ void k_reduce2(int n, const double* a, const double* b, double* out) {
  __shared__ double sa[1024], sb[1024];
  double x = 0.0, y = 0.0;
  for (int i = threadIdx.x; i < n; i += 1024) {
    x += a[i];
    y += b[i];
  }
  sa[threadIdx.x] = x;
  sb[threadIdx.x] = y;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sa[threadIdx.x] += sa[threadIdx.x + o];
      sb[threadIdx.x] += sb[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sa[0];
    out[1] = sb[0];
  }
}

// Snapshot of the current state (positions of the current buffer, grid
// coordinates, directors, rings, control word) to / from a flat buffer.
__global__ void k_snapshot(int n, int save, Ctl* ctl, double* x, double* y, long long* X, long long* Y, double* theta,
                           int* cnt, int* nbr, Snapshot s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t N = (size_t)n;
  const int cur = save ? ctl->cur : s.ctl->cur;
  if (i < n) {
    if (save) {
      s.x[i] = x[cur * N + i]; s.y[i] = y[cur * N + i];
      s.X[i] = X[cur * N + i]; s.Y[i] = Y[cur * N + i];
      s.theta[i] = theta[i];
      s.cnt[i] = cnt[i];
      for (int a = 0; a < CG_RING; ++a) s.nbr[(size_t)i * CG_RING + a] = nbr[(size_t)i * CG_RING + a];
    } else {
      x[cur * N + i] = s.x[i]; y[cur * N + i] = s.y[i];
      X[cur * N + i] = s.X[i]; Y[cur * N + i] = s.Y[i];
      theta[i] = s.theta[i];
      cnt[i] = s.cnt[i];
      for (int a = 0; a < CG_RING; ++a) nbr[(size_t)i * CG_RING + a] = s.nbr[(size_t)i * CG_RING + a];
    }
  }
  if (i == 0) {
    if (save) *s.ctl = *ctl;
    else *ctl = *s.ctl;
  }
}

void launch_snapshot(int n, int save, Ctl* ctl, double* x, double* y, long long* X, long long* Y, double* theta,
                     int* cnt, int* nbr, const Snapshot& s, cudaStream_t st) {
  k_snapshot<<<(n + 255) / 256, 256, 0, st>>>(n, save, ctl, x, y, X, Y, theta, cnt, nbr, s);
}

void launch_geom_jvp(const JvpArgs& a, cudaStream_t st) {
  if (a.n > 0) k_geom_jvp<<<(a.n + kJvpThreads - 1) / kJvpThreads, kJvpThreads, 0, st>>>(a);
}
void launch_force_jvp(const JvpArgs& a, cudaStream_t st) {
  if (a.n > 0) k_force_jvp<<<(a.n + 127) / 128, 128, 0, st>>>(a);
}
void launch_combine_final(int n, const double* gx, const double* gy, const double2* F, double2* g, cudaStream_t st) {
  if (n > 0) k_combine_final<<<(n + 255) / 256, 256, 0, st>>>(n, gx, gy, F, g);
}
void launch_reduce2(int n, const double* a, const double* b, double* out, cudaStream_t st) {
  k_reduce2<<<1, 1024, 0, st>>>(n, a, b, out);
}

}  // namespace cgk
