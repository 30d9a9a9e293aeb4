// Device-side building blocks of the cellgb SPV path (sm_103a).
//
// Model: self-propelled Voronoi (SPV) model of Sussman, "cellGPU: massively
// parallel simulations of dynamic vertex models", arXiv 1702.02939.
//
// Conventions shared by every kernel
//  * Positions live on the dyadic grid 2^-q of their replica, q = 50 -
//    ceil(log2 max(Lx, Ly)); x (double) and X = x 2^q (int64) hold the same
//    value.  Minimum-image differences of grid values are exact, so every
//    topological decision (orientation, in-circle) is made exactly: a single
//    precision filter with a rigorous error bound, then exact integer
//    arithmetic (128-bit products, 256-bit sums) when the filter is unsure.
//  * Exactly cocircular quadruples are resolved by the lifting perturbation
//    |p|^2 + eps_p with eps_p growing with the cell tag (a phantom repair
//    generator counts as larger than every tag).
//  * Rings are stored row-major, CG_RING int32 slots per cell, CCW.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "dir_math.cuh"

#define CG_RING 16

namespace cgk {

// Status codes (mirrors include/cellgb.h).
enum : int {
  kOK = 0,
  kEINVAL = -1,
  kECUDA = -2,
  kERING = -3,
  kEREPAIR_CAP = -4,
  kETOPO = -5,
  kENONFINITE = -6,
  kEBOX = -7,
  kEDEGEN = -8,
  kECAND = -9,
  kET1CAP = -10,
};

// Per-replica constants.
struct Rep {
  double Lx, Ly, hLx, hLy;  // box and half box (on the grid)
  double scale, inv_scale;  // 2^q and 2^-q
  double bsx, bsy;          // cell-list bin size (the last bin of a row is wider)
  long long LX, LY;         // box in grid units
  long long W2;             // twice the initial repair half-width, grid units
  int cell0, ncell;         // cell range
  int nbx, nby, bin0;       // cell-list bins
  int q;
  double v0, p0;            // defaults for the replica's cells
  int hord;                 // Hilbert curve order of the replica's sort grid
  int hkey0;                // first sort key of the replica
  int bshift;               // cell-list bin width = 2^bshift grid units
  int hshift;               // Hilbert grid cell = 2^hshift grid units
  // Frame of a sub-box of a larger periodic box (a domain of a decomposed
  // system, cg_set_frame): the move of Eq. 3 is evaluated in the larger box's
  // coordinates (origin X0, Y0 and sides LXg, LYg in grid units, Lxg, Lyg in
  // box units) so that it rounds exactly as there.  framed = 0: the box is
  // the whole system.
  int framed;
  long long X0, Y0, LXg, LYg;
  double x0, y0, Lxg, Lyg;
};

// Cell-list bin of a position in grid units (integer only: every bin is
// 2^bshift grid units wide, the last bin of a row absorbs the remainder).
__device__ __forceinline__ void bin_of_grid(const Rep& R, long long X, long long Y, int& bx, int& by) {
  long long b = X >> R.bshift, c = Y >> R.bshift;
  bx = (int)(b < R.nbx ? b : R.nbx - 1);
  by = (int)(c < R.nby ? c : R.nby - 1);
}

// Mutable device globals of one context.
struct Ctl {
  int status;        // first error code raised by any kernel (0 = OK)
  int cur;           // which position buffer holds the current state
  long long step;    // global step counter (Philox counter)
  int count[2];      // flagged-list lengths (double-buffered)
  int round_count;   // repair rounds used in the last step
  int max_rounds;    // max over steps
  long long flagged_total, repaired_total;
  int last_flagged;
  int pad;
  unsigned int done;  // last-block counter of the repair-round check
  int dirty_count;    // cells whose ring a repair round rewrote in this step
  long long loop_total;  // iterations of the repair-round (or T1-pass) loop node
  int t1_more;        // the current T1 pass may leave work for another (AVM)
  int force_count;    // cells whose force the step recomputes after the repair rounds
};

// True in exactly one block of the grid: the last one to get here.  Every
// thread of every block must call it; each block's global writes are fenced
// before it counts itself, and the last block fences again before reading.
// The last block resets the counter for the next launch.
__device__ __forceinline__ bool last_block(unsigned int* done) {
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(done, 1u) == gridDim.x - 1);
  __syncthreads();
  if (s_last) {
    __threadfence();
    if (threadIdx.x == 0) *done = 0u;
  }
  return s_last;
}

// Bins per block of the block-local scans; the global start of bin b is the
// block-local exclusive prefix plus one offset per scan block.
constexpr int kScanChunk = 256 * 8;
__device__ __forceinline__ int bin_begin(const int* local, const int* partial, int b) {
  return local[b] + partial[b / kScanChunk];
}

// Position of grid cell (x, y) along the Hilbert curve of side 2^order:
// at each level the quadrant fixes two digits of the index, and the
// coordinates inside the quadrant are rotated/reflected so that the curve
// enters every sub-square at its start.
__device__ __forceinline__ unsigned hilbert_index(int order, unsigned x, unsigned y) {
  unsigned d = 0;
  for (int lev = order - 1; lev >= 0; --lev) {
    const unsigned s = 1u << lev;
    const unsigned rx = (x >> lev) & 1u, ry = (y >> lev) & 1u;
    d += s * s * ((3u * rx) ^ ry);
    x &= s - 1u;
    y &= s - 1u;
    if (ry == 0) {
      if (rx == 1) {
        x = s - 1u - x;
        y = s - 1u - y;
      }
      const unsigned t = x;
      x = y;
      y = t;
    }
  }
  return d;
}

__device__ __forceinline__ void raise_status(Ctl* ctl, int code) {
  atomicCAS(&ctl->status, 0, code);
}

__device__ __forceinline__ long long min_image_i(long long d, long long L) {
  long long h = L >> 1;
  if (d > h) d -= L;
  else if (d < -h) d += L;
  return d;
}

// ----------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11) and the director noise of Eq. 3.
// ----------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// The 53 high bits of hi:lo, plus one: the uniform (k + 1) 2^-53 in (0, 1]
// as an integer k + 1 in [1, 2^53].
__device__ __forceinline__ unsigned long long bits53p1(unsigned hi, unsigned lo) {
  return (((((unsigned long long)hi) << 32) | lo) >> 11) + 1ull;
}
// (k + 1) 2^-53 exactly, on the integer pipes.
__device__ __forceinline__ double unit53_of(unsigned long long kp1) {
  return kp1 == (1ull << 53) ? 1.0 : i2d_int((long long)kp1, -53);
}
// (53 high bits of hi:lo, plus one) * 2^-53, in (0, 1].
__device__ __forceinline__ double unit53(unsigned hi, unsigned lo) { return unit53_of(bits53p1(hi, lo)); }

// 1/d to ~1 ulp: hardware reciprocal approximation r = (1 - e)/d refined by
// one third-order step r (1 + e + e^2), e = 1 - d r (the geometric series of
// 1/(1 - e) to e^2; the error left is e^3 plus rounding): 3 FP64 FMAs
// instead of an IEEE division.
__device__ __forceinline__ double fast_rcp(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  const double e = fma(-d, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

// 1/sqrt(x) for a positive normal x: hardware approximation y refined by one
// third-order step y (1 + e/2 + 3 e^2/8), e = 1 - x y^2 (the binomial series
// of (1 - e)^(-1/2) to e^2; the error left is about (5/16) e^3 plus
// rounding): 5 FP64 operations.
__device__ __forceinline__ double fast_rsqrt(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y * y, 1.0);
  return fma(y * e, fma(e, 0.375, 0.5), y);
}

// A 128-bit integer rounded to the nearest double (ties to even), on the
// integer pipes: the magnitude shifted so that its leading one is bit 127,
// its top 64 bits rounded to 53 with a sticky bit for the rest (a carry out
// of the mantissa lands in the exponent field); times 2^e2 (exact).
__device__ __forceinline__ double i128_to_double(__int128 v, int e2 = 0) {
  const bool neg = v < 0;
  const unsigned __int128 a = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
  const unsigned long long hi = (unsigned long long)(a >> 64), lo = (unsigned long long)a;
  int nb;  // significant bits
  unsigned long long top;
  bool sticky;
  if (hi) {
    const int lz = __clzll((long long)hi);
    nb = 128 - lz;
    const unsigned __int128 sh = a << lz;
    top = (unsigned long long)(sh >> 64);
    sticky = (unsigned long long)sh != 0;
  } else if (lo) {
    const int lz = __clzll((long long)lo);
    nb = 64 - lz;
    top = lo << lz;
    sticky = false;
  } else {
    return 0.0;
  }
  unsigned long long m = top >> 11;
  const unsigned long long rem = top & 0x7ff;
  if (rem > 0x400 || (rem == 0x400 && (sticky || (m & 1)))) m += 1;
  const unsigned long long bits = ((unsigned long long)(nb + 1021 + e2) << 52) + m;
  return __longlong_as_double((long long)(bits | (neg ? 0x8000000000000000ull : 0ull)));
}

// Puts cell i on a list once per use of the bitmap: the caller that sets
// its bit appends it (the force pass's fix-up list of a step).
__device__ __forceinline__ void claim_fix(unsigned* bits, int* list, int* count, int i) {
  const unsigned bit = 1u << (i & 31);
  if (!(atomicOr(&bits[i >> 5], bit) & bit)) list[atomicAdd(count, 1)] = i;
}

// Significant bits of a 128-bit magnitude (0 for 0).
__device__ __forceinline__ int u128_bits(unsigned __int128 v) {
  const unsigned long long hi = (unsigned long long)(v >> 64), lo = (unsigned long long)v;
  return hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);
}

// 1/d and 1/sqrt(x) with the refinement on the integer pipes: the mantissa
// (53 bits) in fixed point, an FP32 hardware seed (rcp/rsqrt.approx of the
// mantissa's top 23 bits, relative error ~2^-22), one third-order step in
// Q1.62 (r (1 + e + e^2) with e = 1 - m r; y (1 + e/2 + 3 e^2/8) with
// e = 1 - m y^2; the error left is ~e^3 ~ 2^-66), and one rounding to double
// with the exponent put back: within 1 ulp, like fast_rcp / fast_rsqrt, with
// no FP64 instruction.  Zero, subnormal, infinite and NaN inputs take the
// FP64 functions.
__device__ __forceinline__ long long seed_q62(float yf) {  // yf in (0.5, 1]: yf 2^62
  const int b = __float_as_int(yf);
  const long long mant = (long long)((b & 0x7fffff) | 0x800000);
  return mant << (39 + ((b >> 23) & 0xff) - 127);  // 62 - 23 + exponent (0 or -1)
}
__device__ __forceinline__ double fx_rcp(double d) {
  const long long b = __double_as_longlong(d);
  const int ef = (int)((b >> 52) & 0x7ff);
  if (ef == 0 || ef == 0x7ff) return fast_rcp(d);
  const long long m = (b & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;  // mantissa in [1, 2) times 2^52
  float yf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(__int_as_float(0x3f800000 | (int)((b >> 29) & 0x7fffff))));
  long long y = seed_q62(yf);
  const long long e = kQOne - mulq(m << 10, y);  // 1 - m y
  y += mulq(y, e + mulq(e, e));
  const double r = q2d(y, -62 - (ef - 1023));
  return b < 0 ? -r : r;
}
__device__ __forceinline__ double fx_rsqrt(double x) {
  const long long b = __double_as_longlong(x);
  const int ef = (int)((b >> 52) & 0x7ff);
  if (ef == 0 || ef == 0x7ff || b < 0) return fast_rsqrt(x);
  const int E = ef - 1023, odd = E & 1;
  const long long m = (b & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;
  // x = m' 2^(E - odd) with m' = m 2^(odd - 52) in [1, 4), held as m' 2^61
  const long long mq61 = m << (9 + odd);
  float yf;
  asm("rsqrt.approx.ftz.f32 %0, %1;"
      : "=f"(yf)
      : "f"(__int_as_float((odd ? 0x40000000 : 0x3f800000) | (int)((b >> 29) & 0x7fffff))));
  long long y = seed_q62(yf);
  const long long my2 = (long long)(((__int128)mq61 * mulq(y, y)) >> 61);  // m' y^2 in Q1.62
  const long long e = kQOne - my2;
  y += mulq(y, mulq(e, (kQOne >> 1) + mulq(e, 3 * (kQOne >> 3))));
  return q2d(y, -62 - (E - odd) / 2);
}

// Standard normal for (seed, cell tag, step), cosine branch of Box-Muller,
// with the table-driven ln and cos(pi .) of dir_math.cuh (tab: the 512-entry
// director table).
__device__ __forceinline__ double director_noise(unsigned long long seed, int tag, long long step,
                                                 const double2* __restrict__ tab) {
  uint4 r = philox_10(make_uint4((unsigned)tag, (unsigned)(unsigned long long)step,
                                 (unsigned)((unsigned long long)step >> 32), 0u),
                      make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
  const double u1 = unit53(r.x, r.y);
  const unsigned long long k2 = bits53p1(r.z, r.w);  // u2 = k2 2^-53
  // sqrt(x) as x / sqrt(x) (within 2 ulp; u1 = 1 gives x = -0 and R = 0);
  // cos(2 pi u2) as cos(pi t), t = 2 u2 exact
  const double x = -2.0 * dm_log(u1, tab);
  const double R = (__double_as_longlong(x) > 0) ? x * fast_rsqrt(x) : 0.0;
  return R * dm_cospi_grid52(k2, tab);  // cos(2 pi u2) = cos(pi k2 2^-52)
}

// ----------------------------------------------------------------------------
// Exact predicates on integer grid coordinates.
// ----------------------------------------------------------------------------
typedef __int128 s128;
typedef unsigned __int128 u128;

// 256-bit two's complement value as (hi, lo).
struct W256 {
  u128 hi, lo;
};

__device__ __forceinline__ W256 w256_neg(W256 v) {
  W256 r;
  r.lo = ~v.lo + 1;
  r.hi = ~v.hi + (r.lo == 0 ? 1 : 0);
  return r;
}
__device__ __forceinline__ W256 w256_add(W256 a, W256 b) {
  W256 r;
  r.lo = a.lo + b.lo;
  r.hi = a.hi + b.hi + (r.lo < a.lo ? 1 : 0);
  return r;
}
// Signed product of two 128-bit integers whose magnitudes are below 2^110.
static __device__ __noinline__ W256 w256_mul(s128 a, s128 b) {
  bool neg = (a < 0) != (b < 0);
  u128 x = a < 0 ? (u128)(-a) : (u128)a;
  u128 y = b < 0 ? (u128)(-b) : (u128)b;
  unsigned long long x0 = (unsigned long long)x, x1 = (unsigned long long)(x >> 64);
  unsigned long long y0 = (unsigned long long)y, y1 = (unsigned long long)(y >> 64);
  u128 p00 = (u128)x0 * y0;
  u128 mid = (u128)x0 * y1 + (u128)x1 * y0;  // < 2^127 for our operand sizes
  u128 p11 = (u128)x1 * y1;
  W256 r;
  r.lo = p00 + (mid << 64);
  u128 carry = (r.lo < p00) ? 1 : 0;
  r.hi = p11 + (mid >> 64) + carry;
  return neg ? w256_neg(r) : r;
}
__device__ __forceinline__ int w256_sign(W256 v) {
  if (v.hi == 0 && v.lo == 0) return 0;
  return ((long long)(unsigned long long)(v.hi >> 64) < 0) ? -1 : 1;
}

__device__ __forceinline__ int orient_exact(long long ax, long long ay, long long bx, long long by) {
  s128 d = (s128)ax * by - (s128)ay * bx;
  return (d > 0) - (d < 0);
}

// Sign of (b - a) x (c - a) for integer points, exact.
__device__ __forceinline__ int orient3_exact(long long ax, long long ay, long long bx, long long by,
                                             long long cx, long long cy) {
  return orient_exact(bx - ax, by - ay, cx - ax, cy - ay);
}

// Exact sign of det[[a, |a|^2], [b, |b|^2], [c, |c|^2]] (rows relative to the
// query point), for |coordinates| < 2^52.
static __device__ __noinline__ int incircle_rows_exact(long long ax, long long ay, long long bx, long long by,
                                                long long cx, long long cy) {
  s128 la = (s128)ax * ax + (s128)ay * ay;
  s128 lb = (s128)bx * bx + (s128)by * by;
  s128 lc = (s128)cx * cx + (s128)cy * cy;
  s128 xbc = (s128)bx * cy - (s128)by * cx;
  s128 xca = (s128)cx * ay - (s128)cy * ax;
  s128 xab = (s128)ax * by - (s128)ay * bx;
  W256 s = w256_add(w256_add(w256_mul(la, xbc), w256_mul(lb, xca)), w256_mul(lc, xab));
  return w256_sign(s);
}

// v * sc as a float for |v| < 2^51, without 64-bit conversion instructions
// (which issue on the FP64 pipe of this GPU): |v| is split into 22-bit chunks,
// each converted exactly by adding it to the bit pattern of 1.5 * 2^23 and
// subtracting 1.5 * 2^23; two FMAs recombine them.  Relative error <= 2u + u^2
// (u = 2^-24); sc must be a power of two.
__device__ __forceinline__ float i2f_scaled(long long v, float sc) {
  const bool neg = v < 0;
  const unsigned long long a = neg ? (unsigned long long)(-v) : (unsigned long long)v;
  const int c0 = (int)(a & 0x3FFFFFull), c1 = (int)((a >> 22) & 0x3FFFFFull), c2 = (int)(a >> 44);
  const float f0 = __int_as_float(0x4B400000 + c0) - 12582912.0f;
  const float f1 = __int_as_float(0x4B400000 + c1) - 12582912.0f;
  const float f2 = __int_as_float(0x4B400000 + c2) - 12582912.0f;
  const float f = fmaf(f2, 0x1p44f, fmaf(f1, 0x1p22f, f0)) * sc;
  return neg ? -f : f;
}

// Orientation of (0, a, b), coordinates in grid units; sc = 2^-q (float).
__device__ __forceinline__ int orient_sign(long long ax, long long ay, long long bx, long long by, float sc) {
  float fax = i2f_scaled(ax, sc), fay = i2f_scaled(ay, sc), fbx = i2f_scaled(bx, sc), fby = i2f_scaled(by, sc);
  float l = fax * fby, r = fay * fbx;
  float det = l - r;
  // conversion (<= 4u per product) + product (u) + difference (u): <= 6u * (|l|+|r|)
  float bound = 1.0e-6f * (fabsf(l) + fabsf(r));
  if (bound > 1.0e-30f) {
    if (det > bound) return 1;
    if (det < -bound) return -1;
  }
  return orient_exact(ax, ay, bx, by);
}

// Lifting-perturbed in-circle of (p, q, r, s): > 0 iff s is inside the circle
// through p, q, r (p, q, r counter-clockwise).  Integer grid coordinates with
// a common origin; keys order the infinitesimal lifts.  Never returns 0 for
// four distinct points.
__device__ __forceinline__ int incircle_sign(long long px, long long py, long long qx, long long qy,
                                             long long rx, long long ry, long long sx, long long sy,
                                             int kp, int kq, int kr, int ks, float sc) {
  long long ax = px - sx, ay = py - sy, bx = qx - sx, by = qy - sy, cx = rx - sx, cy = ry - sy;
  float fax = i2f_scaled(ax, sc), fay = i2f_scaled(ay, sc), fbx = i2f_scaled(bx, sc), fby = i2f_scaled(by, sc);
  float fcx = i2f_scaled(cx, sc), fcy = i2f_scaled(cy, sc);
  float la = fax * fax + fay * fay, lb = fbx * fbx + fby * fby, lc = fcx * fcx + fcy * fcy;
  float t1 = fbx * fcy, t2 = fby * fcx, t3 = fcx * fay, t4 = fcy * fax, t5 = fax * fby, t6 = fay * fbx;
  float det = la * (t1 - t2) + lb * (t3 - t4) + lc * (t5 - t6);
  float perm = la * (fabsf(t1) + fabsf(t2)) + lb * (fabsf(t3) + fabsf(t4)) + lc * (fabsf(t5) + fabsf(t6));
  // input conversion (<= 8u per degree-4 monomial) + evaluation (<= 10u): 2e-6 ~ 34u.
  float bound = 2.0e-6f * perm;
  if (bound > 1.0e-30f && bound < 1.0e30f) {
    if (det > bound) return 1;
    if (det < -bound) return -1;
  }
  int s = incircle_rows_exact(ax, ay, bx, by, cx, cy);
  if (s != 0) return s;
  // Tie: the highest-key point's lift decides (its cofactor is a non-zero
  // orientation because no three of four distinct cocircular points are collinear).
  int top = 0, kt = kp;
  if (kq > kt) { top = 1; kt = kq; }
  if (kr > kt) { top = 2; kt = kr; }
  if (ks > kt) { top = 3; kt = ks; }
  switch (top) {
    case 0: return orient3_exact(qx, qy, rx, ry, sx, sy);
    case 1: return orient3_exact(rx, ry, px, py, sx, sy);
    case 2: return orient3_exact(px, py, qx, qy, sx, sy);
    default: return -orient3_exact(px, py, qx, qy, rx, ry);
  }
}

// incircle_sign(0, q, r, s) with the float values of q, r, s (real units,
// converted once by the caller) for the filter: translating the lifted
// determinant to the first point instead of the last only flips its sign,
// det3(q, r, s) = -det3(0 - s, q - s, r - s).  The filter bound is the one of
// incircle_sign; an inconclusive filter defers to incircle_sign itself, so
// every decision (ties included) is the same.
// The tags of the four cells (for the symbolic perturbation of the exact
// fallback) are read only when the filter cannot decide.
__device__ __forceinline__ int incircle0_sign(float fqx, float fqy, float frx, float fry, float fsx, float fsy,
                                              long long qx, long long qy, long long rx, long long ry, long long sx,
                                              long long sy, const int* __restrict__ tag, int ip, int iq, int ir,
                                              int is, float sc) {
  float la = fqx * fqx + fqy * fqy, lb = frx * frx + fry * fry, lc = fsx * fsx + fsy * fsy;
  float t1 = frx * fsy, t2 = fry * fsx, t3 = fsx * fqy, t4 = fsy * fqx, t5 = fqx * fry, t6 = fqy * frx;
  float det = la * (t1 - t2) + lb * (t3 - t4) + lc * (t5 - t6);
  float perm = la * (fabsf(t1) + fabsf(t2)) + lb * (fabsf(t3) + fabsf(t4)) + lc * (fabsf(t5) + fabsf(t6));
  float bound = 2.0e-6f * perm;
  if (bound > 1.0e-30f && bound < 1.0e30f) {
    if (det > bound) return -1;
    if (det < -bound) return 1;
  }
  return incircle_sign(0, 0, qx, qy, rx, ry, sx, sy, tag[ip], tag[iq], tag[ir], tag[is], sc);
}

// orient_sign(a, b) with the float values of a and b converted by the caller.
__device__ __forceinline__ int orient0_sign(float fax, float fay, float fbx, float fby, long long ax, long long ay,
                                            long long bx, long long by) {
  float l = fax * fby, r = fay * fbx;
  float det = l - r;
  float bound = 1.0e-6f * (fabsf(l) + fabsf(r));
  if (bound > 1.0e-30f) {
    if (det > bound) return 1;
    if (det < -bound) return -1;
  }
  return orient_exact(ax, ay, bx, by);
}

// ----------------------------------------------------------------------------
// Shared by the FP64 and FP32 step kernels.
// ----------------------------------------------------------------------------
// Periodic reduction of a finite coordinate: v' = fmod(v, L) (exact), rounded
// to the grid, then wrapped into [0, L) in integer grid units.  For v in
// [-L, 2L) fmod is a single exact subtraction or nothing.
__device__ __forceinline__ long long wrap_to_grid(double v, double L, double scale, long long LI) {
  double r;
  // the common case 0 <= v < L decided on the integer pipe (non-negative
  // doubles order like their bit patterns; -0 and NaN fail it)
  if ((unsigned long long)__double_as_longlong(v) < (unsigned long long)__double_as_longlong(L)) r = v;
  else if (v >= L && v < 2.0 * L) r = v - L;
  else if (v < 0.0 && v >= -L) r = v;
  else r = fmod(v, L);
  // rint(r * scale) for |r * scale| < 2^51 (scale is a power of two, so the
  // product is exact): adding 1.5 * 2^52 rounds to the nearest integer, ties to
  // even, and leaves it in the low bits
  const long long X0 = __double_as_longlong(r * scale + 0x1.8p52) - 0x4338000000000000LL;
  long long X = X0;
  if (X < 0) X += LI;
  else if (X >= LI) X -= LI;
  return X;
}

// Position update of Eq. 3 on one axis in a framed box (a domain of a
// larger periodic box, Rep::framed): x + dt v is formed in the larger box's
// coordinates, x = xi + x0 reduced into [0, Lg) (both exact on the grid), so
// that it rounds exactly as in the undivided system; the grid value is then
// brought back into the frame (a cell that left the frame is wrapped into
// it: only halo cells can, and their positions are replaced).
__device__ __forceinline__ long long move_framed(double xi, double dt, double v, double x0, double Lg, double scale,
                                                 long long X0, long long LG, long long LI) {
  double x = xi + x0;
  if (x >= Lg) x -= Lg;
  long long X = wrap_to_grid(fma(dt, v, x), Lg, scale, LG) - X0;
  if (X < 0) X += LG;
  if (X >= LI) X %= LI;
  return X;
}

// Exact int64 -> double for |v| < 2^51: v added to the bit pattern of 1.5 * 2^52
// (integer pipe) lands in [2^52, 2^53) where doubles are spaced by one; one
// FP64 subtraction removes the offset.
__device__ __forceinline__ double i2d_exact(long long v) {
  return __longlong_as_double(0x4338000000000000LL + v) - 0x1.8p52;
}

// Position of cell i in the ring of cell j, or -1.
__device__ __forceinline__ int ring_pos(const int* __restrict__ nbr, const int* __restrict__ cnt, int j, int i) {
  const int4* row = reinterpret_cast<const int4*>(nbr + (size_t)j * CG_RING);
  const int mj = cnt[j];
  int pos = -1;
#pragma unroll
  for (int q = 0; q < CG_RING / 4; ++q) {
    if (4 * q >= mj) break;
    int4 v = row[q];
    if (v.x == i && 4 * q + 0 < mj) pos = 4 * q + 0;
    if (v.y == i && 4 * q + 1 < mj) pos = 4 * q + 1;
    if (v.z == i && 4 * q + 2 < mj) pos = 4 * q + 2;
    if (v.w == i && 4 * q + 3 < mj) pos = 4 * q + 3;
  }
  return pos;
}

}  // namespace cgk
