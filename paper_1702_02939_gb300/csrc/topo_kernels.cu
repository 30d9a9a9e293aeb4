// Topology maintenance: cell list, local repair by Voronoi-cell clipping and
// the ring-consistency check.
//
// The paper repairs flagged cells on the CPU: a candidate "Delaunay 1-ring"
// from the locality lemma of Chen et al., reduced to the true neighbours with
// CGAL (Sussman, arXiv 1702.02939, Sec. 2.C.4).  Here the repair stays on the
// GPU: each flagged cell's Voronoi polygon is rebuilt by clipping a large
// square with the bisectors of nearby cells taken from a periodic cell list,
// nearest first.  A polygon vertex v_a (circumcentre of i, g_a, g_{a+1})
// is cut away by candidate j exactly when j lies inside the circle through
// (i, g_a, g_{a+1}), so every keep/drop decision is the exact, perturbed
// in-circle predicate and the result is the exact Delaunay ring of i.  The
// search stops once every unvisited cell is farther than twice the polygon's
// circumradius (the security radius), which is the locality argument of the
// paper in its simplest form.
#include "cg_device.cuh"
#include "cg_kernels.h"

#include <climits>

namespace cgk {

constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
static_assert(kScanChunk == kScanThreads * kScanPer, "scan block size");

__global__ void k_bin_count(CellListArgs g) {
  if (g.only_if_flagged && g.ctl->count[0] == 0) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const int cur = g.ctl->cur;
  const Rep R = g.reps[g.rep[i]];
  int bx, by;
  bin_of_grid(R, g.X[(size_t)cur * g.n + i], g.Y[(size_t)cur * g.n + i], bx, by);
  const int b = R.bin0 + by * R.nbx + bx;
  g.cell_bin[i] = b;
  g.cell_rank[i] = atomicAdd(&g.bin_count[b], 1);
}

// Block-local exclusive scan of bin counts; block totals to scan_partials.
__global__ void __launch_bounds__(kScanThreads) k_scan_local(CellListArgs g) {
  if (g.only_if_flagged && g.ctl->count[0] == 0) return;
  __shared__ int warp_tot[kScanThreads / 32];
  const int base = blockIdx.x * kScanChunk + threadIdx.x * kScanPer;
  int v[kScanPer];
  int sum = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    int b = base + k;
    v[k] = (b < g.nbins) ? g.bin_count[b] : 0;
    sum += v[k];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  int woff = 0;
  for (int w = 0; w < wid; ++w) woff += warp_tot[w];
  int run = woff + incl - sum;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    int b = base + k;
    if (b < g.nbins) g.bin_start[b] = run;
    else if (b == g.nbins) g.bin_start[b] = run;  // sentinel
    run += v[k];
  }
  if (threadIdx.x == kScanThreads - 1) {
    int tot = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) tot += warp_tot[w];
    g.scan_partials[blockIdx.x] = tot;
  }
}

// Exclusive scan of the block totals (one block); also records step statistics.
__global__ void __launch_bounds__(1024) k_scan_partials(CellListArgs g, int nblocks) {
  Ctl* ctl = g.ctl;
  if (threadIdx.x == 0 && g.only_if_flagged) {  // per-step build: record statistics
    int c = ctl->count[0];
    ctl->last_flagged = c;
    ctl->flagged_total += c;
  }
  if (g.only_if_flagged && ctl->count[0] == 0) return;
  __shared__ int buf[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base <= nblocks; base += 1024) {
    int idx = base + threadIdx.x;
    int v = (idx < nblocks) ? g.scan_partials[idx] : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      int t = (threadIdx.x >= o) ? buf[threadIdx.x - o] : 0;
      __syncthreads();
      buf[threadIdx.x] += t;
      __syncthreads();
    }
    int excl = carry + buf[threadIdx.x] - v;
    __syncthreads();
    if (idx < nblocks) g.scan_partials[idx] = excl;
    else if (idx == nblocks) g.scan_partials[idx] = excl;  // total
    if (threadIdx.x == 1023) carry += buf[1023];
    __syncthreads();
  }
}

__global__ void k_bin_scatter(CellListArgs g) {
  if (g.only_if_flagged && g.ctl->count[0] == 0) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const int b = g.cell_bin[i];
  g.ids[bin_begin(g.bin_start, g.scan_partials, b) + g.cell_rank[i]] = i;
  g.bin_count[b] = 0;  // ready for the next build
}

void launch_cell_list(const CellListArgs& a, cudaStream_t st) {
  if (a.n <= 0) return;
  const int nblk = (a.nbins + 1 + kScanChunk - 1) / kScanChunk;
  k_bin_count<<<(a.n + 255) / 256, 256, 0, st>>>(a);
  k_scan_local<<<nblk, kScanThreads, 0, st>>>(a);
  k_scan_partials<<<1, 1024, 0, st>>>(a, nblk);
  k_bin_scatter<<<(a.n + 255) / 256, 256, 0, st>>>(a);
}

void launch_scan(const CellListArgs& a, cudaStream_t st) {
  const int nblk = (a.nbins + 1 + kScanChunk - 1) / kScanChunk;
  k_scan_local<<<nblk, kScanThreads, 0, st>>>(a);
  k_scan_partials<<<1, 1024, 0, st>>>(a, nblk);
}

// ---------------------------------------------------------------------------
// Repair: one warp per cell.
// ---------------------------------------------------------------------------

// Upper bound on |v|^2 for the polygon vertex v = circumcentre of (0, a, b)
// (real units; a, b in grid units).  Used only for the security radius, so it
// may over-estimate but never under-estimate.  Single precision with a
// first-order error bound: inputs carry relative error <= 2u (u = 2^-24, see
// i2f_scaled), the determinant is accepted when its error bound is below 1/64
// of it; otherwise (nearly collinear generators) the vertex is recomputed in
// double precision from the exact integer determinant.
__device__ __noinline__ float vertex_r2_fp64(long long aX, long long aY, long long bX, long long bY, double inv_scale) {
  const s128 D = (s128)aX * bY - (s128)aY * bX;
  const long long dhi = (long long)(D >> 64);
  const unsigned long long dlo = (unsigned long long)D;
  const double det = ((double)dhi * 0x1.0p64 + (double)dlo) * inv_scale * inv_scale;
  if (det == 0.0) return 3.0e38f;
  const double ax = (double)aX * inv_scale, ay = (double)aY * inv_scale;
  const double bx = (double)bX * inv_scale, by = (double)bY * inv_scale;
  const double la = ax * ax + ay * ay, lb = bx * bx + by * by;
  const double inv = 0.5 / det;
  const double vx = (by * la - ay * lb) * inv, vy = (ax * lb - bx * la) * inv;
  const double r2 = (vx * vx + vy * vy) * (1.0 + 1e-9);
  return r2 < 3.0e38 ? (float)r2 * 1.000001f : 3.0e38f;
}

__device__ __forceinline__ float vertex_r2_bound(long long aX, long long aY, long long bX, long long bY, float sc,
                                                 double inv_scale) {
  const float u = 0x1p-24f;
  const float ax = i2f_scaled(aX, sc), ay = i2f_scaled(aY, sc), bx = i2f_scaled(bX, sc), by = i2f_scaled(bY, sc);
  const float p1 = ax * by, p2 = ay * bx;
  const float det = p1 - p2;
  const float edet = 8.0f * u * (fabsf(p1) + fabsf(p2));
  if (!(fabsf(det) > 64.0f * edet) || !(fabsf(det) > 1e-30f)) return vertex_r2_fp64(aX, aY, bX, bY, inv_scale);
  const float la = ax * ax + ay * ay, lb = bx * bx + by * by;
  const float n1 = by * la, n2 = ay * lb, n3 = ax * lb, n4 = bx * la;
  const float hinv = 0.5f / det;
  const float hx = (n1 - n2) * hinv, hy = (n3 - n4) * hinv;
  // numerator: 6u from the inputs of the degree-3 terms + 4u from evaluation
  const float ad = fabsf(det);
  const float rel = edet / ad;  // <= 1/64
  const float dhx = (10.0f * u * (fabsf(n1) + fabsf(n2)) * 0.5f / ad + fabsf(hx) * rel) * 1.05f;
  const float dhy = (10.0f * u * (fabsf(n3) + fabsf(n4)) * 0.5f / ad + fabsf(hy) * rel) * 1.05f;
  const float r = sqrtf(hx * hx + hy * hy) * (1.0f + 4.0f * u) + sqrtf(dhx * dhx + dhy * dhy);
  return r * r * (1.0f + 8.0f * u);
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// (dx, dy) of the idx-th bin on the Chebyshev ring k around the origin bin.
__device__ __forceinline__ void ring_bin(int k, int idx, int& dx, int& dy) {
  if (k == 0) { dx = 0; dy = 0; return; }
  const int side = 2 * k;  // bins per side, walking CCW from (-k, -k)
  const int s = idx / side, t = idx % side;
  switch (s) {
    case 0: dx = -k + t; dy = -k; break;
    case 1: dx = k; dy = -k + t; break;
    case 2: dx = k - t; dy = k; break;
    default: dx = -k; dy = k - t; break;
  }
}

struct Poly {
  long long gX, gY;  // this lane's generator (grid units, relative to the cell)
  int gid, gkey;     // generator cell index (phantoms < 0) and perturbation key
  float r2;          // upper bound of |v|^2, v = vertex between this generator and the next
  int m;             // generators in use (warp-uniform)
  float R2;          // max over the polygon of r2 (warp-uniform)
  int err;
};

constexpr int kPhantomKey = INT_MAX - 8;
constexpr float kSelfKey = 1e37f;  // sort key of the cell itself
constexpr float kPadKey = 3e38f;   // sort key of unused buffer slots

// Clip the polygon by the bisector of candidate j.
__device__ __forceinline__ void clip(Poly& p, long long jX, long long jY, int jid, int jkey, int ikey, float sc,
                                     double inv_scale, int lane) {
  const int m = p.m;
  const int nl = (lane + 1 == m) ? 0 : (lane + 1) % 32;
  const long long nX = __shfl_sync(0xffffffffu, p.gX, nl);
  const long long nY = __shfl_sync(0xffffffffu, p.gY, nl);
  const int nkey = __shfl_sync(0xffffffffu, p.gkey, nl);
  int rem = 0;
  if (lane < m) rem = incircle_sign(0, 0, p.gX, p.gY, nX, nY, jX, jY, ikey, p.gkey, nkey, jkey, sc) > 0;
  const unsigned mask = __ballot_sync(0xffffffffu, rem);
  if (mask == 0) return;
  const int r = __popc(mask);
  if (r == m) { p.err = kEDEGEN; return; }
  const int pl = (lane == 0) ? m - 1 : lane - 1;
  const int prevrem = (mask >> pl) & 1;
  const unsigned smask = __ballot_sync(0xffffffffu, lane < m && rem && !prevrem);
  if (__popc(smask) != 1) { p.err = kEDEGEN; return; }
  const int s = __ffs(smask) - 1;
  int e = s + r - 1;  // (s + r - 1) mod m, with s, r - 1 < m
  if (e >= m) e -= m;
  const int m2 = m - r + 2;
  if (m2 > 32) { p.err = kERING; return; }
  // (lane + e + 1) mod m for the lanes that keep a generator (lane < m2 <= m + 1,
  // so lane + e + 1 <= 2m); other lanes read any lane
  int src = lane + e + 1;
  if (src >= m) src -= m;
  if (src >= m) src -= m;
  long long ngX = __shfl_sync(0xffffffffu, p.gX, src);
  long long ngY = __shfl_sync(0xffffffffu, p.gY, src);
  int ngid = __shfl_sync(0xffffffffu, p.gid, src);
  int ngkey = __shfl_sync(0xffffffffu, p.gkey, src);
  float nr2 = __shfl_sync(0xffffffffu, p.r2, src);
  if (lane == m2 - 1) { ngX = jX; ngY = jY; ngid = jid; ngkey = jkey; }
  p.gX = ngX; p.gY = ngY; p.gid = ngid; p.gkey = ngkey; p.r2 = nr2;
  p.m = m2;
  const int nl2 = (lane + 1 == m2) ? 0 : (lane + 1) % 32;
  const long long n2X = __shfl_sync(0xffffffffu, p.gX, nl2);
  const long long n2Y = __shfl_sync(0xffffffffu, p.gY, nl2);
  if (lane == m2 - 2 || lane == m2 - 1) p.r2 = vertex_r2_bound(p.gX, p.gY, n2X, n2Y, sc, inv_scale);
  p.R2 = warp_max(lane < m2 ? p.r2 : 0.0f);
}

// Sort the warp's candidate buffer by squared distance and clip with every
// candidate that can still reach the polygon.  The 64 keys live in registers,
// two per lane (entries lane and lane + 32), and are sorted by a bitonic
// network of register shuffles; the clips then take the entries in order.
__device__ void process_candidates(Poly& p, int nbuf, const int* s_id, const long long* s_X, const long long* s_Y,
                                   const float* s_d2, const int* s_tag, int ikey, float sc, double inv_scale,
                                   int lane) {
  static_assert(kCand == 64, "two keys per lane");
  if (nbuf == 0) return;
  float k0 = (lane < nbuf) ? s_d2[lane] : kPadKey, k1 = (lane + 32 < nbuf) ? s_d2[lane + 32] : kPadKey;
  int v0 = lane, v1 = lane + 32;
#pragma unroll
  for (int k = 2; k <= 64; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j == 32) {  // entries lane and lane + 32, ascending (k = 64)
        if (k0 > k1) {
          const float tk = k0; k0 = k1; k1 = tk;
          const int tv = v0; v0 = v1; v1 = tv;
        }
      } else {
        const bool lower = (lane & j) == 0;
        // entry q = lane (+ 32): ascending block when (q & k) == 0
        const bool up0 = (lane & k) == 0, up1 = ((lane + 32) & k) == 0;
        const float p0 = __shfl_xor_sync(0xffffffffu, k0, j), p1 = __shfl_xor_sync(0xffffffffu, k1, j);
        const int w0 = __shfl_xor_sync(0xffffffffu, v0, j), w1 = __shfl_xor_sync(0xffffffffu, v1, j);
        // the lower entry of a pair keeps the minimum in an ascending block
        if (lower == up0 ? p0 < k0 : p0 > k0) { k0 = p0; v0 = w0; }
        if (lower == up1 ? p1 < k1 : p1 > k1) { k1 = p1; v1 = w1; }
      }
    }
  }
  for (int c = 0; c < nbuf; ++c) {
    const int src = c & 31;
    const float d2 = __shfl_sync(0xffffffffu, c < 32 ? k0 : k1, src);
    const int e = __shfl_sync(0xffffffffu, c < 32 ? v0 : v1, src);
    if (d2 >= kSelfKey) break;  // the cell itself and padding sort last
    // a cell can cut the polygon only if it is nearer than twice its circumradius
    // (d2 carries a relative error below 1e-6; the margin is 1e-3)
    if (d2 > 4.0f * p.R2 * (1.0f + 1e-3f)) break;
    clip(p, s_X[e], s_Y[e], s_id[e], s_tag[e], ikey, sc, inv_scale, lane);
    if (p.err) break;
  }
  __syncwarp();
}

__global__ void __launch_bounds__(kRepairWarps * 32) k_repair(RepairArgs g) {
  __shared__ int s_id[kRepairWarps][kCand];
  __shared__ long long s_X[kRepairWarps][kCand], s_Y[kRepairWarps][kCand];
  __shared__ float s_d2[kRepairWarps][kCand];
  __shared__ int s_tag[kRepairWarps][kCand];  // perturbation keys, loaded with the positions
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gw = blockIdx.x * kRepairWarps + wib, nw = gridDim.x * kRepairWarps;
  // stop the round loop unless this round's check asks for another
  if (g.dyn && g.loop && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(g.loop, 0);
  const int which_in = g.dyn ? (g.ctl->round_count & 1) : g.which_in;
  const int* list_in = g.dyn ? (which_in ? g.lists[1] : g.lists[0]) : g.list_in;
  const int total = g.all_cells ? g.n : g.ctl->count[which_in];
  // the list this round's check fills must start empty
  if (!g.all_cells && blockIdx.x == 0 && threadIdx.x == 0) g.ctl->count[which_in ^ 1] = 0;
  if (total == 0) return;
  const int cur = g.ctl->cur;
  const size_t N = (size_t)g.n;
  const long long* __restrict__ X = g.X + cur * N;
  const long long* __restrict__ Y = g.Y + cur * N;
  if (blockIdx.x == 0 && threadIdx.x == 0 && !g.all_cells) {
    if (!g.dyn) atomicAdd(&g.ctl->round_count, 1);  // counted by the check otherwise
    atomicAdd((unsigned long long*)&g.ctl->repaired_total, (unsigned long long)total);
  }

  for (int item = gw; item < total; item += nw) {
    const int i = g.all_cells ? item : list_in[item];
    const Rep R = g.reps[g.rep[i]];
    const long long Xi = X[i], Yi = Y[i];
    const int ikey = g.tag[i];
    const float sc = (float)R.inv_scale;
    // keep the old ring for the consistency check
    const int oc = g.cnt[i];
    if (lane < CG_RING) g.old_nbr[(size_t)i * CG_RING + lane] = g.nbr[(size_t)i * CG_RING + lane];
    if (lane == 0) g.old_cnt[i] = oc;

    // initial polygon: the square of half-width W (vertices (+-W, +-W)), cut
    // out by four phantom generators at (+-2W, 0) and (0, +-2W)
    Poly p;
    p.m = 4;
    p.err = 0;
    p.gX = (lane == 0) ? R.W2 : (lane == 2 ? -R.W2 : 0);
    p.gY = (lane == 1) ? R.W2 : (lane == 3 ? -R.W2 : 0);
    p.gid = -1 - (lane & 3);
    p.gkey = kPhantomKey + (lane & 3);
    {
      const float W = 0.5f * i2f_scaled(R.W2, sc);  // power of two: exact
      p.r2 = 2.0f * W * W;
      p.R2 = p.r2;
    }
    int bxi, byi;
    bin_of_grid(R, Xi, Yi, bxi, byi);
    const float bs = (float)R.bsx;  // every bin is at least this wide
    const int kmax = min((R.nbx - 1) / 2, (R.nby - 1) / 2);
    int nbuf = 0;
    bool done = false;
    // rings 0..2 (25 bins) are gathered in one pass, one bin per lane, unless
    // they hold more candidates than the buffer; then ring by ring
    bool batch = kmax >= 2;
    for (int k = 0; k <= kmax && !done && !p.err; ++k) {
      const bool first = batch && k == 0;
      const int nring = first ? 25 : ((k == 0) ? 1 : 8 * k);
      bool retry = false;
      for (int base = 0; base < nring && !p.err; base += 32) {
        const int idx = base + lane;
        int start = 0, count = 0;
        if (idx < nring) {
          int dx, dy;
          if (first) ring_bin(idx == 0 ? 0 : (idx <= 8 ? 1 : 2), idx == 0 ? 0 : (idx <= 8 ? idx - 1 : idx - 9), dx, dy);
          else ring_bin(k, idx, dx, dy);
          int bx = bxi + dx, by = byi + dy;
          bx += (bx < 0) ? R.nbx : (bx >= R.nbx ? -R.nbx : 0);
          by += (by < 0) ? R.nby : (by >= R.nby ? -R.nby : 0);
          const int b = R.bin0 + by * R.nbx + bx;
          start = bin_begin(g.bin_start, g.bin_partials, b);
          count = bin_begin(g.bin_start, g.bin_partials, b + 1) - start;
        }
        int incl = count;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += t;
        }
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        if (first && tot > kCand) {
          retry = true;
          break;
        }
        if (nbuf + tot > kCand) {
          process_candidates(p, nbuf, s_id[wib], s_X[wib], s_Y[wib], s_d2[wib], s_tag[wib],
                             ikey, sc, R.inv_scale, lane);
          nbuf = 0;
          if (tot > kCand) p.err = kECAND;
        }
        if (!p.err) {
          int slot = nbuf + incl - count;
          bool same = false;  // another cell on exactly this grid point
          for (int t = 0; t < count; ++t) {
            const int j = g.ids[start + t];
            s_tag[wib][slot] = g.tag[j];
            if (j == i) {
              s_d2[wib][slot] = kSelfKey;  // never clips
              s_id[wib][slot] = j;
              s_X[wib][slot] = 0;
              s_Y[wib][slot] = 0;
            } else {
              const long long dX = min_image_i(X[j] - Xi, R.LX), dY = min_image_i(Y[j] - Yi, R.LY);
              same |= (dX == 0 && dY == 0);
              const float dx = i2f_scaled(dX, sc), dy = i2f_scaled(dY, sc);
              s_d2[wib][slot] = dx * dx + dy * dy;
              s_id[wib][slot] = j;
              s_X[wib][slot] = dX;
              s_Y[wib][slot] = dY;
            }
            ++slot;
          }
          nbuf += tot;
          if (__any_sync(0xffffffffu, same)) p.err = kEDEGEN;  // no bisector between them
        }
        __syncwarp();
      }
      if (retry) {  // the ring-by-ring gathering from ring 0
        batch = false;
        k = -1;
        continue;
      }
      if (p.err) break;
      if (first) k = 2;  // rings 1 and 2 are in the batch
      // rings 0..2 are gathered into one batch before clipping
      if (k < 2 && k < kmax) continue;
      process_candidates(p, nbuf, s_id[wib], s_X[wib], s_Y[wib], s_d2[wib], s_tag[wib], ikey,
                         sc, R.inv_scale, lane);
      nbuf = 0;
      // every unvisited cell is farther than k*bs from cell i
      const float reach = k * bs;
      if (reach * reach > 4.0f * p.R2 * (1.0f + 1e-3f)) done = true;
    }
    int err = p.err;
    if (!err && !done) err = kEBOX;
    if (!err) {
      const unsigned ph = __ballot_sync(0xffffffffu, lane < p.m && p.gid < 0);
      if (ph) err = kEBOX;
      if (p.m > CG_RING) err = kERING;
    }
    if (err) {
      if (lane == 0) raise_status(g.ctl, err);
      continue;
    }
    // canonical CCW ring: start at the smallest tag
    int kmin = (lane < p.m) ? p.gkey : INT_MAX;
    int lmin = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int ok = __shfl_xor_sync(0xffffffffu, kmin, o);
      const int ol = __shfl_xor_sync(0xffffffffu, lmin, o);
      if (ok < kmin || (ok == kmin && ol < lmin)) { kmin = ok; lmin = ol; }
    }
    if (lane < p.m) {
      const int slot = (lane - lmin + p.m) % p.m;
      g.nbr[(size_t)i * CG_RING + slot] = p.gid;
    } else if (lane < CG_RING) {
      g.nbr[(size_t)i * CG_RING + lane] = -1;
    }
    if (lane == 0) {
      g.cnt[i] = p.m;
      atomicAnd(&g.flags[i >> 5], ~(1u << (i & 31)));
      if (g.dirty_list && !g.all_cells) {
        const unsigned bit = 1u << (i & 31);
        if (!(atomicOr(&g.dirty_bits[i >> 5], bit) & bit)) g.dirty_list[atomicAdd(&g.ctl->dirty_count, 1)] = i;
      }
    }
  }
}

void launch_repair(const RepairArgs& a, int grid_blocks, cudaStream_t st) {
  if (a.n <= 0) return;
  k_repair<<<grid_blocks, kRepairWarps * 32, 0, st>>>(a);
}

// ---------------------------------------------------------------------------
// Ring consistency after a repair round: j in ring(i) <=> i in ring(j).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool in_ring(const int* nbr, const int* cnt, int j, int i) {
  const int mj = cnt[j];
  const int4* row = reinterpret_cast<const int4*>(nbr + (size_t)j * CG_RING);
  bool found = false;
#pragma unroll
  for (int q = 0; q < CG_RING / 4; ++q) {
    const int4 v = row[q];
    found |= (v.x == i && 4 * q + 0 < mj) || (v.y == i && 4 * q + 1 < mj) || (v.z == i && 4 * q + 2 < mj) ||
             (v.w == i && 4 * q + 3 < mj);
  }
  return found;
}

__device__ __forceinline__ void flag_into(unsigned* flags, int* list, int* count, int c) {
  const unsigned bit = 1u << (c & 31);
  const unsigned old = atomicOr(&flags[c >> 5], bit);
  if (!(old & bit)) list[atomicAdd(count, 1)] = c;
}

// One warp per listed cell i: lanes 0-15 take the entries of i's new ring
// (j must list i), lanes 16-31 those of its old ring (a neighbour i dropped
// must have dropped i too).  Every lookup of a ring row runs in parallel.
__global__ void k_check(CheckArgs g) {
  const int which_in = g.dyn ? (g.ctl->round_count & 1) : g.which_in;
  const int which_out = which_in ^ 1;
  const int* list_in = g.dyn ? (which_in ? g.lists[1] : g.lists[0]) : g.list_in;
  int* list_out = g.dyn ? (which_out ? g.lists[1] : g.lists[0]) : g.list_out;
  const int total = g.all_cells ? g.n : g.ctl->count[which_in];
  int* count_out = &g.ctl->count[which_out];
  const int lane = threadIdx.x & 31, a = lane & 15;
  const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  for (int item = warp; item < total; item += nwarps) {  // warp-uniform
    const int i = g.all_cells ? item : list_in[item];
    const int m = g.cnt[i];
    const int rj = (lane < 16 && a < m) ? g.nbr[(size_t)i * CG_RING + a] : -1;  // new ring of i
    int j = -1;
    bool mine = false;
    if (lane < 16) {
      j = rj;
      mine = a < m;
    } else if (a < g.old_cnt[i]) {
      j = g.old_nbr[(size_t)i * CG_RING + a];
      mine = j >= 0 && j < g.n;
    }
    bool kept = false;  // j still in the new ring of i
#pragma unroll
    for (int b = 0; b < 16; ++b) kept |= (__shfl_sync(0xffffffffu, rj, b) == j);
    bool flag = false;
    if (mine) {
      const bool lists_i = in_ring(g.nbr, g.cnt, j, i);
      flag = (lane < 16) ? !lists_i : (!kept && lists_i);
    }
    if (flag) flag_into(g.flags, list_out, count_out, j);
    const bool bad = __any_sync(0xffffffffu, flag);
    if (bad && g.last_round && !g.dyn && lane == 0) raise_status(g.ctl, kEREPAIR_CAP);
  }
  if (!g.dyn) return;  // uniform over the grid
  if (last_block(&g.ctl->done) && threadIdx.x == 0) {
    Ctl* ctl = g.ctl;
    if (ctl->round_count == 0 && which_in == 0) {  // first round: the test's flags
      ctl->last_flagged = total;
      ctl->flagged_total += total;
    }
    const int produced = *(volatile int*)count_out;
    const int r = ctl->round_count + (total > 0 ? 1 : 0);
    ctl->round_count = r;
    ctl->loop_total += 1;
    if (produced > 0) {
      if (r >= g.cap) atomicCAS(&ctl->status, 0, (int)kEREPAIR_CAP);
      else if (g.loop) cudaGraphSetConditional(g.loop, 1);
    }
  }
}

void launch_check(const CheckArgs& a, int grid_blocks, cudaStream_t st) {
  if (a.n <= 0) return;
  k_check<<<grid_blocks, 256, 0, st>>>(a);
}

// ---------------------------------------------------------------------------
// State preparation and user-order transfers.
// ---------------------------------------------------------------------------
__global__ void k_snap(int n, const Rep* reps, const int* rep, const double* xin, const double* yin, double* x,
                       double* y, long long* X, long long* Y, Ctl* ctl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Rep R = reps[rep[i]];
  const double xv = xin[i], yv = yin[i];
  if (!(xv >= -R.Lx && xv < 2.0 * R.Lx && yv >= -R.Ly && yv < 2.0 * R.Ly)) {
    raise_status(ctl, kEINVAL);
    x[i] = y[i] = 0.0;
    X[i] = Y[i] = 0;
    return;
  }
  long long Xv = (long long)rint(xv * R.scale), Yv = (long long)rint(yv * R.scale);
  if (Xv >= R.LX) Xv -= R.LX; else if (Xv < 0) Xv += R.LX;
  if (Yv >= R.LY) Yv -= R.LY; else if (Yv < 0) Yv += R.LY;
  X[i] = Xv;
  Y[i] = Yv;
  x[i] = (double)Xv * R.inv_scale;
  y[i] = (double)Yv * R.inv_scale;
}

void launch_snap(int n, const Rep* reps, const int* rep, const double* xin, const double* yin, double* x, double* y,
                 long long* X, long long* Y, Ctl* ctl, cudaStream_t st) {
  if (n <= 0) return;
  k_snap<<<(n + 255) / 256, 256, 0, st>>>(n, reps, rep, xin, yin, x, y, X, Y, ctl);
}

// Inputs handed in from outside must be finite (directors, p0, v0).
__global__ void k_check_finite(int n, const double* v, Ctl* ctl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !isfinite(v[i])) raise_status(ctl, kEINVAL);
}
void launch_check_finite(int n, const double* v, Ctl* ctl, cudaStream_t st) {
  if (n > 0) k_check_finite<<<(n + 255) / 256, 256, 0, st>>>(n, v, ctl);
}

__global__ void k_gather_d(int n, const int* tag, const double* src, double* dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[tag[i]] = src[i];
}
// Current positions (buffer ctl->cur of x2, y2, each [2][n]) in user order.
__global__ void k_gather_cur_xy(int n, const int* tag, const double* x2, const double* y2, const Ctl* ctl,
                                int pending, double* dst_x, double* dst_y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const size_t off = (size_t)(ctl->cur ^ pending) * n + i;
  const int u = tag[i];
  if (dst_x) dst_x[u] = x2[off];
  if (dst_y) dst_y[u] = y2[off];
}
__global__ void k_scatter_d(int n, const int* tag, const double* src, double* dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[tag[i]];
}
__global__ void k_gather_ring(int n, const int* tag, const int* cnt, const int* nbr, int* cnt_u, int* nbr_u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int t = tag[i], m = cnt[i];
  cnt_u[t] = m;
  for (int a = 0; a < CG_RING; ++a) {
    const int j = (a < m) ? nbr[(size_t)i * CG_RING + a] : -1;
    nbr_u[(size_t)t * CG_RING + a] = (j >= 0 && j < n) ? tag[j] : -1;
  }
}
__global__ void __launch_bounds__(1024) k_reduce_sum(int n, const double* v, double* out) {
  __shared__ double buf[1024];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 1024) s += v[i];
  buf[threadIdx.x] = s;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (threadIdx.x < o) buf[threadIdx.x] += buf[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = buf[0];
}

void launch_gather_d(int n, const int* tag, const double* src, double* dst_user, cudaStream_t st) {
  if (n > 0) k_gather_d<<<(n + 255) / 256, 256, 0, st>>>(n, tag, src, dst_user);
}
void launch_gather_cur_xy(int n, const int* tag, const double* x2, const double* y2, const Ctl* ctl, int pending,
                          double* dst_x, double* dst_y, cudaStream_t st) {
  if (n > 0) k_gather_cur_xy<<<(n + 255) / 256, 256, 0, st>>>(n, tag, x2, y2, ctl, pending, dst_x, dst_y);
}
void launch_scatter_d(int n, const int* tag, const double* src_user, double* dst, cudaStream_t st) {
  if (n > 0) k_scatter_d<<<(n + 255) / 256, 256, 0, st>>>(n, tag, src_user, dst);
}

__global__ void k_scatter_i(int n, const int* tag, const int* src, int* dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[tag[i]];
}
void launch_scatter_i(int n, const int* tag, const int* src_user, int* dst, cudaStream_t st) {
  if (n > 0) k_scatter_i<<<(n + 255) / 256, 256, 0, st>>>(n, tag, src_user, dst);
}

// Halo exchange of a decomposed system.  The exchanged values are the
// pending positions (position buffer cur ^ 1: where the next step starts),
// as grid coordinates of the larger box a framed replica belongs to, so a
// cell's position crosses from one domain's frame to another's exactly.
// slot[u] (user order) is the cell's place in the message, or -1.
__global__ void k_halo_pack(int n, const int* tag, const int* slot, const Rep* reps, const int* rep, const Ctl* ctl,
                            const long long* X2, const long long* Y2, long long* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int s = slot[tag[i]];
  if (s < 0) return;
  const size_t nxt = (size_t)(ctl->cur ^ 1) * n + i;
  const Rep R = reps[rep[i]];
  long long X = X2[nxt], Y = Y2[nxt];
  if (R.framed) {
    X += R.X0;
    if (X >= R.LXg) X -= R.LXg;
    Y += R.Y0;
    if (Y >= R.LYg) Y -= R.LYg;
  }
  out[2 * (size_t)s] = X;
  out[2 * (size_t)s + 1] = Y;
}

// The received positions replace the pending positions of the listed cells;
// a position that does not fall inside the replica's frame (a halo cell that
// drifted out of the domain's box: the halo must be re-partitioned) raises
// CG_EINVAL and leaves the cell unchanged.
__global__ void k_halo_unpack(int n, const int* tag, const int* slot, const Rep* reps, const int* rep, Ctl* ctl,
                              const long long* in, double* x2, double* y2, long long* X2, long long* Y2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int s = slot[tag[i]];
  if (s < 0) return;
  const Rep R = reps[rep[i]];
  long long X = in[2 * (size_t)s], Y = in[2 * (size_t)s + 1];
  const long long LXo = R.framed ? R.LXg : R.LX, LYo = R.framed ? R.LYg : R.LY;
  if (X < 0 || X >= LXo || Y < 0 || Y >= LYo) {
    raise_status(ctl, kEINVAL);
    return;
  }
  if (R.framed) {
    X -= R.X0;
    if (X < 0) X += R.LXg;
    Y -= R.Y0;
    if (Y < 0) Y += R.LYg;
  }
  if (X >= R.LX || Y >= R.LY) {
    raise_status(ctl, kEINVAL);
    return;
  }
  const size_t nxt = (size_t)(ctl->cur ^ 1) * n + i;
  X2[nxt] = X;
  Y2[nxt] = Y;
  x2[nxt] = i2d_int(X, -R.q);
  y2[nxt] = i2d_int(Y, -R.q);
}

void launch_halo_pack(int n, const int* tag, const int* slot, const Rep* reps, const int* rep, const Ctl* ctl,
                      const long long* X2, const long long* Y2, long long* out, cudaStream_t st) {
  if (n > 0) k_halo_pack<<<(n + 255) / 256, 256, 0, st>>>(n, tag, slot, reps, rep, ctl, X2, Y2, out);
}
void launch_halo_unpack(int n, const int* tag, const int* slot, const Rep* reps, const int* rep, Ctl* ctl,
                        const long long* in, double* x2, double* y2, long long* X2, long long* Y2, cudaStream_t st) {
  if (n > 0) k_halo_unpack<<<(n + 255) / 256, 256, 0, st>>>(n, tag, slot, reps, rep, ctl, in, x2, y2, X2, Y2);
}
void launch_gather_ring(int n, const int* tag, const int* cnt, const int* nbr, int* cnt_user, int* nbr_user,
                        cudaStream_t st) {
  if (n > 0) k_gather_ring<<<(n + 255) / 256, 256, 0, st>>>(n, tag, cnt, nbr, cnt_user, nbr_user);
}
void launch_reduce_sum(int n, const double* v, double* out, cudaStream_t st) {
  k_reduce_sum<<<1, 1024, 0, st>>>(n, v, out);
}

}  // namespace cgk
