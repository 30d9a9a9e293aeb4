// Allocation-free triangulation entry point: cg_triangulate_noalloc().
//
// Some callers cannot call cudaMalloc at all: code running under a device
// memory pool that forbids growth, inside allocator hooks or plugins of other
// runtimes, or in applications that must reserve every byte of device memory
// up front.  For them, this entry point computes the periodic Delaunay
// neighbour rings of a point set using scratch memory that is part of the
// library image itself: a file-scope __device__ array loaded with the module,
// held by every GPU that loads the library until the process exits.
//
// Limits and rules
//  * at most CG_NOALLOC_MAX_CELLS cells and kMaxBins cell-list bins;
//    larger inputs are rejected with CG_EINVAL before any GPU work;
//  * every call reuses the same array and leaves its contents behind; what
//    must start at zero (control word, flags, bin counts, rings) is cleared by
//    each call; two calls whose GPU work overlaps (different streams, or
//    different host threads on one device) race on the array;
//  * the first call on a device looks up the array's device address with
//    cudaGetSymbolAddress and caches it; that first call should therefore
//    come before any stream capture, and a cudaDeviceReset() of the device
//    (which reloads the module elsewhere) ends the use of this function on it;
//  * no cudaMalloc, cudaFree or allocating library routine is called.
#include "../../include/cellgb.h"
#include "cg_device.cuh"
#include "cg_kernels.h"

#include <cmath>
#include <cstring>
#include <mutex>

using namespace cgk;

namespace {

constexpr int kMaxCells = CG_NOALLOC_MAX_CELLS;
constexpr int kMaxBins = 4 * CG_NOALLOC_MAX_CELLS;
constexpr int kScanChunk = 256 * 8;  // bins per scan block of the cell-list kernels
constexpr int kMaxPartials = (kMaxBins + 1 + kScanChunk - 1) / kScanChunk + 1;

// byte offsets inside the static scratch array (all 256-byte aligned)
constexpr size_t al(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kOffCtl = 0;
constexpr size_t kOffRep = kOffCtl + al(sizeof(Ctl));
constexpr size_t kOffX = kOffRep + al(sizeof(Rep));
constexpr size_t kOffY = kOffX + al(8 * (size_t)kMaxCells);
constexpr size_t kOffXi = kOffY + al(8 * (size_t)kMaxCells);
constexpr size_t kOffYi = kOffXi + al(8 * (size_t)kMaxCells);
constexpr size_t kOffTag = kOffYi + al(8 * (size_t)kMaxCells);
constexpr size_t kOffRepIdx = kOffTag + al(4 * (size_t)kMaxCells);
constexpr size_t kOffCnt = kOffRepIdx + al(4 * (size_t)kMaxCells);
constexpr size_t kOffNbr = kOffCnt + al(4 * (size_t)kMaxCells);
constexpr size_t kOffOldCnt = kOffNbr + al(4 * (size_t)kMaxCells * CG_RING);
constexpr size_t kOffOldNbr = kOffOldCnt + al(4 * (size_t)kMaxCells);
constexpr size_t kOffFlags = kOffOldNbr + al(4 * (size_t)kMaxCells * CG_RING);
constexpr size_t kOffList0 = kOffFlags + al(4 * (size_t)((kMaxCells + 31) / 32));
constexpr size_t kOffList1 = kOffList0 + al(4 * (size_t)kMaxCells);
constexpr size_t kOffBinCount = kOffList1 + al(4 * (size_t)kMaxCells);
constexpr size_t kOffBinStart = kOffBinCount + al(4 * (size_t)kMaxBins);
constexpr size_t kOffPartials = kOffBinStart + al(4 * (size_t)(kMaxBins + 1));
constexpr size_t kOffCellBin = kOffPartials + al(4 * (size_t)kMaxPartials);
constexpr size_t kOffCellRank = kOffCellBin + al(4 * (size_t)kMaxCells);
constexpr size_t kOffIds = kOffCellRank + al(4 * (size_t)kMaxCells);
constexpr size_t kScratchBytes = kOffIds + al(4 * (size_t)kMaxCells);

}  // namespace

// The scratch itself (about 3.7 MB for 16384 cells).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (looked up once).
int scratch_address(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CG_ECUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return CG_ECUDA;
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return CG_OK;
}

int ceil_log2(double v) {
  int ex;
  const double fr = std::frexp(v, &ex);
  return (fr == 0.5) ? ex - 1 : ex;
}

// Replica constants for one box (same grid and bin rules as cg_create).
bool make_rep(int n, double Lx, double Ly, Rep& p) {
  std::memset(&p, 0, sizeof(p));
  const int e = ceil_log2(std::fmax(Lx, Ly));
  p.q = 50 - e;
  p.scale = std::ldexp(1.0, p.q);
  p.inv_scale = std::ldexp(1.0, -p.q);
  p.LX = (long long)std::rint(std::ldexp(Lx, p.q));
  p.LY = (long long)std::rint(std::ldexp(Ly, p.q));
  p.Lx = std::ldexp((double)p.LX, -p.q);
  p.Ly = std::ldexp((double)p.LY, -p.q);
  p.hLx = 0.5 * p.Lx;
  p.hLy = 0.5 * p.Ly;
  // cell-list bins 2^bshift grid units wide (about one mean spacing, at least
  // 9 per side); the last bin of each row absorbs the remainder of the box
  const double spacing = std::sqrt(p.Lx * p.Ly / n);
  int bshift = (int)std::lround(std::log2(spacing)) + p.q;
  while (bshift > 0 && ((p.LX >> bshift) < 9 || (p.LY >> bshift) < 9)) --bshift;
  p.bshift = bshift;
  p.nbx = (int)(p.LX >> bshift);
  p.nby = (int)(p.LY >> bshift);
  p.bsx = p.bsy = std::ldexp(1.0, bshift - p.q);
  if ((long long)p.nbx * p.nby > kMaxBins) return false;
  const int ew = ceil_log2(std::fmax(p.Lx, p.Ly) / 4.0);
  p.W2 = (long long)std::ldexp(2.0, ew + p.q);
  p.cell0 = 0;
  p.ncell = n;
  p.bin0 = 0;
  return true;
}

__global__ void k_noalloc_index(int n, int* tag, int* rep) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    tag[i] = i;
    rep[i] = 0;
  }
}

}  // namespace

extern "C" int cg_triangulate_noalloc(int32_t n, double Lx, double Ly, const double* d_x, const double* d_y,
                                      int32_t* d_cnt, int32_t* d_nbr, void* stream) {
  if (n < 16 || n > kMaxCells || !d_x || !d_y || !d_cnt || !d_nbr) return CG_EINVAL;
  if (!(Lx > 0) || !(Ly > 0) || !std::isfinite(Lx) || !std::isfinite(Ly)) return CG_EINVAL;
  Rep rep;
  if (!make_rep(n, Lx, Ly, rep)) return CG_EINVAL;
  unsigned char* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Ctl* ctl = reinterpret_cast<Ctl*>(base + kOffCtl);
  Rep* d_rep = reinterpret_cast<Rep*>(base + kOffRep);
  double* x = reinterpret_cast<double*>(base + kOffX);
  double* y = reinterpret_cast<double*>(base + kOffY);
  long long* X = reinterpret_cast<long long*>(base + kOffXi);
  long long* Y = reinterpret_cast<long long*>(base + kOffYi);
  int* tag = reinterpret_cast<int*>(base + kOffTag);
  int* repi = reinterpret_cast<int*>(base + kOffRepIdx);
  int* cnt = reinterpret_cast<int*>(base + kOffCnt);
  int* nbr = reinterpret_cast<int*>(base + kOffNbr);
  unsigned* flags = reinterpret_cast<unsigned*>(base + kOffFlags);
  const int nbins = rep.nbx * rep.nby;

  // state that must start at zero (the array keeps the previous call's contents)
  if (cudaMemsetAsync(ctl, 0, sizeof(Ctl), st) != cudaSuccess) return CG_ECUDA;
  if (cudaMemsetAsync(flags, 0, 4 * (size_t)((n + 31) / 32), st) != cudaSuccess) return CG_ECUDA;
  if (cudaMemsetAsync(base + kOffBinCount, 0, 4 * (size_t)nbins, st) != cudaSuccess) return CG_ECUDA;
  if (cudaMemsetAsync(cnt, 0, 4 * (size_t)n, st) != cudaSuccess) return CG_ECUDA;
  if (cudaMemsetAsync(nbr, 0xff, 4 * (size_t)n * CG_RING, st) != cudaSuccess) return CG_ECUDA;
  if (cudaMemcpyAsync(d_rep, &rep, sizeof(Rep), cudaMemcpyHostToDevice, st) != cudaSuccess) return CG_ECUDA;
  k_noalloc_index<<<(n + 255) / 256, 256, 0, st>>>(n, tag, repi);
  launch_snap(n, d_rep, repi, d_x, d_y, x, y, X, Y, ctl, st);

  CellListArgs cl{};  // every field starts zero or null
  cl.n = n;
  cl.nbins = nbins;
  cl.reps = d_rep;
  cl.rep = repi;
  cl.ctl = ctl;
  cl.X = X;
  cl.Y = Y;
  cl.bin_count = reinterpret_cast<int*>(base + kOffBinCount);
  cl.bin_start = reinterpret_cast<int*>(base + kOffBinStart);
  cl.cell_bin = reinterpret_cast<int*>(base + kOffCellBin);
  cl.cell_rank = reinterpret_cast<int*>(base + kOffCellRank);
  cl.ids = reinterpret_cast<int*>(base + kOffIds);
  cl.scan_partials = reinterpret_cast<int*>(base + kOffPartials);
  cl.only_if_flagged = 0;
  launch_cell_list(cl, st);

  RepairArgs ra{};  // every field starts zero or null
  ra.n = n;
  ra.reps = d_rep;
  ra.rep = repi;
  ra.ctl = ctl;
  ra.x = x;
  ra.y = y;
  ra.X = X;
  ra.Y = Y;
  ra.tag = tag;
  ra.bin_start = cl.bin_start;
  ra.bin_partials = cl.scan_partials;
  ra.ids = cl.ids;
  ra.cnt = cnt;
  ra.nbr = nbr;
  ra.old_cnt = reinterpret_cast<int*>(base + kOffOldCnt);
  ra.old_nbr = reinterpret_cast<int*>(base + kOffOldNbr);
  ra.flags = flags;
  ra.list_in = reinterpret_cast<int*>(base + kOffList0);
  ra.which_in = 0;
  ra.all_cells = 1;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  launch_repair(ra, sms * 8, st);

  CheckArgs ck{};  // every field starts zero or null
  ck.n = n;
  ck.ctl = ctl;
  ck.cnt = cnt;
  ck.nbr = nbr;
  ck.old_cnt = ra.old_cnt;
  ck.old_nbr = ra.old_nbr;
  ck.flags = flags;
  ck.list_in = ra.list_in;
  ck.list_out = reinterpret_cast<int*>(base + kOffList1);
  ck.which_in = 0;
  ck.which_out = 1;
  ck.last_round = 1;
  ck.all_cells = 1;
  launch_check(ck, (n + 255) / 256, st);

  launch_gather_ring(n, tag, cnt, nbr, d_cnt, d_nbr, st);
  if (cudaGetLastError() != cudaSuccess) return CG_ECUDA;
  // the status word read on the caller's stream, behind the kernels above
  int status = 0;
  if (cudaMemcpyAsync(&status, &ctl->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return CG_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return CG_ECUDA;
  return status;
}
