// C ABI of libcellgb.so: context, workspace layout, step graph, getters.
#include "../../include/cellgb.h"
#include "cg_device.cuh"
#include "cg_kernels.h"
#include "cg_graph.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

using namespace cgk;

namespace {

struct Layout {
  size_t total = 0;
  size_t take(size_t bytes) {
    size_t off = total;
    total += (bytes + 255) & ~(size_t)255;
    return off;
  }
};

struct Offsets {
  size_t key, rank, perm, key_count, key_start, key_partials, theta_alt, p0_alt, v0_alt, tag_alt, rep_alt,
      cnt_alt, nbr_alt;
  size_t x, y, X, Y, theta, p0, v0, A, P, Fx, Fy, ecell, tmp, tmp2, scalar, nrm, xi;
  size_t tag, nid, nid_alt, rep, cnt, nbr, old_cnt, old_nbr;
  size_t fs, s, w, order;
  size_t flags, list0, list1, dirty_list, dirty_bits, fix_list, fix_bits;
  size_t bin_count, bin_start, partials, cell_bin, cell_rank, ids;
  size_t reps, ctl, dir_tab;
  size_t io_v0, io_xy;  // staging of cg_run_io: [2][n] v0, [2][2][n] positions
  size_t total;
};

constexpr int kScanChunkHost = 256 * 8;

Offsets layout(int64_t N, int64_t NB, int64_t NK, int R) {
  Layout L;
  Offsets o;
  const size_t d = sizeof(double), i4 = sizeof(int), i8 = sizeof(long long);
  o.key = L.take(N * i4);
  o.rank = L.take(N * i4);
  o.perm = L.take(N * i4);
  o.key_count = L.take(NK * i4);
  o.key_start = L.take((NK + 1) * i4);
  o.key_partials = L.take(((NK + 1 + kScanChunkHost - 1) / kScanChunkHost + 1) * i4);
  o.theta_alt = L.take(N * d);
  o.p0_alt = L.take(N * d);
  o.v0_alt = L.take(N * d);
  o.tag_alt = L.take(N * i4);
  o.rep_alt = L.take(N * i4);
  o.cnt_alt = L.take(N * i4);
  o.nbr_alt = L.take(N * CG_RING * i4);
  o.x = L.take(2 * N * d);
  o.y = L.take(2 * N * d);
  o.X = L.take(2 * N * i8);
  o.Y = L.take(2 * N * i8);
  o.theta = L.take(N * d);
  o.p0 = L.take(N * d);
  o.v0 = L.take(N * d);
  o.A = L.take(N * d);
  o.P = L.take(N * d);
  o.Fx = L.take(N * d);
  o.Fy = L.take(N * d);
  o.ecell = L.take(N * d);
  o.tmp = L.take(N * d);
  o.tmp2 = L.take(N * d);
  o.scalar = L.take(4 * d);
  o.nrm = L.take(N * sizeof(double2));
  o.xi = L.take(N * d);
  o.tag = L.take(N * i4);
  o.nid = L.take(N * i4);
  o.nid_alt = L.take(N * i4);
  o.rep = L.take(N * i4);
  o.cnt = L.take(N * i4);
  o.nbr = L.take(N * CG_RING * i4);
  o.old_cnt = L.take(N * i4);
  o.old_nbr = L.take(N * CG_RING * i4);
  o.fs = L.take(N * CG_RING * sizeof(double2));
  o.s = L.take(N * CG_RING * sizeof(double2));
  o.w = L.take(N * CG_RING * sizeof(double2));
  o.order = L.take(N * i4);
  o.flags = L.take(((N + 31) / 32) * 4);
  o.list0 = L.take(N * i4);
  o.list1 = L.take(N * i4);
  o.dirty_list = L.take(N * i4);
  o.dirty_bits = L.take(((N + 31) / 32) * 4);
  o.fix_list = L.take(N * i4);
  o.fix_bits = L.take(((N + 31) / 32) * 4);
  o.bin_count = L.take(NB * i4);
  o.bin_start = L.take((NB + 1) * i4);
  o.partials = L.take(((NB + 1 + kScanChunkHost - 1) / kScanChunkHost + 1) * i4);
  o.cell_bin = L.take(N * i4);
  o.cell_rank = L.take(N * i4);
  o.ids = L.take(N * i4);
  o.reps = L.take(R * sizeof(Rep));
  o.ctl = L.take(sizeof(Ctl));
  o.dir_tab = L.take(kDirTabEntries * sizeof(double2));
  o.io_v0 = L.take(2 * N * d);
  o.io_xy = L.take(4 * N * d);
  o.total = L.total;
  return o;
}

struct RepHost {
  Rep r;
};

// Smallest e with 2^e >= v.
int ceil_log2(double v) {
  int ex;
  double fr = std::frexp(v, &ex);
  return (fr == 0.5) ? ex - 1 : ex;
}

bool build_reps(int R, const cg_replica* reps, std::vector<Rep>& out, int64_t& N, int64_t& NB, int64_t& NK,
                std::string& err) {
  out.resize(R);
  N = 0;
  NB = 0;
  NK = 0;
  for (int r = 0; r < R; ++r) {
    const cg_replica& c = reps[r];
    if (c.n < 16 || !(c.Lx > 0) || !(c.Ly > 0) || !std::isfinite(c.Lx) || !std::isfinite(c.Ly)) {
      err = "replica " + std::to_string(r) + ": need n >= 16 and positive finite box";
      return false;
    }
    Rep& p = out[r];
    std::memset(&p, 0, sizeof(p));
    const int e = ceil_log2(std::fmax(c.Lx, c.Ly));
    p.q = 50 - e;
    p.scale = std::ldexp(1.0, p.q);
    p.inv_scale = std::ldexp(1.0, -p.q);
    p.LX = (long long)std::rint(std::ldexp(c.Lx, p.q));
    p.LY = (long long)std::rint(std::ldexp(c.Ly, p.q));
    p.Lx = std::ldexp((double)p.LX, -p.q);
    p.Ly = std::ldexp((double)p.LY, -p.q);
    p.hLx = 0.5 * p.Lx;
    p.hLy = 0.5 * p.Ly;
    // cell-list bins 2^bshift grid units wide (about one mean spacing, at least
    // 9 per side); the last bin of each row absorbs the remainder of the box
    const double spacing = std::sqrt(p.Lx * p.Ly / c.n);
    int bshift = (int)std::lround(std::log2(spacing)) + p.q;
    while (bshift > 0 && ((p.LX >> bshift) < 9 || (p.LY >> bshift) < 9)) --bshift;
    p.bshift = bshift;
    p.nbx = (int)(p.LX >> bshift);
    p.nby = (int)(p.LY >> bshift);
    p.bsx = p.bsy = std::ldexp(1.0, bshift - p.q);
    // initial repair square: half-width W = 2^ceil(log2(max(L)/4)) >= L/4
    const int ew = ceil_log2(std::fmax(p.Lx, p.Ly) / 4.0);
    p.W2 = (long long)std::ldexp(2.0, ew + p.q);
    p.cell0 = (int)N;
    p.ncell = c.n;
    p.bin0 = (int)NB;
    p.v0 = c.v0;
    p.p0 = c.p0;
    // Hilbert sort grid: the smallest power of two covering the bin grid
    p.hord = std::max(1, ceil_log2((double)std::max(p.nbx, p.nby)));
    p.hshift = std::max(0, ceil_log2((double)std::max(p.LX, p.LY)) - p.hord);
    p.hkey0 = (int)NK;
    N += c.n;
    NB += (int64_t)p.nbx * p.nby;
    NK += (int64_t)1 << (2 * p.hord);
    if (N > (int64_t)1 << 30 || NB > (int64_t)1 << 30 || NK > (int64_t)1 << 30 || p.hord > 15) {
      err = "too many cells or bins";
      return false;
    }
  }
  return true;
}

}  // namespace

struct cg_ctx {
  int R = 0;
  int64_t N = 0, NB = 0, NK = 0;
  int64_t host_step = 0;  // steps enqueued (decides when to re-sort)
  cg_params par{};
  std::vector<Rep> reps;
  char* ws = nullptr;
  Offsets off{};
  cudaStream_t stream = nullptr;    // user stream
  cudaStream_t capture = nullptr;   // private stream used for graph capture
  cudaStream_t side[3] = {nullptr, nullptr, nullptr};  // branches of the captured step
  cudaEvent_t fork = nullptr, join_dir = nullptr, join_list = nullptr, join_terms = nullptr;
  // cg_run_io: copy streams and the events that order the double-buffered staging
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t in_ready[2] = {}, in_free[2] = {}, out_ready[2] = {}, out_free[2] = {};
  cg_launch launch{4, 4, 4, 1, 0, 8, 1, 5, 0};    // launch shapes of the step graph
  std::vector<cg_replica> user_reps;           // as passed to cg_create
  cudaGraphExec_t step_exec = nullptr;
  int graph_steps = 0;
  int seen_status = 0;  // a device status read back earlier (the context then stays refused)
  std::string last_error;

  template <class T>
  T* at(size_t o) const { return reinterpret_cast<T*>(ws + o); }
  Ctl* ctl() const { return at<Ctl>(off.ctl); }
};

namespace {

int fail(cg_ctx* c, int code, const std::string& msg) {
  if (c) c->last_error = msg;
  return code;
}

#define CG_CUDA(ctx, call)                                                                 \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(ctx, CG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));      \
  } while (0)

GeomArgs geom_args(cg_ctx* c) {
  GeomArgs g{};  // every field starts zero or null
  g.n = (int)c->N;
  g.reps = c->at<Rep>(c->off.reps);
  g.rep = c->at<int>(c->off.rep);
  g.ctl = c->ctl();
  g.X = c->at<long long>(c->off.X);
  g.Y = c->at<long long>(c->off.Y);
  g.cnt = c->at<int>(c->off.cnt);
  g.nbr = c->at<int>(c->off.nbr);
  g.p0 = c->at<double>(c->off.p0);
  g.A0 = c->par.A0;
  g.sqrtA0 = std::sqrt(c->par.A0);
  g.KA = c->par.KA;
  g.KP = c->par.KP;
  g.A = c->at<double>(c->off.A);
  g.P = c->at<double>(c->off.P);
  g.energy_out = nullptr;
  g.fs = c->at<double2>(c->off.fs);
  g.s = c->at<double2>(c->off.s);
  g.w = c->at<double2>(c->off.w);
  g.list = nullptr;
  g.list_count = nullptr;
  g.list_bits = nullptr;
  g.tolerant = 0;
  g.order = (c->launch.ring_order & 1) ? c->at<int>(c->off.order) : nullptr;
  return g;
}

ForceArgs force_args(cg_ctx* c, int integrate) {
  ForceArgs f{};  // every field starts zero or null
  f.n = (int)c->N;
  f.reps = c->at<Rep>(c->off.reps);
  f.rep = c->at<int>(c->off.rep);
  f.ctl = c->ctl();
  f.cnt = c->at<int>(c->off.cnt);
  f.nbr = c->at<int>(c->off.nbr);
  f.tag = c->at<int>(c->off.tag);
  f.fs = c->at<double2>(c->off.fs);
  f.s = c->at<double2>(c->off.s);
  f.w = c->at<double2>(c->off.w);
  f.Fx = c->at<double>(c->off.Fx);
  f.Fy = c->at<double>(c->off.Fy);
  f.integrate = integrate;
  f.x = c->at<double>(c->off.x);
  f.y = c->at<double>(c->off.y);
  f.X = c->at<long long>(c->off.X);
  f.Y = c->at<long long>(c->off.Y);
  f.theta = c->at<double>(c->off.theta);
  f.v0 = c->at<double>(c->off.v0);
  f.mu = c->par.mu;
  f.dt = c->par.dt;
  f.noise_amp = std::sqrt(2.0 * c->par.Dr * c->par.dt);
  f.seed = c->par.seed;
  f.nrm = c->at<double2>(c->off.nrm);
  f.xi = c->at<double>(c->off.xi);
  f.order = (c->launch.ring_order & 2) ? c->at<int>(c->off.order) : nullptr;
  return f;
}

// Ring-size grouping of the cells for the geometry and force kernels (always
// a permutation of the cells, so a stale one is only slower, never wrong).
void run_order(cg_ctx* c, cudaStream_t st) {
  launch_order((int)c->N, c->at<int>(c->off.cnt), c->at<int>(c->off.order), st);
}

DirArgs dir_args(cg_ctx* c) {
  DirArgs d{};  // every field starts zero or null
  d.n = (int)c->N;
  d.ctl = c->ctl();
  d.theta = c->at<double>(c->off.theta);
  d.tag = c->at<int>(c->off.nid);  // the noise counter of each cell
  d.seed = c->par.seed;
  d.nrm = c->at<double2>(c->off.nrm);
  d.xi = c->at<double>(c->off.xi);
  d.advance = 0;
  d.noise_amp = std::sqrt(2.0 * c->par.Dr * c->par.dt);
  d.tab = c->at<double2>(c->off.dir_tab);
  return d;
}

DirArgs dir_args_step(cg_ctx* c) {
  DirArgs d = dir_args(c);
  d.advance = 1;
  return d;
}

// Kernels of the chosen precision (cg_params.precision).
bool fp32(const cg_ctx* c) { return c->par.precision == 1; }
void run_geom(const cg_ctx* c, const GeomArgs& a, cudaStream_t st, int blocks = 0) {
  if (fp32(c)) launch_geom_f32(a, st, blocks);
  else launch_geom(a, st, blocks);
}
void run_force(const cg_ctx* c, const ForceArgs& a, cudaStream_t st, int blocks = 0) {
  if (fp32(c)) launch_force_f32(a, st, blocks);
  else launch_force(a, st, blocks);
}
void run_dir(const cg_ctx* c, const DirArgs& a, cudaStream_t st, int blocks = 0) {
  if (fp32(c)) launch_dir_f32(a, st, blocks);
  else launch_dir(a, st, blocks);
}


TestArgs test_args(cg_ctx* c) {
  TestArgs t{};  // every field starts zero or null
  t.n = (int)c->N;
  t.reps = c->at<Rep>(c->off.reps);
  t.rep = c->at<int>(c->off.rep);
  t.ctl = c->ctl();
  t.X = c->at<long long>(c->off.X);
  t.Y = c->at<long long>(c->off.Y);
  t.cnt = c->at<int>(c->off.cnt);
  t.nbr = c->at<int>(c->off.nbr);
  t.tag = c->at<int>(c->off.tag);
  t.flags = c->at<unsigned>(c->off.flags);
  t.list = c->at<int>(c->off.list0);
  t.order = (c->launch.ring_order & 4) ? c->at<int>(c->off.order) : nullptr;
  return t;
}

CellListArgs cell_list_args(cg_ctx* c, int only_if_flagged) {
  CellListArgs a{};  // every field starts zero or null
  a.n = (int)c->N;
  a.nbins = (int)c->NB;
  a.reps = c->at<Rep>(c->off.reps);
  a.rep = c->at<int>(c->off.rep);
  a.ctl = c->ctl();
  a.X = c->at<long long>(c->off.X);
  a.Y = c->at<long long>(c->off.Y);
  a.bin_count = c->at<int>(c->off.bin_count);
  a.bin_start = c->at<int>(c->off.bin_start);
  a.cell_bin = c->at<int>(c->off.cell_bin);
  a.cell_rank = c->at<int>(c->off.cell_rank);
  a.ids = c->at<int>(c->off.ids);
  a.scan_partials = c->at<int>(c->off.partials);
  a.only_if_flagged = only_if_flagged;
  return a;
}

RepairArgs repair_args(cg_ctx* c, int which_in, int all_cells) {
  RepairArgs r{};  // every field starts zero or null
  r.n = (int)c->N;
  r.reps = c->at<Rep>(c->off.reps);
  r.rep = c->at<int>(c->off.rep);
  r.ctl = c->ctl();
  r.x = c->at<double>(c->off.x);
  r.y = c->at<double>(c->off.y);
  r.X = c->at<long long>(c->off.X);
  r.Y = c->at<long long>(c->off.Y);
  r.tag = c->at<int>(c->off.tag);
  r.bin_start = c->at<int>(c->off.bin_start);
  r.bin_partials = c->at<int>(c->off.partials);
  r.ids = c->at<int>(c->off.ids);
  r.cnt = c->at<int>(c->off.cnt);
  r.nbr = c->at<int>(c->off.nbr);
  r.old_cnt = c->at<int>(c->off.old_cnt);
  r.old_nbr = c->at<int>(c->off.old_nbr);
  r.flags = c->at<unsigned>(c->off.flags);
  r.list_in = c->at<int>(which_in ? c->off.list1 : c->off.list0);
  r.which_in = which_in;
  r.all_cells = all_cells;
  r.dyn = 0;
  r.lists[0] = r.lists[1] = nullptr;
  r.loop = 0;
  r.dirty_list = nullptr;
  r.dirty_bits = nullptr;
  return r;
}

CheckArgs check_args(cg_ctx* c, int which_in, int last_round, int all_cells) {
  CheckArgs k{};  // every field starts zero or null
  k.n = (int)c->N;
  k.ctl = c->ctl();
  k.cnt = c->at<int>(c->off.cnt);
  k.nbr = c->at<int>(c->off.nbr);
  k.old_cnt = c->at<int>(c->off.old_cnt);
  k.old_nbr = c->at<int>(c->off.old_nbr);
  k.flags = c->at<unsigned>(c->off.flags);
  k.list_in = c->at<int>(which_in ? c->off.list1 : c->off.list0);
  k.list_out = c->at<int>(which_in ? c->off.list0 : c->off.list1);
  k.which_in = which_in;
  k.which_out = which_in ^ 1;
  k.last_round = last_round;
  k.all_cells = all_cells;
  k.dyn = 0;
  k.cap = 0;
  k.lists[0] = k.lists[1] = nullptr;
  k.loop = 0;
  return k;
}

SortArgs sort_args(cg_ctx* c) {
  SortArgs a{};  // every field starts zero or null
  a.n = (int)c->N;
  a.nkeys = (int)c->NK;
  a.reps = c->at<Rep>(c->off.reps);
  a.ctl = c->ctl();
  a.x = c->at<double>(c->off.x);
  a.y = c->at<double>(c->off.y);
  a.X = c->at<long long>(c->off.X);
  a.Y = c->at<long long>(c->off.Y);
  a.theta = c->at<double>(c->off.theta);
  a.p0 = c->at<double>(c->off.p0);
  a.v0 = c->at<double>(c->off.v0);
  a.tag = c->at<int>(c->off.tag);
  a.rep = c->at<int>(c->off.rep);
  a.cnt = c->at<int>(c->off.cnt);
  a.nbr = c->at<int>(c->off.nbr);
  a.key = c->at<int>(c->off.key);
  a.rank = c->at<int>(c->off.rank);
  a.perm = c->at<int>(c->off.perm);
  a.key_count = c->at<int>(c->off.key_count);
  a.key_start = c->at<int>(c->off.key_start);
  a.key_partials = c->at<int>(c->off.key_partials);
  a.theta_alt = c->at<double>(c->off.theta_alt);
  a.p0_alt = c->at<double>(c->off.p0_alt);
  a.v0_alt = c->at<double>(c->off.v0_alt);
  a.tag_alt = c->at<int>(c->off.tag_alt);
  a.rep_alt = c->at<int>(c->off.rep_alt);
  a.cnt_alt = c->at<int>(c->off.cnt_alt);
  a.nbr_alt = c->at<int>(c->off.nbr_alt);
  a.nid = c->at<int>(c->off.nid);
  a.nid_alt = c->at<int>(c->off.nid_alt);
  return a;
}

int sm_count() {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}
// Per-step repair rounds handle a few hundred flagged cells: a modest
// persistent grid (warps loop over the list) keeps empty rounds cheap.
int repair_grid(const cg_ctx* c) { return sm_count() * c->launch.repair_blocks_per_sm; }
int check_grid(const cg_ctx* c) { return sm_count() * c->launch.check_blocks_per_sm; }
int dir_grid(const cg_ctx* c) { return sm_count() * c->launch.dir_blocks_per_sm; }    // 0: full
int geom_grid(const cg_ctx* c) { return sm_count() * c->launch.geom_blocks_per_sm; }  // 0: full
int test_grid(const cg_ctx* c) { return sm_count() * c->launch.test_blocks_per_sm; }  // 0: full
// Full triangulation: one warp per cell over every cell.
int repair_grid_all(const cg_ctx*) { return sm_count() * 16; }
int check_grid_all(const cg_ctx* c) { return (int)((c->N + 255) / 256); }

// One time step, enqueued on stream st (also used for capture).
// One step as captured into the step graph.  When a step starts, the move of
// Eq. 3 from the current state is already computed (the "pending move", in
// the other position buffer): the step makes it current, then runs three
// branches — the circumcircle test, the cell-list build, and, at low
// priority, the director terms (rotation by the previous noise, n(theta),
// new noise) followed by the geometry and force sets of the new positions,
// which overlaps the latency-bound repair rounds (rings rewritten meanwhile
// are recomputed by the fix-up after the rounds) — and ends with the forces
// and the next pending move, while the force sets are still in L2.  With
// dir_beside_geom the director terms take a fourth branch and run beside the
// geometry instead of before it.
void enqueue_step_prefix(cg_ctx* c, cudaStream_t st) {
  launch_begin_topology(c->ctl(), 1, st);
  cudaEventRecord(c->fork, st);
  cudaStreamWaitEvent(c->side[0], c->fork, 0);
  cudaStreamWaitEvent(c->side[1], c->fork, 0);
  if (c->launch.dir_beside_geom) {
    cudaStreamWaitEvent(c->side[2], c->fork, 0);
    run_dir(c, dir_args_step(c), c->side[2], dir_grid(c));
    cudaEventRecord(c->join_terms, c->side[2]);
  } else {
    run_dir(c, dir_args_step(c), c->side[0], dir_grid(c));
  }
  GeomArgs g = geom_args(c);
  g.tolerant = 1;
  run_geom(c, g, c->side[0], geom_grid(c));
  if (c->launch.force_beside) {
    // the forces and the pending move of every cell, beside the rounds; the
    // cells around rings the rounds rewrite are done again afterwards
    if (c->launch.dir_beside_geom) cudaStreamWaitEvent(c->side[0], c->join_terms, 0);
    ForceArgs f = force_args(c, 1);
    f.tolerant = 1;
    f.fix_list = c->at<int>(c->off.fix_list);
    f.fix_bits = c->at<unsigned>(c->off.fix_bits);
    run_force(c, f, c->side[0]);
  }
  cudaEventRecord(c->join_dir, c->side[0]);
  launch_cell_list(cell_list_args(c, 0), c->side[1]);
  cudaEventRecord(c->join_list, c->side[1]);
  launch_test(test_args(c), st, test_grid(c));
  cudaStreamWaitEvent(st, c->join_list, 0);
}

// After the repair rounds and the concurrent geometry: the geometry of every
// cell whose ring a round rewrote, then the forces and the next pending move
// (with force_beside only of the cells around those rings and of the cells
// the pass beside the rounds could not decide).
void enqueue_step_suffix(cg_ctx* c, cudaStream_t st) {
  cudaStreamWaitEvent(st, c->join_dir, 0);
  if (c->launch.force_beside) {
    ForceFixArgs x{};
    x.n = (int)c->N;
    x.cnt = c->at<int>(c->off.cnt);
    x.nbr = c->at<int>(c->off.nbr);
    x.dirty_list = c->at<int>(c->off.dirty_list);
    x.dirty_count = &c->ctl()->dirty_count;
    x.fix_list = c->at<int>(c->off.fix_list);
    x.fix_bits = c->at<unsigned>(c->off.fix_bits);
    x.ctl = c->ctl();
    launch_force_fix_list(x, sm_count() * 4, st);
  }
  GeomArgs g = geom_args(c);
  g.list = c->at<int>(c->off.dirty_list);
  g.list_count = &c->ctl()->dirty_count;
  g.list_bits = c->at<unsigned>(c->off.dirty_bits);
  // one warp per rewritten ring (about 1% of the cells per step): every cell
  // of the list at once rather than a few per warp one after another
  run_geom(c, g, st, sm_count() * 16);
  if (c->launch.dir_beside_geom) cudaStreamWaitEvent(st, c->join_terms, 0);
  if (c->launch.ring_order) {
    // the ring-size grouping of the next step, from the rings this step
    // leaves, beside the force pass (both only read the rings)
    cudaEventRecord(c->fork, st);
    cudaStreamWaitEvent(c->side[0], c->fork, 0);
    run_order(c, c->side[0]);
    cudaEventRecord(c->join_dir, c->side[0]);
  }
  if (c->launch.force_beside) {
    ForceArgs f = force_args(c, 1);
    f.list = c->at<int>(c->off.fix_list);
    f.list_count = &c->ctl()->force_count;
    f.list_bits = c->at<unsigned>(c->off.fix_bits);
    run_force(c, f, st, sm_count() * 8);
  } else {
    run_force(c, force_args(c, 1), st);
  }
  if (c->launch.ring_order) cudaStreamWaitEvent(st, c->join_dir, 0);
}

// Director terms, geometry, force sets and the pending move of the current
// state (before the first step and after anything outside a step changes the
// positions, directors, step counter, storage order, p0, v0 or the moduli).
enum : int { kPrimeDir = 1, kPrimeGeom = 2, kPrimeMove = 4, kPrimeAll = 7 };
void prime(cg_ctx* c, int what = kPrimeAll) {
  run_order(c, c->stream);
  if (what & kPrimeDir) run_dir(c, dir_args(c), c->stream);
  if (what & kPrimeGeom) run_geom(c, geom_args(c), c->stream);
  if (what & kPrimeMove) run_force(c, force_args(c, 1), c->stream);
}

// One repair round (repair + consistency check) for a conditional loop node:
// the round counter in the control word picks the lists.
void enqueue_repair_round(cg_ctx* c, cudaGraphConditionalHandle h, cudaStream_t st) {
  RepairArgs r = repair_args(c, 0, 0);
  r.dyn = 1;
  r.lists[0] = c->at<int>(c->off.list0);
  r.lists[1] = c->at<int>(c->off.list1);
  r.loop = h;
  r.dirty_list = c->at<int>(c->off.dirty_list);
  r.dirty_bits = c->at<unsigned>(c->off.dirty_bits);
  CheckArgs k = check_args(c, 0, 0, 0);
  k.dyn = 1;
  k.cap = c->par.repair_cap > 0 ? c->par.repair_cap : 4;
  k.lists[0] = c->at<int>(c->off.list0);
  k.lists[1] = c->at<int>(c->off.list1);
  k.loop = h;
  launch_repair(r, repair_grid(c), st);
  launch_check(k, check_grid(c), st);
}

// Full triangulation of the current positions (every cell repaired).
int triangulate_all(cg_ctx* c) {
  cudaStream_t st = c->stream;
  CG_CUDA(c, cudaMemsetAsync(c->at<int>(c->off.cnt), 0, c->N * sizeof(int), st));
  CG_CUDA(c, cudaMemsetAsync(c->at<int>(c->off.nbr), 0xff, c->N * CG_RING * sizeof(int), st));
  CG_CUDA(c, cudaMemsetAsync(c->at<unsigned>(c->off.flags), 0, ((c->N + 31) / 32) * 4, st));
  CG_CUDA(c, cudaMemsetAsync(c->at<int>(c->off.bin_count), 0, c->NB * sizeof(int), st));
  launch_begin_topology(c->ctl(), 0, st);
  launch_cell_list(cell_list_args(c, 0), st);
  launch_repair(repair_args(c, 0, 1), repair_grid_all(c), st);
  launch_check(check_args(c, 0, 1, 1), check_grid_all(c), st);
  launch_begin_topology(c->ctl(), 0, st);
  CG_CUDA(c, cudaGetLastError());
  return CG_OK;
}

int read_status(cg_ctx* c) {
  Ctl h;
  // the control word read on the context's stream (ordered after its work)
  CG_CUDA(c, cudaMemcpyAsync(&h, c->ctl(), sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
  CG_CUDA(c, cudaStreamSynchronize(c->stream));
  if (h.status != 0) {
    c->seen_status = h.status;
    return fail(c, h.status, std::string("device status: ") + cg_status_string(h.status));
  }
  return CG_OK;
}

int load_positions(cg_ctx* c, const double* x, const double* y) {
  cudaStream_t st = c->stream;
  double* tx = c->at<double>(c->off.tmp);
  double* ty = c->at<double>(c->off.tmp2);
  CG_CUDA(c, cudaMemcpyAsync(tx, x, c->N * sizeof(double), cudaMemcpyDefault, st));
  CG_CUDA(c, cudaMemcpyAsync(ty, y, c->N * sizeof(double), cudaMemcpyDefault, st));
  // user order == storage order until the first sort; scatter through tags
  double* sx = c->at<double>(c->off.A);  // staging in storage order
  double* sy = c->at<double>(c->off.P);
  launch_scatter_d((int)c->N, c->at<int>(c->off.tag), tx, sx, st);
  launch_scatter_d((int)c->N, c->at<int>(c->off.tag), ty, sy, st);
  Ctl h;
  CG_CUDA(c, cudaMemcpyAsync(&h, c->ctl(), sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  CG_CUDA(c, cudaStreamSynchronize(st));
  const size_t cur = (size_t)h.cur;
  launch_snap((int)c->N, c->at<Rep>(c->off.reps), c->at<int>(c->off.rep), sx, sy,
              c->at<double>(c->off.x) + cur * c->N, c->at<double>(c->off.y) + cur * c->N,
              c->at<long long>(c->off.X) + cur * c->N, c->at<long long>(c->off.Y) + cur * c->N, c->ctl(), st);
  CG_CUDA(c, cudaGetLastError());
  return CG_OK;
}

// One step as a graph: the prefix, then the repair rounds as a conditional
// while node that stops at the first round leaving no cell flagged.
int build_graph(cg_ctx* c) {
  if (c->step_exec) return CG_OK;
  cudaError_t e = build_loop_graph(
      c->capture, [&](cudaGraphConditionalHandle, cudaStream_t st) { enqueue_step_prefix(c, st); },
      [&](cudaGraphConditionalHandle h, cudaStream_t st) { enqueue_repair_round(c, h, st); },
      [&](cudaStream_t st) { enqueue_step_suffix(c, st); }, &c->step_exec,
      c->launch.dir_low_priority ? (unsigned long long)cudaGraphInstantiateFlagUseNodePriority : 0ull);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->step_exec = nullptr;
    return fail(c, CG_ECUDA, std::string("step graph: ") + cudaGetErrorString(e));
  }
  return CG_OK;
}

// ---------------------------------------------------------------------------
// Backward pass: checkpointed forward run and reverse accumulation.
// ---------------------------------------------------------------------------
struct BwdLayout {
  size_t snap_bytes = 0;                 // one state snapshot
  size_t snaps = 0, seg = 0;             // checkpoints (+ final state), segment states
  size_t v, fsd, sd, wd, gp0, gv0, gKA, gKP, cA, cP, gx, gy, F, red;
  size_t total = 0;
};

BwdLayout bwd_layout(int64_t N, int64_t nsteps, int32_t every) {
  BwdLayout b;
  Layout L;
  const size_t d = sizeof(double), i4 = sizeof(int);
  Layout s;
  s.take(N * d); s.take(N * d); s.take(N * d);           // x, y, theta
  s.take(N * 8); s.take(N * 8);                          // X, Y
  s.take(N * i4); s.take(N * CG_RING * i4);              // cnt, nbr
  s.take(sizeof(Ctl));
  b.snap_bytes = s.total;
  const int64_t nck = (nsteps + every - 1) / every;
  b.snaps = L.take((size_t)(nck + 1) * b.snap_bytes);
  b.seg = L.take((size_t)every * b.snap_bytes);
  b.v = L.take(N * sizeof(double2));
  b.fsd = L.take(N * CG_RING * sizeof(double2));
  b.sd = L.take(N * CG_RING * sizeof(double2));
  b.wd = L.take(N * CG_RING * sizeof(double2));
  b.gp0 = L.take(N * d);
  b.gv0 = L.take(N * d);
  b.gKA = L.take(N * d);
  b.gKP = L.take(N * d);
  b.cA = L.take(N * d);
  b.cP = L.take(N * d);
  b.gx = L.take(N * d);
  b.gy = L.take(N * d);
  b.F = L.take(N * sizeof(double2));
  b.red = L.take(4 * d);
  b.total = L.total;
  return b;
}

Snapshot snapshot_at(char* base, size_t N) {
  Snapshot s;
  Layout L;
  const size_t d = sizeof(double), i4 = sizeof(int);
  s.x = reinterpret_cast<double*>(base + L.take(N * d));
  s.y = reinterpret_cast<double*>(base + L.take(N * d));
  s.theta = reinterpret_cast<double*>(base + L.take(N * d));
  s.X = reinterpret_cast<long long*>(base + L.take(N * 8));
  s.Y = reinterpret_cast<long long*>(base + L.take(N * 8));
  s.cnt = reinterpret_cast<int*>(base + L.take(N * i4));
  s.nbr = reinterpret_cast<int*>(base + L.take(N * CG_RING * i4));
  s.ctl = reinterpret_cast<Ctl*>(base + L.take(sizeof(Ctl)));
  return s;
}

// Saves (save = 1) or restores the state; a restore recomputes what the next
// use needs (`after_restore`: kPrime* flags; the tangent kernels of the
// reverse pass compute their own geometry and need none).
void snapshot(cg_ctx* c, int save, const Snapshot& s, int after_restore = kPrimeAll) {
  launch_snapshot((int)c->N, save, c->ctl(), c->at<double>(c->off.x), c->at<double>(c->off.y),
                  c->at<long long>(c->off.X), c->at<long long>(c->off.Y), c->at<double>(c->off.theta),
                  c->at<int>(c->off.cnt), c->at<int>(c->off.nbr), s, c->stream);
  if (!save && after_restore) prime(c, after_restore);
}

JvpArgs jvp_args(cg_ctx* c, char* bw, const BwdLayout& b) {
  JvpArgs a{};  // every field starts zero or null
  a.n = (int)c->N;
  a.reps = c->at<Rep>(c->off.reps);
  a.rep = c->at<int>(c->off.rep);
  a.ctl = c->ctl();
  a.X = c->at<long long>(c->off.X);
  a.Y = c->at<long long>(c->off.Y);
  a.cnt = c->at<int>(c->off.cnt);
  a.nbr = c->at<int>(c->off.nbr);
  a.p0 = c->at<double>(c->off.p0);
  a.theta = c->at<double>(c->off.theta);
  a.A0 = c->par.A0;
  a.sqrtA0 = std::sqrt(c->par.A0);
  a.KA = c->par.KA;
  a.KP = c->par.KP;
  a.dt = c->par.dt;
  a.dtmu = c->par.dt * c->par.mu;
  a.coefA = a.coefP = nullptr;
  a.v = reinterpret_cast<double2*>(bw + b.v);
  a.A = a.P = nullptr;
  a.Adot = a.Pdot = nullptr;
  a.fs = c->at<double2>(c->off.fs);
  a.s = c->at<double2>(c->off.s);
  a.w = c->at<double2>(c->off.w);
  a.fsd = reinterpret_cast<double2*>(bw + b.fsd);
  a.sd = reinterpret_cast<double2*>(bw + b.sd);
  a.wd = reinterpret_cast<double2*>(bw + b.wd);
  a.gp0 = a.gv0 = a.gKA = a.gKP = nullptr;
  a.F = a.Hv = nullptr;
  a.update = 0;
  return a;
}

int check_bwd(cg_ctx* c, int64_t nsteps, int32_t every, void* d_bw, size_t bytes, BwdLayout& b) {
  if (!c || nsteps < 1 || every < 1 || !d_bw || ((uintptr_t)d_bw & 255)) return CG_EINVAL;
  if (fp32(c)) return fail(c, CG_EINVAL, "the backward pass runs in double precision only");
  b = bwd_layout(c->N, nsteps, every);
  if (bytes < b.total) return CG_EINVAL;
  return CG_OK;
}

}  // namespace

extern "C" {

int cg_workspace_bytes(int32_t R, const cg_replica* reps, size_t* bytes) {
  if (R <= 0 || !reps || !bytes) return CG_EINVAL;
  std::vector<Rep> r;
  int64_t N, NB, NK;
  std::string err;
  if (!build_reps(R, reps, r, N, NB, NK, err)) return CG_EINVAL;
  *bytes = layout(N, NB, NK, R).total;
  return CG_OK;
}

int cg_create(int32_t R, const cg_replica* reps, const cg_params* params, const double* x, const double* y,
              const double* theta, void* d_ws, size_t ws_bytes, void* stream, cg_ctx** out) {
  if (!out) return CG_EINVAL;
  *out = nullptr;
  if (R <= 0 || !reps || !params || !x || !y || !theta || !d_ws) return CG_EINVAL;
  if (((uintptr_t)d_ws & 255) != 0) return CG_EINVAL;
  if (!(params->dt > 0) || !(params->mu >= 0) || !(params->Dr >= 0) || !(params->A0 > 0)) return CG_EINVAL;
  for (double v : {params->A0, params->KA, params->KP, params->mu, params->Dr, params->dt})
    if (!std::isfinite(v)) return CG_EINVAL;
  cg_ctx* c = new (std::nothrow) cg_ctx();
  if (!c) return CG_EINVAL;
  std::string err;
  if (!build_reps(R, reps, c->reps, c->N, c->NB, c->NK, err)) {
    delete c;
    return CG_EINVAL;
  }
  c->R = R;
  c->par = *params;
  c->user_reps.assign(reps, reps + R);
  if (c->par.repair_cap <= 0) c->par.repair_cap = 4;
  if ((c->par.precision != 0 && c->par.precision != 1) || c->par.reserved != 0) {
    delete c;
    return CG_EINVAL;
  }
  // FP64 defaults (measured at N = 262144): the geometry pass and the
  // circumcircle test in ring-size groups (the geometry pass is bound by the
  // FP64 pipe, where idle lanes cost most) with the director terms on a
  // branch of their own beside the geometry.  The FP32 kernels gain
  // more from the plain (coalesced) order and keep the director terms first
  // on the geometry branch.
  if (c->par.precision == 1) {
    c->launch.ring_order = 0;
    c->launch.dir_beside_geom = 0;
    c->launch.dir_blocks_per_sm = 2;
  }
  c->off = layout(c->N, c->NB, c->NK, R);
  if (ws_bytes < c->off.total) {
    delete c;
    return CG_EINVAL;
  }
  c->ws = static_cast<char*>(d_ws);
  c->stream = static_cast<cudaStream_t>(stream);
  int rc = CG_OK;
  do {
    // the critical path (capture stream, cell-list branch) at the highest
    // priority, the director branch at the lowest; the priorities take effect
    // when the graph is instantiated with node priorities (dir_low_priority)
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->capture, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->side[0], cudaStreamNonBlocking, lo);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->side[1], cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->side[2], cudaStreamNonBlocking, lo);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->join_dir, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->join_list, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->join_terms, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->d2h, cudaStreamNonBlocking);
    for (int b = 0; b < 2; ++b)
      for (cudaEvent_t* ev : {&c->in_ready[b], &c->in_free[b], &c->out_ready[b], &c->out_free[b]})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) { rc = fail(c, CG_ECUDA, cudaGetErrorString(e)); break; }
    cudaStream_t st = c->stream;
    // replica table and per-cell constants
    std::vector<int> tag(c->N), rep(c->N);
    std::vector<double> p0(c->N), v0(c->N);
    for (int r = 0; r < R; ++r)
      for (int k = 0; k < c->reps[r].ncell; ++k) {
        int i = c->reps[r].cell0 + k;
        tag[i] = i;
        rep[i] = r;
        p0[i] = c->reps[r].p0;
        v0[i] = c->reps[r].v0;
      }
    Ctl h;
    std::memset(&h, 0, sizeof(h));
#define TRY(call) do { cudaError_t e2 = (call); if (e2 != cudaSuccess) { rc = fail(c, CG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e2)); } } while (0)
    TRY(cudaMemcpyAsync(c->at<Rep>(c->off.reps), c->reps.data(), R * sizeof(Rep), cudaMemcpyHostToDevice, st));
    TRY(cudaMemcpyAsync(c->at<int>(c->off.tag), tag.data(), c->N * sizeof(int), cudaMemcpyHostToDevice, st));
    // noise counters: the cell's index in user order (cg_set_noise_ids may replace them)
    TRY(cudaMemcpyAsync(c->at<int>(c->off.nid), tag.data(), c->N * sizeof(int), cudaMemcpyHostToDevice, st));
    TRY(cudaMemcpyAsync(c->at<int>(c->off.rep), rep.data(), c->N * sizeof(int), cudaMemcpyHostToDevice, st));
    TRY(cudaMemcpyAsync(c->at<double>(c->off.p0), p0.data(), c->N * sizeof(double), cudaMemcpyHostToDevice, st));
    TRY(cudaMemcpyAsync(c->at<double>(c->off.v0), v0.data(), c->N * sizeof(double), cudaMemcpyHostToDevice, st));
    TRY(cudaMemcpyAsync(c->ctl(), &h, sizeof(Ctl), cudaMemcpyHostToDevice, st));
    TRY(cudaMemsetAsync(c->at<int>(c->off.key_count), 0, c->NK * sizeof(int), st));
    TRY(cudaMemsetAsync(c->at<int>(c->off.cnt), 0, c->N * sizeof(int), st));
    TRY(cudaMemcpyAsync(c->at<double>(c->off.tmp), theta, c->N * sizeof(double), cudaMemcpyDefault, st));
#undef TRY
    if (rc) break;
    launch_init_dir_tables(c->at<double2>(c->off.dir_tab), st);
    launch_scatter_d((int)c->N, c->at<int>(c->off.tag), c->at<double>(c->off.tmp), c->at<double>(c->off.theta), st);
    launch_check_finite((int)c->N, c->at<double>(c->off.theta), c->ctl(), st);
    rc = load_positions(c, x, y);
    if (rc) break;
    launch_sort(sort_args(c), st);  // spatial order before the first triangulation
    if (cudaMemsetAsync(c->at<unsigned>(c->off.dirty_bits), 0, ((c->N + 31) / 32) * 4, st) != cudaSuccess ||
        cudaMemsetAsync(c->at<unsigned>(c->off.fix_bits), 0, ((c->N + 31) / 32) * 4, st) != cudaSuccess) {
      rc = fail(c, CG_ECUDA, "clearing the dirty bitmap");
      break;
    }
    rc = triangulate_all(c);
    if (rc) break;
    prime(c);
    rc = read_status(c);
    if (rc) break;
    rc = build_graph(c);
  } while (0);
  if (rc) {
    cg_destroy(c);
    return rc;
  }
  *out = c;
  return CG_OK;
}

int cg_step(cg_ctx* c, int64_t nsteps) {
  if (!c || nsteps < 0) return CG_EINVAL;
  for (int64_t s = 0; s < nsteps; ++s) {
    if (c->par.sort_every > 0 && c->host_step > 0 && c->host_step % c->par.sort_every == 0) {
      launch_sort(sort_args(c), c->stream);
      prime(c);
    }
    CG_CUDA(c, cudaGraphLaunch(c->step_exec, c->stream));
    ++c->host_step;
  }
  return CG_OK;
}

int cg_run_io(cg_ctx* c, int64_t nsteps, const double* v0, int64_t v0_stride, double* x, double* y,
              int64_t out_stride) {
  if (!c || nsteps < 0 || v0_stride < 0 || out_stride < 0) return CG_EINVAL;
  // no synchronisation on entry: a status raised by earlier work is returned
  // at the end (the status word keeps the first one); one already read back
  // refuses the call
  if (c->seen_status)
    return fail(c, c->seen_status, std::string("device status: ") + cg_status_string(c->seen_status));
  const size_t N = (size_t)c->N;
  const int n = (int)c->N;
  cudaStream_t st = c->stream;
  const int* tag = c->at<int>(c->off.tag);
  // several steps: the uploads on a stream of their own, overlapping the
  // previous step's kernels; one step: the upload on the context's stream
  // (the step needs it first).  The downloads always take a stream of their
  // own: the positions after a step are its pending move, complete before
  // the step starts, so they are gathered then and downloaded while the
  // step's kernels run
  const bool sep = nsteps > 1;
  cudaStream_t sin = sep ? c->h2d : st, sout = c->d2h;
  // device buffers are read and written by the kernels in place (no staging
  // copy); host buffers, page-locked or not, go through staging and the copy
  // engines, which move them faster than the kernels' own loads and stores
  // across the host link
  auto addressable = [](const void* p) -> const void* {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return a.type == cudaMemoryTypeDevice ? p : nullptr;
  };
  const double* dv0 = static_cast<const double*>(addressable(v0));
  double* dx = static_cast<double*>(const_cast<void*>(addressable(x)));
  double* dy = static_cast<double*>(const_cast<void*>(addressable(y)));
  const bool direct_out = (!x || dx) && (!y || dy);
  for (int64_t k = 0; k < nsteps; ++k) {
    const int b = (int)(k & 1);
    if (v0 && dv0) {
      // this step's v0 read in place, the pending move redone with it
      ForceArgs f = force_args(c, 2);
      f.v0_user = dv0 + k * v0_stride;
      run_force(c, f, st);
    } else if (v0) {
      // H2D into staging b once the scatter that last read it is done
      double* in = c->at<double>(c->off.io_v0) + b * N;
      if (sep) CG_CUDA(c, cudaStreamWaitEvent(sin, c->in_free[b], 0));
      CG_CUDA(c, cudaMemcpyAsync(in, v0 + k * v0_stride, N * sizeof(double), cudaMemcpyDefault, sin));
      if (sep) {
        CG_CUDA(c, cudaEventRecord(c->in_ready[b], sin));
        CG_CUDA(c, cudaStreamWaitEvent(st, c->in_ready[b], 0));
      }
      // this step's v0 into storage order and the pending move redone with it
      // (as cg_set_v0), in one kernel
      ForceArgs f = force_args(c, 2);
      f.v0_user = in;
      run_force(c, f, st);
      CG_CUDA(c, cudaEventRecord(c->in_free[b], st));
    }
    if (c->par.sort_every > 0 && c->host_step > 0 && c->host_step % c->par.sort_every == 0) {
      launch_sort(sort_args(c), st);
      prime(c);
    }
    // the positions after this step: the pending move, now final
    const double* x2 = c->at<double>(c->off.x);
    const double* y2 = c->at<double>(c->off.y);
    if ((x || y) && direct_out) {
      launch_gather_cur_xy(n, tag, x2, y2, c->ctl(), 1, dx ? dx + k * out_stride : nullptr,
                           dy ? dy + k * out_stride : nullptr, st);
    } else if (x || y) {
      // into staging b once its previous D2H is done, then downloaded beside
      // the step
      double* out = c->at<double>(c->off.io_xy) + 2 * b * N;
      CG_CUDA(c, cudaStreamWaitEvent(st, c->out_free[b], 0));
      launch_gather_cur_xy(n, tag, x2, y2, c->ctl(), 1, out, out + N, st);
      CG_CUDA(c, cudaEventRecord(c->out_ready[b], st));
      CG_CUDA(c, cudaStreamWaitEvent(sout, c->out_ready[b], 0));
      if (x) CG_CUDA(c, cudaMemcpyAsync(x + k * out_stride, out, N * sizeof(double), cudaMemcpyDefault, sout));
      if (y) CG_CUDA(c, cudaMemcpyAsync(y + k * out_stride, out + N, N * sizeof(double), cudaMemcpyDefault, sout));
      CG_CUDA(c, cudaEventRecord(c->out_free[b], sout));
    }
    CG_CUDA(c, cudaGraphLaunch(c->step_exec, st));
    ++c->host_step;
  }
  const int rc = read_status(c);
  if (sep) CG_CUDA(c, cudaStreamSynchronize(c->h2d));
  CG_CUDA(c, cudaStreamSynchronize(c->d2h));
  return rc;
}

int cg_profile_step(cg_ctx* c, int64_t nsteps, double* ms_out, int32_t n_out) {
  if (!c || !ms_out || n_out < CG_NUM_PHASES || nsteps < 0) return CG_EINVAL;
  cudaStream_t st = c->stream;
  cudaEvent_t ev[CG_NUM_PHASES + 1];
  for (int k = 0; k <= CG_NUM_PHASES; ++k) CG_CUDA(c, cudaEventCreate(&ev[k]));
  for (int k = 0; k < CG_NUM_PHASES; ++k) ms_out[k] = 0.0;
  const int cap = c->par.repair_cap > 0 ? c->par.repair_cap : 4;
  const int grid = repair_grid(c);
  int rc = CG_OK;
  // the order of the graph step: the pending move becomes current, then the
  // test, cell list, rounds, director terms, geometry, and the next move
  static const int kPhaseOfInterval[CG_NUM_PHASES] = {2, 3, 4, 5, 6, 0, 1};
  for (int64_t s = 0; s < nsteps && !rc; ++s) {
    cudaEventRecord(ev[0], st);
    launch_begin_topology(c->ctl(), 1, st);
    launch_test(test_args(c), st);
    cudaEventRecord(ev[1], st);
    launch_cell_list(cell_list_args(c, 1), st);
    cudaEventRecord(ev[2], st);
    for (int r = 0; r < cap; ++r) {
      launch_repair(repair_args(c, r & 1, 0), grid, st);
      launch_check(check_args(c, r & 1, r == cap - 1, 0), check_grid(c), st);
    }
    cudaEventRecord(ev[3], st);
    run_dir(c, dir_args_step(c), st, dir_grid(c));
    cudaEventRecord(ev[4], st);
    if (c->launch.ring_order) run_order(c, st);
    cudaEventRecord(ev[5], st);
    run_geom(c, geom_args(c), st);
    cudaEventRecord(ev[6], st);
    run_force(c, force_args(c, 1), st);
    cudaEventRecord(ev[7], st);
    if (cudaEventSynchronize(ev[7]) != cudaSuccess) { rc = fail(c, CG_ECUDA, "profile sync"); break; }
    for (int k = 0; k < CG_NUM_PHASES; ++k) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
      ms_out[kPhaseOfInterval[k]] += ms;
    }
  }
  for (int k = 0; k <= CG_NUM_PHASES; ++k) cudaEventDestroy(ev[k]);
  if (rc) return rc;
  return read_status(c);
}

int cg_sync(cg_ctx* c) {
  if (!c) return CG_EINVAL;
  return read_status(c);
}

int cg_get_state(cg_ctx* c, double* x, double* y, double* theta) {
  if (!c) return CG_EINVAL;
  int rc = read_status(c);
  if (rc) return rc;
  Ctl h;
  CG_CUDA(c, cudaMemcpy(&h, c->ctl(), sizeof(Ctl), cudaMemcpyDeviceToHost));
  const size_t cur = (size_t)h.cur;
  cudaStream_t st = c->stream;
  const int* tag = c->at<int>(c->off.tag);
  double* tmp = c->at<double>(c->off.tmp);
  const double* srcs[3] = {c->at<double>(c->off.x) + cur * c->N, c->at<double>(c->off.y) + cur * c->N,
                           c->at<double>(c->off.theta)};
  double* dsts[3] = {x, y, theta};
  for (int k = 0; k < 3; ++k) {
    if (!dsts[k]) continue;
    launch_gather_d((int)c->N, tag, srcs[k], tmp, st);
    CG_CUDA(c, cudaMemcpyAsync(dsts[k], tmp, c->N * sizeof(double), cudaMemcpyDefault, st));
    CG_CUDA(c, cudaStreamSynchronize(st));
  }
  return read_status(c);
}

int cg_set_state(cg_ctx* c, const double* x, const double* y, const double* theta) {
  if (!c || !x || !y) return CG_EINVAL;
  int rc = read_status(c);
  if (rc) return rc;
  if (theta) {
    CG_CUDA(c, cudaMemcpyAsync(c->at<double>(c->off.tmp), theta, c->N * sizeof(double), cudaMemcpyDefault,
                               c->stream));
    launch_scatter_d((int)c->N, c->at<int>(c->off.tag), c->at<double>(c->off.tmp), c->at<double>(c->off.theta),
                     c->stream);
    launch_check_finite((int)c->N, c->at<double>(c->off.theta), c->ctl(), c->stream);
  }
  rc = load_positions(c, x, y);
  if (rc) return rc;
  rc = triangulate_all(c);
  if (rc) return rc;
  prime(c);
  return read_status(c);
}

static int compute_forces(cg_ctx* c, int want_energy) {
  GeomArgs g = geom_args(c);
  if (want_energy) g.energy_out = c->at<double>(c->off.ecell);
  run_geom(c, g, c->stream);
  run_force(c, force_args(c, 0), c->stream);
  if (want_energy) launch_reduce_sum((int)c->N, c->at<double>(c->off.ecell), c->at<double>(c->off.scalar), c->stream);
  CG_CUDA(c, cudaGetLastError());
  return CG_OK;
}

static int gather_out(cg_ctx* c, const double* src, double* dst) {
  if (!dst) return CG_OK;
  double* tmp = c->at<double>(c->off.tmp);
  launch_gather_d((int)c->N, c->at<int>(c->off.tag), src, tmp, c->stream);
  CG_CUDA(c, cudaMemcpyAsync(dst, tmp, c->N * sizeof(double), cudaMemcpyDefault, c->stream));
  CG_CUDA(c, cudaStreamSynchronize(c->stream));
  return CG_OK;
}

int cg_get_geometry(cg_ctx* c, double* A, double* P) {
  if (!c) return CG_EINVAL;
  int rc = compute_forces(c, 0);
  if (!rc) rc = gather_out(c, c->at<double>(c->off.A), A);
  if (!rc) rc = gather_out(c, c->at<double>(c->off.P), P);
  if (rc) return rc;
  return read_status(c);
}

int cg_get_forces(cg_ctx* c, double* Fx, double* Fy, double* energy) {
  if (!c) return CG_EINVAL;
  int rc = compute_forces(c, energy != nullptr);
  if (!rc) rc = gather_out(c, c->at<double>(c->off.Fx), Fx);
  if (!rc) rc = gather_out(c, c->at<double>(c->off.Fy), Fy);
  if (rc) return rc;
  if (energy) {
    CG_CUDA(c, cudaMemcpyAsync(energy, c->at<double>(c->off.scalar), sizeof(double), cudaMemcpyDeviceToHost,
                               c->stream));
  }
  return read_status(c);
}

int cg_get_neighbors(cg_ctx* c, int32_t* cnt, int32_t* nbr) {
  if (!c || !cnt || !nbr) return CG_EINVAL;
  int rc = read_status(c);
  if (rc) return rc;
  // stage in the old-ring scratch (free outside a step)
  int* tc = c->at<int>(c->off.cell_bin);
  int* tn = c->at<int>(c->off.old_nbr);
  launch_gather_ring((int)c->N, c->at<int>(c->off.tag), c->at<int>(c->off.cnt), c->at<int>(c->off.nbr), tc, tn,
                     c->stream);
  CG_CUDA(c, cudaMemcpyAsync(cnt, tc, c->N * sizeof(int), cudaMemcpyDefault, c->stream));
  CG_CUDA(c, cudaMemcpyAsync(nbr, tn, c->N * CG_RING * sizeof(int), cudaMemcpyDefault, c->stream));
  return read_status(c);
}

static int set_percell(cg_ctx* c, const double* src, size_t off) {
  if (!c || !src) return CG_EINVAL;
  double* tmp = c->at<double>(c->off.tmp);
  CG_CUDA(c, cudaMemcpyAsync(tmp, src, c->N * sizeof(double), cudaMemcpyDefault, c->stream));
  launch_scatter_d((int)c->N, c->at<int>(c->off.tag), tmp, c->at<double>(off), c->stream);
  launch_check_finite((int)c->N, c->at<double>(off), c->ctl(), c->stream);
  CG_CUDA(c, cudaStreamSynchronize(c->stream));
  return read_status(c);
}

int cg_set_p0(cg_ctx* c, const double* p0) {
  if (!c) return CG_EINVAL;
  int rc = set_percell(c, p0, c->off.p0);
  if (rc) return rc;
  prime(c, kPrimeGeom | kPrimeMove);  // the force sets and the pending move depend on p0
  return read_status(c);
}
int cg_set_v0(cg_ctx* c, const double* v0) {
  if (!c) return CG_EINVAL;
  int rc = set_percell(c, v0, c->off.v0);
  if (rc) return rc;
  // only the pending move depends on v0; the forces of the current
  // positions are stored, so the move is redone from them
  run_force(c, force_args(c, 2), c->stream);
  return read_status(c);
}

int cg_get_counters(cg_ctx* c, cg_counters* out) {
  if (!c || !out) return CG_EINVAL;
  CG_CUDA(c, cudaStreamSynchronize(c->stream));
  Ctl h;
  CG_CUDA(c, cudaMemcpy(&h, c->ctl(), sizeof(Ctl), cudaMemcpyDeviceToHost));
  out->steps = h.step;
  out->flagged_total = h.flagged_total;
  out->repaired_total = h.repaired_total;
  out->last_flagged = h.last_flagged;
  out->last_rounds = h.round_count;
  out->status = h.status;
  out->reserved = 0;
  out->loop_total = h.loop_total;
  return CG_OK;
}


int cg_director_terms(cg_ctx* c, int32_t n, const double* theta, const int32_t* tag, int64_t step, double* cs,
                      double* sn, double* xi) {
  if (!c || n < 0) return CG_EINVAL;
  if (n == 0) return CG_OK;
  if (!theta || !tag || !cs || !sn || !xi) return CG_EINVAL;
  launch_dir_terms(n, theta, tag, c->par.seed, step, c->at<double2>(c->off.dir_tab), cs, sn, xi, c->stream);
  CG_CUDA(c, cudaGetLastError());
  return CG_OK;
}


int cg_backward_bytes(const cg_ctx* c, int64_t nsteps, int32_t ckpt_every, size_t* bytes) {
  if (!c || nsteps < 1 || ckpt_every < 1 || !bytes) return CG_EINVAL;
  *bytes = bwd_layout(c->N, nsteps, ckpt_every).total;
  return CG_OK;
}

int cg_set_moduli(cg_ctx* c, double KA, double KP) {
  if (!c || !std::isfinite(KA) || !std::isfinite(KP)) return CG_EINVAL;
  int rc = read_status(c);
  if (rc) return rc;
  c->par.KA = KA;
  c->par.KP = KP;
  if (c->step_exec) {  // kernel parameters are baked into the graph: capture again
    cudaGraphExecDestroy(c->step_exec);
    c->step_exec = nullptr;
  }
  rc = build_graph(c);
  if (rc) return rc;
  prime(c, kPrimeGeom | kPrimeMove);  // the force sets and the pending move depend on the moduli
  return read_status(c);
}

int cg_get_launch(const cg_ctx* c, cg_launch* out) {
  if (!c || !out) return CG_EINVAL;
  *out = c->launch;
  return CG_OK;
}

int cg_set_launch(cg_ctx* c, const cg_launch* l) {
  if (!c || !l) return CG_EINVAL;
  if (l->repair_blocks_per_sm < 1 || l->repair_blocks_per_sm > 64 || l->check_blocks_per_sm < 1 ||
      l->check_blocks_per_sm > 64 || l->dir_blocks_per_sm < 0 || l->dir_blocks_per_sm > 64 ||
      (l->dir_low_priority != 0 && l->dir_low_priority != 1) || l->geom_blocks_per_sm < 0 ||
      l->geom_blocks_per_sm > 64 || l->test_blocks_per_sm < 0 || l->test_blocks_per_sm > 64 ||
      (l->dir_beside_geom != 0 && l->dir_beside_geom != 1) || l->ring_order < 0 || l->ring_order > 7 ||
      (l->force_beside != 0 && l->force_beside != 1))
    return CG_EINVAL;
  int rc = read_status(c);
  if (rc) return rc;
  c->launch = *l;
  if (c->step_exec) {
    cudaGraphExecDestroy(c->step_exec);
    c->step_exec = nullptr;
  }
  return build_graph(c);
}

int cg_autotune_bytes(const cg_ctx* c, size_t flush_bytes, size_t* bytes) {
  if (!c || !bytes) return CG_EINVAL;
  *bytes = c->off.total + ((5 * (size_t)c->N * sizeof(double) + 255) & ~(size_t)255) + flush_bytes;
  return CG_OK;
}

int cg_autotune(cg_ctx* c, int32_t steps_per_trial, size_t flush_bytes, void* d_ws2, size_t ws2_bytes,
                cg_launch* best, double* best_ms) {
  if (!c || steps_per_trial < 1 || !d_ws2 || ((uintptr_t)d_ws2 & 255)) return CG_EINVAL;
  size_t need = 0;
  cg_autotune_bytes(c, flush_bytes, &need);
  if (ws2_bytes < need) return CG_EINVAL;
  int rc = read_status(c);
  if (rc) return rc;
  // the current state in user order, after the temporary workspace
  char* base = static_cast<char*>(d_ws2);
  double* sx = reinterpret_cast<double*>(base + c->off.total);
  double* sy = sx + c->N;
  double* sth = sy + c->N;
  double* sp0 = sth + c->N;
  double* sv0 = sp0 + c->N;
  char* flush = base + c->off.total + ((5 * (size_t)c->N * sizeof(double) + 255) & ~(size_t)255);
  if ((rc = cg_get_state(c, sx, sy, sth))) return rc;
  const int* tag = c->at<int>(c->off.tag);
  launch_gather_d((int)c->N, tag, c->at<double>(c->off.p0), sp0, c->stream);
  launch_gather_d((int)c->N, tag, c->at<double>(c->off.v0), sv0, c->stream);
  Ctl h;
  CG_CUDA(c, cudaStreamSynchronize(c->stream));
  CG_CUDA(c, cudaMemcpy(&h, c->ctl(), sizeof(Ctl), cudaMemcpyDeviceToHost));
  cg_ctx* t = nullptr;
  rc = cg_create(c->R, c->user_reps.data(), &c->par, sx, sy, sth, d_ws2, c->off.total, c->stream, &t);
  if (rc) return fail(c, rc, "autotune: temporary context: " + (t ? t->last_error : std::string("create failed")));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto trial = [&](const cg_launch& l, int steps, double& ms) -> int {
    int r = cg_set_launch(t, &l);
    if (!r) r = cg_set_state(t, sx, sy, sth);
    if (!r) r = cg_set_p0(t, sp0);
    if (!r) r = cg_set_v0(t, sv0);
    if (!r) r = cg_set_step(t, h.step);
    if (!r) r = cg_step(t, 2);
    if (r) return r;
    float total = 0.f;
    if (flush_bytes == 0) {
      cudaEventRecord(e0, t->stream);
      r = cg_step(t, steps);
      cudaEventRecord(e1, t->stream);
      if (!r) r = read_status(t);
      cudaEventElapsedTime(&total, e0, e1);
    } else {
      for (int k = 0; k < steps && !r; ++k) {
        cudaMemsetAsync(flush, k & 0xff, flush_bytes, t->stream);  // evicts the L2
        cudaEventRecord(e0, t->stream);
        r = cg_step(t, 1);
        cudaEventRecord(e1, t->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) r = fail(c, CG_ECUDA, "autotune sync");
        float f = 0.f;
        cudaEventElapsedTime(&f, e0, e1);
        total += f;
      }
      if (!r) r = read_status(t);
    }
    ms = total / steps;
    return r;
  };
  static const int repair_opts[] = {2, 4, 8, 16};
  static const int check_opts[] = {1, 2, 4, 8};
  static const int dir_opts[] = {0, 1, 2, 4, 8};
  static const int prio_opts[] = {0, 1};
  static const int geom_opts[] = {0, 4, 8, 16};
  static const int test_opts[] = {0, 2, 4, 8};
  static const int beside_opts[] = {0, 1};
  static const int order_opts[] = {0, 1, 4, 5};
  static const int fb_opts[] = {0, 1};
  const cg_launch start = c->launch;
  cg_launch cur = start;
  double cur_ms = 0.0;
  rc = trial(cur, steps_per_trial, cur_ms);
  struct Field {
    int32_t cg_launch::*member;
    const int* opts;
    int nopt;
  };
  const Field fields[] = {
      {&cg_launch::repair_blocks_per_sm, repair_opts, 4}, {&cg_launch::check_blocks_per_sm, check_opts, 4},
      {&cg_launch::dir_blocks_per_sm, dir_opts, 5},       {&cg_launch::dir_low_priority, prio_opts, 2},
      {&cg_launch::geom_blocks_per_sm, geom_opts, 4},     {&cg_launch::test_blocks_per_sm, test_opts, 4},
      {&cg_launch::dir_beside_geom, beside_opts, 2},      {&cg_launch::ring_order, order_opts, 4},
      {&cg_launch::force_beside, fb_opts, 2}};
  for (int sweep = 0; sweep < 2 && !rc; ++sweep) {
    for (const Field& f : fields) {
      for (int k = 0; k < f.nopt && !rc; ++k) {
        cg_launch cand = cur;
        if (cand.*f.member == f.opts[k]) continue;
        cand.*f.member = f.opts[k];
        double ms = 0.0;
        rc = trial(cand, steps_per_trial, ms);
        if (!rc && ms < cur_ms) {
          cur = cand;
          cur_ms = ms;
        }
      }
      if (rc) break;
    }
  }

  // short trials are noisy: the winner must beat the starting shapes again in
  // two longer, interleaved trials each (best of two)
  if (!rc && std::memcmp(&cur, &start, sizeof(cg_launch)) != 0) {
    double best_cur = 1e30, best_start = 1e30;
    for (int rep = 0; rep < 2 && !rc; ++rep) {
      double ms = 0.0;
      rc = trial(start, 3 * steps_per_trial, ms);
      if (!rc) best_start = std::min(best_start, ms);
      if (!rc) rc = trial(cur, 3 * steps_per_trial, ms);
      if (!rc) best_cur = std::min(best_cur, ms);
    }
    if (!rc) {
      if (best_start <= best_cur) {
        cur = start;
        cur_ms = best_start;
      } else {
        cur_ms = best_cur;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::string terr = rc ? t->last_error : std::string();
  cg_destroy(t);
  if (rc) return fail(c, rc, "autotune trial: " + terr);
  rc = cg_set_launch(c, &cur);
  if (rc) return rc;
  if (best) *best = cur;
  if (best_ms) *best_ms = cur_ms;
  return CG_OK;
}

// ---------------------------------------------------------------------------
// Domain decomposition of one large system (strips with halos): the pieces a
// domain's context needs so that its cells evolve exactly as in the
// undivided system.
// ---------------------------------------------------------------------------
int cg_set_noise_ids(cg_ctx* c, const int32_t* ids) {
  if (!c || !ids) return CG_EINVAL;
  int rc = read_status(c);
  if (rc) return rc;
  std::vector<int32_t> h(c->N);
  CG_CUDA(c, cudaMemcpy(h.data(), ids, c->N * sizeof(int32_t), cudaMemcpyDefault));
  for (int32_t v : h)
    if (v < 0) return fail(c, CG_EINVAL, "noise ids must be non-negative");
  int* tmp = c->at<int>(c->off.tmp);  // staging (user order)
  CG_CUDA(c, cudaMemcpyAsync(tmp, h.data(), c->N * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
  launch_scatter_i((int)c->N, c->at<int>(c->off.tag), tmp, c->at<int>(c->off.nid), c->stream);
  CG_CUDA(c, cudaStreamSynchronize(c->stream));
  prime(c, kPrimeDir | kPrimeMove);  // the noise of the pending move depends on the ids
  return read_status(c);
}

int cg_set_frame(cg_ctx* c, int32_t replica, double x0, double y0, double Lx_outer, double Ly_outer) {
  if (!c || replica < 0 || replica >= c->R) return CG_EINVAL;
  Rep& R = c->reps[replica];
  if (!(Lx_outer > 0) || !(Ly_outer > 0) || !std::isfinite(Lx_outer) || !std::isfinite(Ly_outer))
    return fail(c, CG_EINVAL, "cg_set_frame: the outer box needs positive finite sides");
  if (ceil_log2(std::fmax(Lx_outer, Ly_outer)) != 50 - R.q)
    return fail(c, CG_EINVAL, "cg_set_frame: the outer box must have the same position grid (same ceil(log2(max side)))");
  const long long LXg = (long long)std::rint(std::ldexp(Lx_outer, R.q));
  const long long LYg = (long long)std::rint(std::ldexp(Ly_outer, R.q));
  const double X0d = std::ldexp(x0, R.q), Y0d = std::ldexp(y0, R.q);
  if (!(X0d >= 0 && X0d < (double)LXg && Y0d >= 0 && Y0d < (double)LYg) || X0d != std::rint(X0d) ||
      Y0d != std::rint(Y0d))
    return fail(c, CG_EINVAL, "cg_set_frame: the origin must be a grid point inside the outer box");
  if (R.LX > LXg || R.LY > LYg) return fail(c, CG_EINVAL, "cg_set_frame: the frame must fit in the outer box");
  int rc = read_status(c);
  if (rc) return rc;
  R.framed = 1;
  R.X0 = (long long)X0d;
  R.Y0 = (long long)Y0d;
  R.LXg = LXg;
  R.LYg = LYg;
  R.x0 = std::ldexp((double)R.X0, -R.q);
  R.y0 = std::ldexp((double)R.Y0, -R.q);
  R.Lxg = std::ldexp((double)LXg, -R.q);
  R.Lyg = std::ldexp((double)LYg, -R.q);
  CG_CUDA(c, cudaMemcpyAsync(c->at<Rep>(c->off.reps) + replica, &R, sizeof(Rep), cudaMemcpyHostToDevice, c->stream));
  CG_CUDA(c, cudaStreamSynchronize(c->stream));
  prime(c, kPrimeMove);  // the pending move is rounded in the outer box's coordinates
  return read_status(c);
}

int cg_halo_pack(cg_ctx* c, const int32_t* d_slot, int64_t* d_out) {
  if (!c || !d_slot || !d_out) return CG_EINVAL;
  launch_halo_pack((int)c->N, c->at<int>(c->off.tag), d_slot, c->at<Rep>(c->off.reps), c->at<int>(c->off.rep),
                   c->ctl(), c->at<long long>(c->off.X), c->at<long long>(c->off.Y),
                   reinterpret_cast<long long*>(d_out), c->stream);
  CG_CUDA(c, cudaGetLastError());
  return CG_OK;
}

int cg_halo_unpack(cg_ctx* c, const int32_t* d_slot, const int64_t* d_in) {
  if (!c || !d_slot || !d_in) return CG_EINVAL;
  launch_halo_unpack((int)c->N, c->at<int>(c->off.tag), d_slot, c->at<Rep>(c->off.reps), c->at<int>(c->off.rep),
                     c->ctl(), reinterpret_cast<const long long*>(d_in), c->at<double>(c->off.x),
                     c->at<double>(c->off.y), c->at<long long>(c->off.X), c->at<long long>(c->off.Y), c->stream);
  CG_CUDA(c, cudaGetLastError());
  return CG_OK;
}

int cg_set_step(cg_ctx* c, int64_t step) {
  if (!c || step < 0) return CG_EINVAL;
  int rc = read_status(c);
  if (rc) return rc;
  Ctl h;
  CG_CUDA(c, cudaMemcpy(&h, c->ctl(), sizeof(Ctl), cudaMemcpyDeviceToHost));
  h.step = step;
  CG_CUDA(c, cudaMemcpy(c->ctl(), &h, sizeof(Ctl), cudaMemcpyHostToDevice));
  prime(c, kPrimeDir | kPrimeMove);  // the noise of the pending move depends on the step counter
  return read_status(c);
}

int cg_run_checkpointed(cg_ctx* c, int64_t nsteps, int32_t ckpt_every, void* d_bw, size_t bytes) {
  BwdLayout b;
  int rc = check_bwd(c, nsteps, ckpt_every, d_bw, bytes, b);
  if (rc) return rc;
  rc = read_status(c);
  if (rc) return rc;
  char* bw = static_cast<char*>(d_bw);
  const int64_t nck = (nsteps + ckpt_every - 1) / ckpt_every;
  for (int64_t t = 0; t < nsteps; ++t) {
    if (t % ckpt_every == 0) snapshot(c, 1, snapshot_at(bw + b.snaps + (t / ckpt_every) * b.snap_bytes, c->N));
    CG_CUDA(c, cudaGraphLaunch(c->step_exec, c->stream));
  }
  snapshot(c, 1, snapshot_at(bw + b.snaps + nck * b.snap_bytes, c->N));
  CG_CUDA(c, cudaGetLastError());
  return read_status(c);
}

int cg_backward(cg_ctx* c, int64_t nsteps, int32_t ckpt_every, void* d_bw, size_t bytes, const double* gxT,
                const double* gyT, const double* gAT, const double* gPT, double* gx0, double* gy0, double* gp0,
                double* gv0, double* h_gK) {
  BwdLayout b;
  int rc = check_bwd(c, nsteps, ckpt_every, d_bw, bytes, b);
  if (rc) return rc;
  if (!gxT || !gyT || !gAT || !gPT) return CG_EINVAL;
  rc = read_status(c);
  if (rc) return rc;
  char* bw = static_cast<char*>(d_bw);
  cudaStream_t st = c->stream;
  const int n = (int)c->N;
  const int* tag = c->at<int>(c->off.tag);
  const int64_t nck = (nsteps + ckpt_every - 1) / ckpt_every;
  const Snapshot fin = snapshot_at(bw + b.snaps + nck * b.snap_bytes, c->N);
  snapshot(c, 0, fin, 0);  // the tangent kernels compute their own geometry
  // cotangents of the final state, in storage order
  double* tmp = c->at<double>(c->off.tmp);
  const double* srcs[4] = {gxT, gyT, gAT, gPT};
  double* dsts[4] = {reinterpret_cast<double*>(bw + b.gx), reinterpret_cast<double*>(bw + b.gy),
                     reinterpret_cast<double*>(bw + b.cA), reinterpret_cast<double*>(bw + b.cP)};
  for (int k = 0; k < 4; ++k) {
    CG_CUDA(c, cudaMemcpyAsync(tmp, srcs[k], c->N * sizeof(double), cudaMemcpyDefault, st));
    launch_scatter_d(n, tag, tmp, dsts[k], st);
  }
  JvpArgs a = jvp_args(c, bw, b);
  CG_CUDA(c, cudaMemsetAsync(a.v, 0, c->N * sizeof(double2), st));
  {
    JvpArgs f = a;
    f.coefA = dsts[2];
    f.coefP = dsts[3];
    f.F = reinterpret_cast<double2*>(bw + b.F);
    launch_geom_jvp(f, st);
    launch_force_jvp(f, st);
    launch_combine_final(n, dsts[0], dsts[1], f.F, a.v, st);
  }
  for (size_t off : {b.gp0, b.gv0, b.gKA, b.gKP}) CG_CUDA(c, cudaMemsetAsync(bw + off, 0, c->N * sizeof(double), st));
  a.gp0 = reinterpret_cast<double*>(bw + b.gp0);
  a.gv0 = reinterpret_cast<double*>(bw + b.gv0);
  a.gKA = reinterpret_cast<double*>(bw + b.gKA);
  a.gKP = reinterpret_cast<double*>(bw + b.gKP);
  a.update = 1;
  for (int64_t ck = nck - 1; ck >= 0; --ck) {
    const int64_t t0 = ck * ckpt_every, t1 = std::min<int64_t>(t0 + ckpt_every, nsteps);
    snapshot(c, 0, snapshot_at(bw + b.snaps + ck * b.snap_bytes, c->N));
    for (int64_t t = t0; t < t1; ++t) {  // recompute the segment, keeping every step's input state
      snapshot(c, 1, snapshot_at(bw + b.seg + (t - t0) * b.snap_bytes, c->N));
      if (t + 1 < t1) CG_CUDA(c, cudaGraphLaunch(c->step_exec, st));
    }
    for (int64_t t = t1 - 1; t >= t0; --t) {  // the tangent kernels compute their own geometry
      snapshot(c, 0, snapshot_at(bw + b.seg + (t - t0) * b.snap_bytes, c->N), 0);
      launch_geom_jvp(a, st);
      launch_force_jvp(a, st);
    }
  }
  snapshot(c, 0, fin);  // leave the context in the final state
  // results in user order
  double2* v = a.v;
  double* vx = reinterpret_cast<double*>(bw + b.gx);
  double* vy = reinterpret_cast<double*>(bw + b.gy);
  CG_CUDA(c, cudaMemcpy2DAsync(vx, sizeof(double), v, sizeof(double2), sizeof(double), c->N, cudaMemcpyDeviceToDevice, st));
  CG_CUDA(c, cudaMemcpy2DAsync(vy, sizeof(double), reinterpret_cast<double*>(v) + 1, sizeof(double2), sizeof(double), c->N,
                               cudaMemcpyDeviceToDevice, st));
  const double* outs_src[4] = {vx, vy, a.gp0, a.gv0};
  double* outs_dst[4] = {gx0, gy0, gp0, gv0};
  for (int k = 0; k < 4; ++k) {
    if (!outs_dst[k]) continue;
    launch_gather_d(n, tag, outs_src[k], tmp, st);
    CG_CUDA(c, cudaMemcpyAsync(outs_dst[k], tmp, c->N * sizeof(double), cudaMemcpyDefault, st));
  }
  if (h_gK) {
    double* red = reinterpret_cast<double*>(bw + b.red);
    launch_reduce2(n, a.gKA, a.gKP, red, st);
    CG_CUDA(c, cudaMemcpyAsync(h_gK, red, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  CG_CUDA(c, cudaGetLastError());
  return read_status(c);
}

int cg_hvp(cg_ctx* c, const double* vx, const double* vy, double* hvx, double* hvy, double* Adot, double* Pdot,
           void* d_bw, size_t bytes) {
  BwdLayout b;
  int rc = check_bwd(c, 1, 1, d_bw, bytes, b);
  if (rc) return rc;
  if (!vx || !vy) return CG_EINVAL;
  rc = read_status(c);
  if (rc) return rc;
  char* bw = static_cast<char*>(d_bw);
  cudaStream_t st = c->stream;
  const int n = (int)c->N;
  const int* tag = c->at<int>(c->off.tag);
  double* tmp = c->at<double>(c->off.tmp);
  double* sx = reinterpret_cast<double*>(bw + b.gx);
  double* sy = reinterpret_cast<double*>(bw + b.gy);
  CG_CUDA(c, cudaMemcpyAsync(tmp, vx, c->N * sizeof(double), cudaMemcpyDefault, st));
  launch_scatter_d(n, tag, tmp, sx, st);
  CG_CUDA(c, cudaMemcpyAsync(tmp, vy, c->N * sizeof(double), cudaMemcpyDefault, st));
  launch_scatter_d(n, tag, tmp, sy, st);
  JvpArgs a = jvp_args(c, bw, b);
  CG_CUDA(c, cudaMemcpy2DAsync(a.v, sizeof(double2), sx, sizeof(double), sizeof(double), c->N, cudaMemcpyDeviceToDevice, st));
  CG_CUDA(c, cudaMemcpy2DAsync(reinterpret_cast<double*>(a.v) + 1, sizeof(double2), sy, sizeof(double), sizeof(double), c->N,
                               cudaMemcpyDeviceToDevice, st));
  double* Ad = reinterpret_cast<double*>(bw + b.gKA);
  double* Pd = reinterpret_cast<double*>(bw + b.gKP);
  a.Adot = Ad;
  a.Pdot = Pd;
  a.Hv = reinterpret_cast<double2*>(bw + b.F);
  launch_geom_jvp(a, st);
  launch_force_jvp(a, st);
  CG_CUDA(c, cudaMemcpy2DAsync(sx, sizeof(double), a.Hv, sizeof(double2), sizeof(double), c->N, cudaMemcpyDeviceToDevice, st));
  CG_CUDA(c, cudaMemcpy2DAsync(sy, sizeof(double), reinterpret_cast<double*>(a.Hv) + 1, sizeof(double2), sizeof(double), c->N,
                               cudaMemcpyDeviceToDevice, st));
  const double* srcs[4] = {sx, sy, Ad, Pd};
  double* dsts[4] = {hvx, hvy, Adot, Pdot};
  for (int k = 0; k < 4; ++k) {
    if (!dsts[k]) continue;
    launch_gather_d(n, tag, srcs[k], tmp, st);
    CG_CUDA(c, cudaMemcpyAsync(dsts[k], tmp, c->N * sizeof(double), cudaMemcpyDefault, st));
  }
  CG_CUDA(c, cudaGetLastError());
  return read_status(c);
}

int64_t cg_num_cells(const cg_ctx* c) { return c ? c->N : -1; }

int cg_destroy(cg_ctx* c) {
  if (!c) return CG_EINVAL;
  if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
  if (c->capture) cudaStreamDestroy(c->capture);
  for (cudaStream_t sd : c->side)
    if (sd) cudaStreamDestroy(sd);
  for (cudaEvent_t ev : {c->fork, c->join_dir, c->join_list, c->join_terms})
    if (ev) cudaEventDestroy(ev);
  for (cudaStream_t sc : {c->h2d, c->d2h})
    if (sc) cudaStreamDestroy(sc);
  for (int b = 0; b < 2; ++b)
    for (cudaEvent_t ev : {c->in_ready[b], c->in_free[b], c->out_ready[b], c->out_free[b]})
      if (ev) cudaEventDestroy(ev);
  delete c;
  return CG_OK;
}

const char* cg_status_string(int s) {
  switch (s) {
    case CG_OK: return "ok";
    case CG_EINVAL: return "invalid argument";
    case CG_ECUDA: return "CUDA runtime error";
    case CG_ERING_OVERFLOW: return "ring overflow (more than 16 neighbours)";
    case CG_EREPAIR_CAP: return "topology inconsistent after the repair cap";
    case CG_ETOPO_INCONSISTENT: return "inconsistent neighbour rings";
    case CG_ENONFINITE: return "non-finite position";
    case CG_EBOX_TOO_SMALL: return "box too small for the Voronoi search";
    case CG_EDEGENERATE: return "degenerate input (coincident cells)";
    case CG_ECANDIDATES: return "too many repair candidates";
    case CG_ET1_CAP: return "T1 candidates left after the pass cap";
    default: return "unknown status";
  }
}

const char* cg_last_error(const cg_ctx* c) { return c ? c->last_error.c_str() : "null context"; }

}  // extern "C"
