// C ABI of the active vertex model (AVM) mode of libcellgb.so.
#include "../../include/cellgb.h"
#include "cg_device.cuh"
#include "cg_kernels.h"
#include "cg_graph.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

using namespace cgk;

namespace {

struct Lay {
  size_t total = 0;
  size_t take(size_t b) {
    size_t o = total;
    total += (b + 255) & ~(size_t)255;
    return o;
  }
};

struct AvmOff {
  size_t spv, spv_bytes;
  size_t hx, hy, hf, vc, vn, cc, cv, theta, thn, p0, v0, a0, P0, A, P, ka, kp, energy, act, Fx, Fy, lock, cand_e, cand,
      done;
  size_t owned, base_local, base_partial, xs, ys, cnt, nbr, scalar, ctl, dir_tab;
  size_t div_cells, div_dirs, div_made, div_cslots, div_vslots, div_lock;  // staging of cg_avm_divide
  size_t div_flag, div_ctl;                                                // its rounds
  // storage order: tags of the slots, slots of the tags, candidate priorities
  size_t vtag, ctag, vslot, cslot, cand_k;
  size_t cand_v, cand_w;  // a T1 candidate's other end and outer neighbours
  // re-sort scratch (keys, ranks, new places, key counts, permuted copies);
  // between re-sorts the copies stage the API's tag-ordered transfers
  size_t vkey, vrank, vperm, ckey, crank, cperm, kcount_v, kstart_v, kpart_v, kcount_c, kstart_c, kpart_c;
  size_t vc_s, vn_s, cc_s, cv_s, vtag_s, ctag_s, theta_s, p0_s, v0_s, a0_s, P0_s;
  size_t total;
};

AvmOff avm_layout(int64_t n, size_t spv_bytes) {
  Lay L;
  AvmOff o;
  const int64_t V = 2 * n;
  const size_t d = sizeof(double), i4 = sizeof(int);
  o.spv_bytes = spv_bytes;
  o.spv = L.take(spv_bytes);
  o.hx = L.take(2 * V * d);
  o.hy = L.take(2 * V * d);
  o.hf = L.take(V * sizeof(float2));
  o.vc = L.take(3 * V * i4);
  o.vn = L.take(3 * V * i4);
  o.cc = L.take(n * i4);
  o.cv = L.take(n * CG_RING * i4);
  o.theta = L.take(n * d);
  o.thn = L.take(n * d);
  o.p0 = L.take(n * d);
  o.v0 = L.take(n * d);
  o.a0 = L.take(n * d);
  o.P0 = L.take(n * d);
  o.A = L.take(n * d);
  o.P = L.take(n * d);
  o.ka = L.take(n * d);
  o.kp = L.take(n * d);
  o.energy = L.take(n * d);
  o.act = L.take(n * 2 * d);
  o.Fx = L.take(V * d);
  o.Fy = L.take(V * d);
  o.lock = L.take(n * sizeof(unsigned long long));
  o.cand_e = L.take((3 * V / 2 + n + 1) * i4);  // at most one entry per edge and per cell
  o.cand = L.take((3 * V / 2 + n + 1) * sizeof(int4));
  o.done = L.take(2 * sizeof(unsigned int));
  o.owned = L.take(n * i4);
  o.base_local = L.take((n + 1) * i4);
  o.base_partial = L.take(((n + 1 + kScanChunk - 1) / kScanChunk + 1) * i4);
  o.xs = L.take(n * d);
  o.ys = L.take(n * d);
  o.cnt = L.take(n * i4);
  o.nbr = L.take(n * CG_RING * i4);
  o.scalar = L.take(4 * d);
  o.ctl = L.take(sizeof(Ctl));
  o.dir_tab = L.take(kDirTabEntries * sizeof(double2));
  o.div_cells = L.take(n * i4);
  o.div_dirs = L.take(2 * n * d);
  o.div_made = L.take(n * i4);
  o.div_cslots = L.take(n * i4);
  o.div_vslots = L.take(2 * n * i4);
  o.div_lock = L.take(n * sizeof(unsigned long long));
  o.div_flag = L.take(kDivWindow * i4);
  o.div_ctl = L.take(sizeof(DivCtl));
  o.vtag = L.take(V * i4);
  o.ctag = L.take(n * i4);
  o.vslot = L.take(V * i4);
  o.cslot = L.take(n * i4);
  o.cand_k = L.take((3 * V / 2 + n + 1) * i4);
  o.cand_v = L.take((3 * V / 2 + n + 1) * sizeof(int4));
  o.cand_w = L.take((3 * V / 2 + n + 1) * i4);
  o.vkey = L.take(V * i4);
  o.vrank = L.take(V * i4);
  o.vperm = L.take(V * i4);
  o.ckey = L.take(n * i4);
  o.crank = L.take(n * i4);
  o.cperm = L.take(n * i4);
  // key counts: at most V + 1 (Hilbert keys <= V plus the last key, or V tags)
  o.kcount_v = L.take((V + 2) * i4);
  o.kstart_v = L.take((V + 2) * i4);
  o.kpart_v = L.take(((V + 2) / kScanChunk + 2) * i4);
  o.kcount_c = L.take((n + 2) * i4);
  o.kstart_c = L.take((n + 2) * i4);
  o.kpart_c = L.take(((n + 2) / kScanChunk + 2) * i4);
  o.vc_s = L.take(3 * V * i4);
  o.vn_s = L.take(3 * V * i4);
  o.cc_s = L.take(n * i4);
  o.cv_s = L.take(n * CG_RING * i4);
  o.vtag_s = L.take(V * i4);
  o.ctag_s = L.take(n * i4);
  o.theta_s = L.take(n * d);
  o.p0_s = L.take(n * d);
  o.v0_s = L.take(n * d);
  o.a0_s = L.take(n * d);
  o.P0_s = L.take(n * d);
  o.total = L.total;
  return o;
}

}  // namespace

struct cg_avm_ctx {
  int n = 0, V = 0;        // cell slots (the capacity) and vertex slots (2n)
  int n_seed = 0;          // cells of the initial network (slots 0 .. n_seed-1)
  double Lx = 0, Ly = 0;
  cg_avm_params par{};
  char* ws = nullptr;
  AvmOff off{};
  cudaStream_t stream = nullptr, capture = nullptr;
  cudaStream_t side = nullptr;                     // the director branch of the step graph
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaGraphExec_t exec = nullptr;     // one step
  cudaGraphExec_t t1_exec = nullptr;  // T1 passes alone
  cudaGraphExec_t div_exec = nullptr;  // the division rounds of cg_avm_divide
  int sms = 0;
  int hord_v = 0, hord_c = 0;  // Hilbert grids of the re-sort
  int since_sort = 0;          // steps since the last re-sort
  bool permuted = false;       // slots differ from tags (a re-sort ran)
  bool broken = false;  // a device status was seen: no further steps
  std::string last_error;
  template <class T>
  T* at(size_t o) const { return reinterpret_cast<T*>(ws + o); }
  Ctl* ctl() const { return at<Ctl>(off.ctl); }
};

namespace {

int afail(cg_avm_ctx* c, int code, const std::string& m) {
  if (c) c->last_error = m;
  return code;
}

#define AV_CUDA(ctx, call)                                                              \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return afail(ctx, CG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

int cap_of(const cg_avm_ctx* c) { return c->par.t1_cap > 0 ? c->par.t1_cap : 16; }

Axis axis(double L) {
  Axis a;
  a.L = L;
  const double h = 0.5 * L;
  std::memcpy(&a.L_bits, &L, sizeof(double));
  std::memcpy(&a.half_bits, &h, sizeof(double));
  return a;
}

// FP32 squared lengths certainly below / above thr^2.  A float copy of a
// position in [0, L) is off by at most L 2^-24, the float difference and its
// periodic correction add 3 L 2^-24 more, so each component of the float edge
// vector is within delta = 5 L 2^-24 of the exact one and its length within
// sqrt(2) delta; the margin doubles that, and the factors (1 +- 2^-20) cover
// the rounding of the float squared length.
void t1_bounds(double thr, double L, float& lo, float& hi) {
  const double m = 2.0 * std::sqrt(2.0) * 5.0 * L * std::ldexp(1.0, -24);
  const double h = (thr + m) * (1.0 + std::ldexp(1.0, -20));
  hi = std::nextafter((float)(h * h), INFINITY);
  if (thr > m) {
    const double l = (thr - m) * (1.0 - std::ldexp(1.0, -20));
    lo = std::nextafter((float)(l * l), 0.0f);
  } else {
    lo = 0.0f;
  }
}

AvmArgs avm_args(cg_avm_ctx* c) {
  AvmArgs a{};  // every field starts zero or null
  a.n = c->n;
  a.V = c->V;
  a.ctl = c->ctl();
  a.Lx = c->Lx;
  a.Ly = c->Ly;
  a.ax = axis(c->Lx);
  a.ay = axis(c->Ly);
  a.Lxf = (float)c->Lx;
  a.Lyf = (float)c->Ly;
  a.hx = c->at<double>(c->off.hx);
  a.hy = c->at<double>(c->off.hy);
  a.vc = c->at<int>(c->off.vc);
  a.vn = c->at<int>(c->off.vn);
  a.cc = c->at<int>(c->off.cc);
  a.cv = c->at<int>(c->off.cv);
  a.theta = c->at<double>(c->off.theta);
  a.p0 = c->at<double>(c->off.p0);
  a.v0 = c->at<double>(c->off.v0);
  a.a0 = c->at<double>(c->off.a0);
  a.P0 = c->at<double>(c->off.P0);
  a.KA = c->par.KA;
  a.KP = c->par.KP;
  a.mu = c->par.mu;
  a.dt = c->par.dt;
  a.noise_amp = std::sqrt(2.0 * c->par.Dr * c->par.dt);
  a.seed = c->par.seed;
  a.tab = c->at<double2>(c->off.dir_tab);
  a.A = c->at<double>(c->off.A);
  a.P = c->at<double>(c->off.P);
  a.ka = c->at<double>(c->off.ka);
  a.kp = c->at<double>(c->off.kp);
  a.energy = nullptr;
  a.act = c->at<double2>(c->off.act);
  a.thn = c->at<double>(c->off.thn);
  a.Fx = c->at<double>(c->off.Fx);
  a.Fy = c->at<double>(c->off.Fy);
  a.move = 1;
  a.thr2 = c->par.t1_threshold * c->par.t1_threshold;
  a.t1_len = c->par.t1_length > 0 ? c->par.t1_length : 1.5 * c->par.t1_threshold;
  a.t2_twice = 2.0 * c->par.t2_area;
  t1_bounds(c->par.t1_threshold, std::fmax(c->Lx, c->Ly), a.t2lo, a.t2hi);
  a.hf = c->at<float2>(c->off.hf);
  a.t1_cap = cap_of(c);
  a.apply_blocks = std::max(1, std::min((c->V + 127) / 128, std::max(c->sms / 2, 1)));
  a.lock = c->at<unsigned long long>(c->off.lock);
  a.cand_e = c->at<int>(c->off.cand_e);
  a.cand = c->at<int4>(c->off.cand);
  a.cand_k = c->at<int>(c->off.cand_k);
  a.cand_v = c->at<int4>(c->off.cand_v);
  a.cand_w = c->at<int>(c->off.cand_w);
  a.vtag = c->at<int>(c->off.vtag);
  a.ctag = c->at<int>(c->off.ctag);
  a.done = c->at<unsigned int>(c->off.done);
  a.loop = 0;
  return a;
}

int avm_status(cg_avm_ctx* c) {
  Ctl h;  // read on the context's stream, after its work
  AV_CUDA(c, cudaMemcpyAsync(&h, c->ctl(), sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
  AV_CUDA(c, cudaStreamSynchronize(c->stream));
  if (h.status) {
    c->broken = true;
    return afail(c, h.status, std::string("device status: ") + cg_status_string(h.status));
  }
  return CG_OK;
}

int copy_in(cg_avm_ctx* c, void* dst, const void* src, size_t bytes) {
  if (!src) return CG_OK;
  AV_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream));
  return CG_OK;
}

int copy_out(cg_avm_ctx* c, void* dst, const void* src, size_t bytes) {
  if (!dst) return CG_OK;
  AV_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream));
  return CG_OK;
}

AvmSortArgs sort_args(cg_avm_ctx* c, int by_tag) {
  AvmSortArgs a{};
  a.n = c->n;
  a.V = c->V;
  a.ctl = c->ctl();
  a.Lx = c->Lx;
  a.Ly = c->Ly;
  a.hord_v = c->hord_v;
  a.hord_c = c->hord_c;
  a.by_tag = by_tag;
  a.hx = a.hx_w = c->at<double>(c->off.hx);
  a.hy = a.hy_w = c->at<double>(c->off.hy);
  a.vc = c->at<int>(c->off.vc);
  a.vn = c->at<int>(c->off.vn);
  a.cc = c->at<int>(c->off.cc);
  a.cv = c->at<int>(c->off.cv);
  a.theta = c->at<double>(c->off.theta);
  a.p0 = c->at<double>(c->off.p0);
  a.v0 = c->at<double>(c->off.v0);
  a.a0 = c->at<double>(c->off.a0);
  a.P0 = c->at<double>(c->off.P0);
  a.vtag = c->at<int>(c->off.vtag);
  a.ctag = c->at<int>(c->off.ctag);
  a.vslot = c->at<int>(c->off.vslot);
  a.cslot = c->at<int>(c->off.cslot);
  a.vkey = c->at<int>(c->off.vkey);
  a.vrank = c->at<int>(c->off.vrank);
  a.vperm = c->at<int>(c->off.vperm);
  a.ckey = c->at<int>(c->off.ckey);
  a.crank = c->at<int>(c->off.crank);
  a.cperm = c->at<int>(c->off.cperm);
  a.kcount_v = c->at<int>(c->off.kcount_v);
  a.kstart_v = c->at<int>(c->off.kstart_v);
  a.kpart_v = c->at<int>(c->off.kpart_v);
  a.kcount_c = c->at<int>(c->off.kcount_c);
  a.kstart_c = c->at<int>(c->off.kstart_c);
  a.kpart_c = c->at<int>(c->off.kpart_c);
  a.vc_s = c->at<int>(c->off.vc_s);
  a.vn_s = c->at<int>(c->off.vn_s);
  a.cc_s = c->at<int>(c->off.cc_s);
  a.cv_s = c->at<int>(c->off.cv_s);
  a.vtag_s = c->at<int>(c->off.vtag_s);
  a.ctag_s = c->at<int>(c->off.ctag_s);
  a.theta_s = c->at<double>(c->off.theta_s);
  a.p0_s = c->at<double>(c->off.p0_s);
  a.v0_s = c->at<double>(c->off.v0_s);
  a.a0_s = c->at<double>(c->off.a0_s);
  a.P0_s = c->at<double>(c->off.P0_s);
  return a;
}

// Re-sort (by_tag 0: along the Hilbert curves; 1: back to the order as
// built), then the float copies, the locks and the next step's director
// terms of the moved state (the same values: they depend on tags only).
int enqueue_sort(cg_avm_ctx* c, int by_tag) {
  cudaStream_t st = c->stream;
  launch_avm_sort(sort_args(c, by_tag), st);
  const AvmArgs a = avm_args(c);
  launch_avm_shadow(a, st);
  launch_fill_u64(c->n, ~0ull, a.lock, st);
  launch_avm_dir(a, st);
  AV_CUDA(c, cudaGetLastError());
  c->permuted = !by_tag;
  c->since_sort = 0;
  return CG_OK;
}

// A per-slot double array in tag order: straight copy when slots are tags,
// else through a staging array (device) of the context.
int out_by_tag(cg_avm_ctx* c, double* dst, const double* src, int count, const int* tags, double* stage) {
  if (!dst) return CG_OK;
  if (!c->permuted) return copy_out(c, dst, src, (size_t)count * sizeof(double));
  launch_gather_d(count, tags, src, stage, c->stream);
  return copy_out(c, dst, stage, (size_t)count * sizeof(double));
}

// A tag-ordered double array into the per-slot array dst.
int in_by_tag(cg_avm_ctx* c, double* dst, const double* src, int count, const int* tags, double* stage) {
  if (!src) return CG_OK;
  if (!c->permuted) return copy_in(c, dst, src, (size_t)count * sizeof(double));
  int rc = copy_in(c, stage, src, (size_t)count * sizeof(double));
  if (rc) return rc;
  launch_scatter_d(count, tags, stage, dst, c->stream);
  return CG_OK;
}

// A graph of `prefix` (captured) followed by a while node whose body is one
// T1 pass (the pass's first kernel clears the handle, its closing block sets
// it again when another pass is due).
template <class Prefix, class Suffix>
int loop_graph(cg_avm_ctx* c, Prefix prefix, Suffix suffix, cudaGraphExec_t* out) {
  if (*out) {
    cudaGraphExecDestroy(*out);
    *out = nullptr;
  }
  AvmArgs a = avm_args(c);
  cudaError_t e = build_loop_graph(
      c->capture,
      [&](cudaGraphConditionalHandle h, cudaStream_t st) {
        a.loop = h;
        prefix(a, st);
      },
      [&](cudaGraphConditionalHandle h, cudaStream_t st) {
        a.loop = h;
        launch_avm_t1_pass(a, st);
      },
      suffix, out);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return afail(c, CG_ECUDA, std::string("building the T1 loop graph: ") + cudaGetErrorString(e));
  }
  return CG_OK;
}

// The first T1 pass of a step runs as plain graph nodes before the while
// node (every step has one); the node then runs only the further passes.
int avm_graphs(cg_avm_ctx* c) {
  // the step: geometry, vertex forces and move; then the T1 passes beside the
  // director terms of the next step (FP64 work on a branch of its own, joined
  // at the end of the step)
  int rc = loop_graph(
      c,
      [c](const AvmArgs& a, cudaStream_t st) {
        launch_avm_move(a, st);
        cudaEventRecord(c->fork, st);
        cudaStreamWaitEvent(c->side, c->fork, 0);
        launch_avm_dir(a, c->side);
        cudaEventRecord(c->join, c->side);
        launch_avm_t1_pass(a, st);
      },
      [c](cudaStream_t st) { cudaStreamWaitEvent(st, c->join, 0); }, &c->exec);
  if (rc) return rc;
  rc = loop_graph(
      c,
      [](const AvmArgs& a, cudaStream_t st) {
        launch_avm_begin_t1(a.ctl, st);
        launch_avm_t1_pass(a, st);
      },
      [](cudaStream_t) {}, &c->t1_exec);
  if (rc) return rc;
  // division rounds: locks, prefix, dry runs, slots, application, advance
  DivArgs d{};
  d.g = avm_args(c);
  d.cells = c->at<int>(c->off.div_cells);
  d.dirs = c->at<double>(c->off.div_dirs);
  d.cslots = c->at<int>(c->off.div_cslots);
  d.vslots = c->at<int>(c->off.div_vslots);
  d.made = c->at<int>(c->off.div_made);
  d.dlock = c->at<unsigned long long>(c->off.div_lock);
  d.flag = c->at<int>(c->off.div_flag);
  d.dc = c->at<DivCtl>(c->off.div_ctl);
  if (c->div_exec) {
    cudaGraphExecDestroy(c->div_exec);
    c->div_exec = nullptr;
  }
  cudaError_t e = build_loop_graph(
      c->capture,
      [&](cudaGraphConditionalHandle h, cudaStream_t st) {
        d.loop = h;
        launch_avm_divide_begin(d, st);
      },
      [&](cudaGraphConditionalHandle h, cudaStream_t st) {
        d.loop = h;
        launch_avm_divide_round(d, st);
      },
      [](cudaStream_t) {}, &c->div_exec);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return afail(c, CG_ECUDA, std::string("building the division graph: ") + cudaGetErrorString(e));
  }
  return CG_OK;
}

}  // namespace

extern "C" {

int cg_avm_workspace_bytes(int32_t n, double Lx, double Ly, size_t* bytes) {
  return cg_avm_workspace_bytes_capacity(n, n, Lx, Ly, bytes);
}

int cg_avm_workspace_bytes_capacity(int32_t n, int32_t capacity, double Lx, double Ly, size_t* bytes) {
  if (!bytes || n < 16 || capacity < n || capacity > (1 << 26)) return CG_EINVAL;
  cg_replica r{n, Lx, Ly, 3.8, 0.0};
  size_t spv = 0;
  int rc = cg_workspace_bytes(1, &r, &spv);
  if (rc) return rc;
  *bytes = avm_layout(capacity, spv).total;
  return CG_OK;
}

int cg_avm_create(int32_t n, double Lx, double Ly, double p0, double v0, const cg_avm_params* par, const double* x,
                  const double* y, const double* theta, void* d_ws, size_t ws_bytes, void* stream, cg_avm_ctx** out) {
  if (!out) return CG_EINVAL;
  *out = nullptr;
  if (!par || !x || !y || !theta || !d_ws || ((uintptr_t)d_ws & 255) || n < 16) return CG_EINVAL;
  if (!(par->dt > 0) || !(par->A0 > 0) || !(par->t1_threshold >= 0) || !(par->t2_area >= 0) || par->sort_every < 0)
    return CG_EINVAL;
  for (double v : {par->A0, par->KA, par->KP, par->mu, par->Dr, par->dt, par->t1_threshold, par->t1_length,
                   par->t2_area, p0, v0})
    if (!std::isfinite(v)) return CG_EINVAL;
  const int ncap = par->cell_capacity > 0 ? par->cell_capacity : n;
  size_t need = 0;
  int rc = cg_avm_workspace_bytes_capacity(n, ncap, Lx, Ly, &need);
  if (rc) return rc;
  if (ws_bytes < need) return CG_EINVAL;
  cg_avm_ctx* c = new (std::nothrow) cg_avm_ctx();
  if (!c) return CG_EINVAL;
  c->n = ncap;
  c->V = 2 * ncap;
  c->n_seed = n;
  c->par = *par;
  c->ws = static_cast<char*>(d_ws);
  c->stream = static_cast<cudaStream_t>(stream);
  cg_replica r{n, Lx, Ly, p0, v0};
  size_t spv_bytes = 0;
  cg_workspace_bytes(1, &r, &spv_bytes);
  c->off = avm_layout(ncap, spv_bytes);
  // Hilbert grids with at most V (n) keys: about two vertices (one cell) each
  while (c->hord_v < 15 && (int64_t(1) << (2 * (c->hord_v + 1))) <= c->V) ++c->hord_v;
  while (c->hord_c < 15 && (int64_t(1) << (2 * (c->hord_c + 1))) <= c->n) ++c->hord_c;
  do {
    if (cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming) != cudaSuccess) { rc = CG_ECUDA; break; }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) { rc = CG_ECUDA; break; }
    // exact Delaunay triangulation of the seeds (temporary SPV context)
    cg_params sp{};
    sp.A0 = par->A0; sp.KA = 1.0; sp.KP = 1.0; sp.mu = 1.0; sp.Dr = 0.0; sp.dt = 0.01; sp.seed = 0;
    sp.repair_cap = 4; sp.sort_every = 0;
    cg_ctx* spv = nullptr;
    rc = cg_create(1, &r, &sp, x, y, theta, c->ws + c->off.spv, spv_bytes, stream, &spv);
    if (rc) { c->last_error = "triangulation of the seeds failed"; break; }
    rc = cg_get_neighbors(spv, c->at<int>(c->off.cnt), c->at<int>(c->off.nbr));
    if (!rc) rc = cg_get_state(spv, c->at<double>(c->off.xs), c->at<double>(c->off.ys), nullptr);
    // box rounded to the position grid 2^-q, as the seeds are
    if (!rc) {
      int ex;
      const double fr = std::frexp(std::fmax(Lx, Ly), &ex);
      const int q = 50 - ((fr == 0.5) ? ex - 1 : ex);
      c->Lx = std::ldexp(std::rint(std::ldexp(Lx, q)), -q);
      c->Ly = std::ldexp(std::rint(std::ldexp(Ly, q)), -q);
    }
    cg_destroy(spv);
    if (rc) break;
    cudaStream_t st = c->stream;
    Ctl h;
    std::memset(&h, 0, sizeof(h));
    if (cudaMemcpyAsync(c->ctl(), &h, sizeof(Ctl), cudaMemcpyHostToDevice, st) != cudaSuccess) { rc = CG_ECUDA; break; }
    // slots past the initial network: empty cells and free vertices
    const size_t Vc = (size_t)c->V;
    if (cudaMemsetAsync(c->at<int>(c->off.cc), 0, (size_t)ncap * sizeof(int), st) != cudaSuccess ||
        cudaMemsetAsync(c->at<int>(c->off.cv), 0xff, (size_t)ncap * CG_RING * sizeof(int), st) != cudaSuccess ||
        cudaMemsetAsync(c->at<int>(c->off.vc), 0xff, 3 * Vc * sizeof(int), st) != cudaSuccess ||
        cudaMemsetAsync(c->at<int>(c->off.vn), 0xff, 3 * Vc * sizeof(int), st) != cudaSuccess ||
        cudaMemsetAsync(c->at<double>(c->off.hx), 0, 2 * Vc * sizeof(double), st) != cudaSuccess ||
        cudaMemsetAsync(c->at<double>(c->off.hy), 0, 2 * Vc * sizeof(double), st) != cudaSuccess ||
        cudaMemsetAsync(c->at<double>(c->off.theta), 0, (size_t)ncap * sizeof(double), st) != cudaSuccess ||
        cudaMemsetAsync(c->at<int>(c->off.kcount_v), 0, ((size_t)c->V + 2) * sizeof(int), st) != cudaSuccess ||
        cudaMemsetAsync(c->at<int>(c->off.kcount_c), 0, ((size_t)ncap + 2) * sizeof(int), st) != cudaSuccess) {
      rc = CG_ECUDA;
      break;
    }
    // slots in the order as built: tag = slot
    launch_iota2(c->V, c->at<int>(c->off.vtag), c->at<int>(c->off.vslot), st);
    launch_iota2(ncap, c->at<int>(c->off.ctag), c->at<int>(c->off.cslot), st);
    AvmBuildArgs b{};  // every field starts zero or null
    b.n = n;
    b.ctl = c->ctl();
    b.Lx = c->Lx;
    b.Ly = c->Ly;
    b.x = c->at<double>(c->off.xs);
    b.y = c->at<double>(c->off.ys);
    b.cnt = c->at<int>(c->off.cnt);
    b.nbr = c->at<int>(c->off.nbr);
    b.owned = c->at<int>(c->off.owned);
    b.base_local = c->at<int>(c->off.base_local);
    b.base_partial = c->at<int>(c->off.base_partial);
    b.vc = c->at<int>(c->off.vc);
    b.vn = c->at<int>(c->off.vn);
    b.cc = c->at<int>(c->off.cc);
    b.cv = c->at<int>(c->off.cv);
    b.hx = c->at<double>(c->off.hx);
    b.hy = c->at<double>(c->off.hy);
    launch_avm_build(b, st);
    launch_avm_validate(avm_args(c), st);
    launch_avm_shadow(avm_args(c), st);
    rc = copy_in(c, c->at<double>(c->off.theta), theta, n * sizeof(double));
    if (rc) break;
    launch_check_finite(n, c->at<double>(c->off.theta), c->ctl(), st);
    launch_init_dir_tables(c->at<double2>(c->off.dir_tab), st);
    launch_fill_d(ncap, p0, c->at<double>(c->off.p0), st);
    launch_fill_d(ncap, c->par.A0, c->at<double>(c->off.a0), st);
    launch_avm_p0s(avm_args(c), st);
    launch_fill_d(ncap, v0, c->at<double>(c->off.v0), st);
    launch_fill_u64(ncap, ~0ull, c->at<unsigned long long>(c->off.lock), st);
    if (cudaMemsetAsync(c->at<unsigned int>(c->off.done), 0, 2 * sizeof(unsigned int), st) != cudaSuccess) {
      rc = CG_ECUDA;
      break;
    }
    launch_avm_dir(avm_args(c), st);
    rc = avm_status(c);
    if (rc) break;
    if (c->par.sort_every > 0 && (rc = enqueue_sort(c, 0))) break;
    rc = avm_graphs(c);
  } while (0);
  if (rc) {
    cg_avm_destroy(c);
    return rc;
  }
  *out = c;
  return CG_OK;
}

int cg_avm_step(cg_avm_ctx* c, int64_t nsteps) {
  if (!c || nsteps < 0) return CG_EINVAL;
  if (c->broken) return afail(c, CG_EINVAL, "context holds a device error: " + c->last_error);
  for (int64_t s = 0; s < nsteps; ++s) {
    AV_CUDA(c, cudaGraphLaunch(c->exec, c->stream));
    if (c->par.sort_every > 0 && ++c->since_sort >= c->par.sort_every) {
      const int rc = enqueue_sort(c, 0);
      if (rc) return rc;
    }
  }
  return CG_OK;
}

int cg_avm_profile_step(cg_avm_ctx* c, int64_t nsteps, double* ms_out, int32_t n_out) {
  if (!c || !ms_out || n_out < CG_AVM_NUM_PHASES || nsteps < 0) return CG_EINVAL;
  int rc = avm_status(c);
  if (rc) return rc;
  cudaStream_t st = c->stream;
  cudaEvent_t ev[3];
  for (int k = 0; k < 3; ++k) AV_CUDA(c, cudaEventCreate(&ev[k]));
  for (int k = 0; k < CG_AVM_NUM_PHASES; ++k) ms_out[k] = 0.0;
  AvmArgs a = avm_args(c);  // loop handle 0: the pass control is read back here
  float ms = 0.f;
  for (int64_t s = 0; s < nsteps && !rc; ++s) {
    cudaEventRecord(ev[0], st);
    launch_avm_move(a, st, 1);
    cudaEventRecord(ev[1], st);
    launch_avm_move(a, st, 2);
    cudaEventRecord(ev[2], st);
    if (cudaEventSynchronize(ev[2]) != cudaSuccess) { rc = afail(c, CG_ECUDA, "profile sync"); break; }
    cudaEventElapsedTime(&ms, ev[0], ev[1]);
    ms_out[0] += ms;
    cudaEventElapsedTime(&ms, ev[1], ev[2]);
    ms_out[1] += ms;
    // the director terms of the next step (beside the T1 passes in the graph)
    cudaEventRecord(ev[0], st);
    launch_avm_dir(a, st);
    cudaEventRecord(ev[1], st);
    if (cudaEventSynchronize(ev[1]) != cudaSuccess) { rc = afail(c, CG_ECUDA, "profile sync"); break; }
    cudaEventElapsedTime(&ms, ev[0], ev[1]);
    ms_out[4] += ms;
    for (int pass = 0; pass <= cap_of(c) + 1; ++pass) {
      cudaEventRecord(ev[0], st);
      launch_avm_t1_pass(a, st);
      cudaEventRecord(ev[1], st);
      Ctl h;
      if (cudaMemcpyAsync(&h, c->ctl(), sizeof(Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) { rc = afail(c, CG_ECUDA, "profile sync"); break; }
      cudaEventElapsedTime(&ms, ev[0], ev[1]);
      ms_out[2] += ms;
      ms_out[3] += 1.0;
      if (!h.pad || h.status) break;
    }
  }
  for (int k = 0; k < 3; ++k) cudaEventDestroy(ev[k]);
  if (rc) return rc;
  return avm_status(c);
}

int cg_avm_sync(cg_avm_ctx* c) { return c ? avm_status(c) : CG_EINVAL; }

int cg_avm_get_state(cg_avm_ctx* c, double* hx, double* hy, double* theta) {
  if (!c) return CG_EINVAL;
  int rc = avm_status(c);
  if (rc) return rc;
  Ctl h;
  AV_CUDA(c, cudaMemcpy(&h, c->ctl(), sizeof(Ctl), cudaMemcpyDeviceToHost));
  const size_t V = c->V;
  const int* vtag = c->at<int>(c->off.vtag);
  const int* ctag = c->at<int>(c->off.ctag);
  // staging: the permuted-copy arrays of the re-sort (3V ints >= V doubles)
  if ((rc = out_by_tag(c, hx, c->at<double>(c->off.hx) + h.cur * V, c->V, vtag, c->at<double>(c->off.vc_s))))
    return rc;
  if ((rc = out_by_tag(c, hy, c->at<double>(c->off.hy) + h.cur * V, c->V, vtag, c->at<double>(c->off.vn_s))))
    return rc;
  if ((rc = out_by_tag(c, theta, c->at<double>(c->off.theta), c->n, ctag, c->at<double>(c->off.theta_s)))) return rc;
  return avm_status(c);
}

int cg_avm_get_topology(cg_avm_ctx* c, int32_t* vc, int32_t* vn, int32_t* cc, int32_t* cv) {
  if (!c) return CG_EINVAL;
  int rc = avm_status(c);
  if (rc) return rc;
  const int *svc = c->at<int>(c->off.vc), *svn = c->at<int>(c->off.vn);
  const int *scc = c->at<int>(c->off.cc), *scv = c->at<int>(c->off.cv);
  if (c->permuted) {  // in tag order, entries renamed to tags
    launch_avm_topology_by_tag(avm_args(c), c->at<int>(c->off.vslot), c->at<int>(c->off.cslot),
                               c->at<int>(c->off.vc_s), c->at<int>(c->off.vn_s), c->at<int>(c->off.cc_s),
                               c->at<int>(c->off.cv_s), c->stream);
    svc = c->at<int>(c->off.vc_s);
    svn = c->at<int>(c->off.vn_s);
    scc = c->at<int>(c->off.cc_s);
    scv = c->at<int>(c->off.cv_s);
  }
  if ((rc = copy_out(c, vc, svc, 3 * (size_t)c->V * sizeof(int)))) return rc;
  if ((rc = copy_out(c, vn, svn, 3 * (size_t)c->V * sizeof(int)))) return rc;
  if ((rc = copy_out(c, cc, scc, (size_t)c->n * sizeof(int)))) return rc;
  if ((rc = copy_out(c, cv, scv, (size_t)c->n * CG_RING * sizeof(int)))) return rc;
  return avm_status(c);
}

int cg_avm_set_state(cg_avm_ctx* c, const double* hx, const double* hy, const double* theta, const int32_t* vc,
                     const int32_t* vn, const int32_t* cc, const int32_t* cv) {
  if (!c || !hx || !hy) return CG_EINVAL;
  int rc = avm_status(c);
  if (rc) return rc;
  // arrays in tag order: slots back to tags first (the next re-sort is due
  // sort_every steps later)
  if (c->permuted && (rc = enqueue_sort(c, 1))) return rc;
  Ctl h;
  AV_CUDA(c, cudaMemcpy(&h, c->ctl(), sizeof(Ctl), cudaMemcpyDeviceToHost));
  const size_t V = c->V;
  if ((rc = copy_in(c, c->at<double>(c->off.hx) + h.cur * V, hx, V * sizeof(double)))) return rc;
  if ((rc = copy_in(c, c->at<double>(c->off.hy) + h.cur * V, hy, V * sizeof(double)))) return rc;
  if ((rc = copy_in(c, c->at<double>(c->off.theta), theta, c->n * sizeof(double)))) return rc;
  if (theta) launch_check_finite(c->n, c->at<double>(c->off.theta), c->ctl(), c->stream);
  launch_check_finite(c->V, c->at<double>(c->off.hx) + h.cur * V, c->ctl(), c->stream);
  launch_check_finite(c->V, c->at<double>(c->off.hy) + h.cur * V, c->ctl(), c->stream);
  if ((rc = copy_in(c, c->at<int>(c->off.vc), vc, 3 * V * sizeof(int)))) return rc;
  if ((rc = copy_in(c, c->at<int>(c->off.vn), vn, 3 * V * sizeof(int)))) return rc;
  if ((rc = copy_in(c, c->at<int>(c->off.cc), cc, c->n * sizeof(int)))) return rc;
  if ((rc = copy_in(c, c->at<int>(c->off.cv), cv, c->n * CG_RING * sizeof(int)))) return rc;
  launch_avm_validate(avm_args(c), c->stream);
  launch_avm_shadow(avm_args(c), c->stream);
  launch_avm_dir(avm_args(c), c->stream);  // director terms of the next step
  return avm_status(c);
}

int cg_avm_get_cell_params(cg_avm_ctx* c, double* p0, double* v0, double* a0) {
  if (!c) return CG_EINVAL;
  int rc = avm_status(c);
  if (rc) return rc;
  const int* ctag = c->at<int>(c->off.ctag);
  if ((rc = out_by_tag(c, p0, c->at<double>(c->off.p0), c->n, ctag, c->at<double>(c->off.p0_s)))) return rc;
  if ((rc = out_by_tag(c, v0, c->at<double>(c->off.v0), c->n, ctag, c->at<double>(c->off.v0_s)))) return rc;
  if ((rc = out_by_tag(c, a0, c->at<double>(c->off.a0), c->n, ctag, c->at<double>(c->off.a0_s)))) return rc;
  return avm_status(c);
}

int cg_avm_set_step(cg_avm_ctx* c, int64_t step) {
  if (!c || step < 0) return CG_EINVAL;
  int rc = avm_status(c);
  if (rc) return rc;
  Ctl h;
  AV_CUDA(c, cudaMemcpy(&h, c->ctl(), sizeof(Ctl), cudaMemcpyDeviceToHost));
  h.step = step;
  AV_CUDA(c, cudaMemcpy(c->ctl(), &h, sizeof(Ctl), cudaMemcpyHostToDevice));
  launch_avm_dir(avm_args(c), c->stream);  // the next step's noise depends on the counter
  return avm_status(c);
}

int cg_avm_get_geometry(cg_avm_ctx* c, double* A, double* P) {
  if (!c) return CG_EINVAL;
  launch_avm_forces(avm_args(c), c->stream);
  int rc;
  const int* ctag = c->at<int>(c->off.ctag);
  if ((rc = out_by_tag(c, A, c->at<double>(c->off.A), c->n, ctag, c->at<double>(c->off.p0_s)))) return rc;
  if ((rc = out_by_tag(c, P, c->at<double>(c->off.P), c->n, ctag, c->at<double>(c->off.v0_s)))) return rc;
  return avm_status(c);
}

int cg_avm_get_forces(cg_avm_ctx* c, double* Fx, double* Fy, double* energy) {
  if (!c) return CG_EINVAL;
  AvmArgs a = avm_args(c);
  a.energy = c->at<double>(c->off.energy);
  launch_avm_forces(a, c->stream);
  int rc;
  const int* vtag = c->at<int>(c->off.vtag);
  if ((rc = out_by_tag(c, Fx, c->at<double>(c->off.Fx), c->V, vtag, c->at<double>(c->off.vc_s)))) return rc;
  if ((rc = out_by_tag(c, Fy, c->at<double>(c->off.Fy), c->V, vtag, c->at<double>(c->off.vn_s)))) return rc;
  if (energy) {
    const double* e = a.energy;
    if (c->permuted) {  // summed in tag order, as without a re-sort
      launch_gather_d(c->n, c->at<int>(c->off.ctag), a.energy, c->at<double>(c->off.theta_s), c->stream);
      e = c->at<double>(c->off.theta_s);
    }
    launch_reduce_sum(c->n, e, c->at<double>(c->off.scalar), c->stream);
    AV_CUDA(c, cudaMemcpyAsync(energy, c->at<double>(c->off.scalar), sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  return avm_status(c);
}

int cg_avm_t1(cg_avm_ctx* c) {
  if (!c) return CG_EINVAL;
  int rc = avm_status(c);
  if (rc) return rc;
  if (c->broken) return afail(c, CG_EINVAL, "context holds a device error: " + c->last_error);
  AV_CUDA(c, cudaGraphLaunch(c->t1_exec, c->stream));
  return avm_status(c);
}

int cg_avm_set_p0(cg_avm_ctx* c, const double* p0) {
  if (!c || !p0) return CG_EINVAL;
  int rc = in_by_tag(c, c->at<double>(c->off.p0), p0, c->n, c->at<int>(c->off.ctag), c->at<double>(c->off.p0_s));
  if (rc) return rc;
  launch_check_finite(c->n, c->at<double>(c->off.p0), c->ctl(), c->stream);
  launch_avm_p0s(avm_args(c), c->stream);
  return avm_status(c);
}
int cg_avm_divide(cg_avm_ctx* c, int32_t count, const int32_t* cells, const double* dirs, int32_t* made,
                  int32_t* n_made) {
  if (!c || count < 0) return CG_EINVAL;
  if (count == 0) {
    if (n_made) *n_made = 0;
    return CG_OK;
  }
  if (!cells || !dirs || count > c->n) return CG_EINVAL;
  if (c->broken) return afail(c, CG_EINVAL, "context holds a device error: " + c->last_error);
  int rc = CG_OK;
  // staged: the cells (tags) and directions; on the device the cells are
  // mapped to slots and the slots the divisions may take listed in order
  // (the empty cells and the free vertices of lowest tag: a call only fills
  // slots); with too few of them the rounds do nothing.  One synchronisation,
  // at the end.
  DivCtl* dctl = c->at<DivCtl>(c->off.div_ctl);
  int* dc = c->at<int>(c->off.div_cells);
  double* dd = c->at<double>(c->off.div_dirs);
  int* dm = c->at<int>(c->off.div_made);
  if ((rc = copy_in(c, dc, cells, (size_t)count * sizeof(int)))) return rc;
  if ((rc = copy_in(c, dd, dirs, 2 * (size_t)count * sizeof(double)))) return rc;
  AV_CUDA(c, cudaMemcpyAsync(&dctl->count, &count, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  launch_check_finite(2 * count, dd, c->ctl(), c->stream);
  DivArgs d{};
  d.g = avm_args(c);
  d.cells = dc;
  d.cslots = c->at<int>(c->off.div_cslots);
  d.vslots = c->at<int>(c->off.div_vslots);
  d.dc = dctl;
  launch_avm_divide_slots(d, c->at<int>(c->off.cslot), c->at<int>(c->off.vslot), c->at<int>(c->off.kcount_c),
                          c->at<int>(c->off.kstart_c), c->at<int>(c->off.kpart_c), c->at<int>(c->off.kcount_v),
                          c->at<int>(c->off.kstart_v), c->at<int>(c->off.kpart_v), c->stream);
  // the re-sort's key counts served as scan input: cleared again
  AV_CUDA(c, cudaMemsetAsync(c->at<int>(c->off.kcount_c), 0, ((size_t)c->n + 2) * sizeof(int), c->stream));
  AV_CUDA(c, cudaMemsetAsync(c->at<int>(c->off.kcount_v), 0, ((size_t)c->V + 2) * sizeof(int), c->stream));
  AV_CUDA(c, cudaGraphLaunch(c->div_exec, c->stream));
  launch_avm_dir(avm_args(c), c->stream);  // the daughters' director terms
  AV_CUDA(c, cudaGetLastError());
  std::vector<int> hm(count);
  DivCtl hd;
  AV_CUDA(c, cudaMemcpyAsync(hm.data(), dm, (size_t)count * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  AV_CUDA(c, cudaMemcpyAsync(&hd, dctl, sizeof(DivCtl), cudaMemcpyDeviceToHost, c->stream));
  rc = avm_status(c);  // synchronizes
  if (rc) return rc;
  if (hd.stop == 2) return afail(c, CG_EINVAL, "not enough free cell slots for the divisions");
  if (made) AV_CUDA(c, cudaMemcpy(made, hm.data(), (size_t)count * sizeof(int), cudaMemcpyDefault));
  if (n_made) {
    int t = 0;
    for (int v : hm) t += v;
    *n_made = t;
  }
  return CG_OK;
}

int cg_avm_set_a0(cg_avm_ctx* c, const double* a0) {
  if (!c || !a0) return CG_EINVAL;
  int rc = in_by_tag(c, c->at<double>(c->off.a0), a0, c->n, c->at<int>(c->off.ctag), c->at<double>(c->off.a0_s));
  if (rc) return rc;
  launch_avm_p0s(avm_args(c), c->stream);  // also refuses a negative or non-finite A0
  return avm_status(c);
}

int cg_avm_set_v0(cg_avm_ctx* c, const double* v0) {
  if (!c || !v0) return CG_EINVAL;
  int rc = in_by_tag(c, c->at<double>(c->off.v0), v0, c->n, c->at<int>(c->off.ctag), c->at<double>(c->off.v0_s));
  if (rc) return rc;
  launch_check_finite(c->n, c->at<double>(c->off.v0), c->ctl(), c->stream);
  launch_avm_dir(avm_args(c), c->stream);  // the activity of the next step
  return avm_status(c);
}

int cg_avm_get_counters(cg_avm_ctx* c, cg_counters* out) {
  if (!c || !out) return CG_EINVAL;
  AV_CUDA(c, cudaStreamSynchronize(c->stream));
  Ctl h;
  AV_CUDA(c, cudaMemcpy(&h, c->ctl(), sizeof(Ctl), cudaMemcpyDeviceToHost));
  out->steps = h.step;
  out->flagged_total = h.flagged_total;    // T2 transitions
  out->repaired_total = h.repaired_total;  // T1 transitions
  out->last_flagged = 0;
  out->last_rounds = h.round_count;        // T1 passes
  out->status = h.status;
  out->reserved = 0;
  out->loop_total = h.loop_total;
  return CG_OK;
}

int cg_avm_sort(cg_avm_ctx* c) {
  if (!c) return CG_EINVAL;
  int rc = avm_status(c);
  if (rc) return rc;
  if ((rc = enqueue_sort(c, 0))) return rc;
  return avm_status(c);
}

int cg_avm_get_tags(cg_avm_ctx* c, int32_t* vtag, int32_t* ctag) {
  if (!c) return CG_EINVAL;
  int rc = avm_status(c);
  if (rc) return rc;
  if ((rc = copy_out(c, vtag, c->at<int>(c->off.vtag), (size_t)c->V * sizeof(int)))) return rc;
  if ((rc = copy_out(c, ctag, c->at<int>(c->off.ctag), (size_t)c->n * sizeof(int)))) return rc;
  return avm_status(c);
}

int cg_avm_destroy(cg_avm_ctx* c) {
  if (!c) return CG_EINVAL;
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->t1_exec) cudaGraphExecDestroy(c->t1_exec);
  if (c->div_exec) cudaGraphExecDestroy(c->div_exec);
  if (c->capture) cudaStreamDestroy(c->capture);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->join) cudaEventDestroy(c->join);
  delete c;
  return CG_OK;
}

const char* cg_avm_last_error(const cg_avm_ctx* c) { return c ? c->last_error.c_str() : "null context"; }

}  // extern "C"
