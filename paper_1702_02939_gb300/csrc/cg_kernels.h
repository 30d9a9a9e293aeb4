// Kernel argument blocks and host-side launchers of the cellgb library.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace cgk {

struct Rep;
struct Ctl;

constexpr int kGeomThreads = 32;   // one warp: finer blocks than 64 cut k_geom by ~4% at N = 262144
constexpr int kGeomSh = 10;        // ring slots of k_geom held in shared memory (longer rings: local)
constexpr int kGeomMinBlocks = 20;  // resident one-warp blocks per SM that k_geom is compiled for
constexpr int kForceThreads = 128;
constexpr int kTestThreads = 128;
constexpr int kRepairWarps = 4;  // warps per repair block
constexpr int kCand = 64;        // candidate buffer per repair warp

struct GeomArgs {
  int n;
  const Rep* reps;
  const int* rep;
  Ctl* ctl;
  const long long *X, *Y;  // [2][n] grid coordinates
  const int *cnt, *nbr;
  const double* p0;
  double A0, sqrtA0, KA, KP;
  double *A, *P;
  double* energy_out;   // per-cell energy or nullptr
  double2 *fs, *s, *w;  // [CG_RING][n]
  // Cells to process: list[0 .. *list_count) if list is set, else all.
  const int* list;
  const int* list_count;
  unsigned* list_bits;  // bit of each listed cell, cleared once processed
  // Rings may be rewritten concurrently (the pass beside the repair rounds):
  // out-of-range entries are skipped and no status is raised; every cell whose
  // ring changes is processed again afterwards.
  int tolerant;
  // Processing order of all cells (a permutation of 0..n-1, cells of equal
  // ring size grouped; see launch_order), or null for 0..n-1.  Unused with list.
  const int* order;
};

struct ForceArgs {
  int n;
  const Rep* reps;
  const int* rep;
  Ctl* ctl;
  const int *cnt, *nbr, *tag;
  const double2 *fs, *s, *w;
  double *Fx, *Fy;
  int integrate;       // 0 forces, 1 forces + move of Eq. 3, 2 the move from the stored Fx, Fy
  double *x, *y;       // [2][n]
  long long *X, *Y;    // [2][n]
  double* theta;
  double* v0;
  // integrate 2 only: new speeds in user order (or nullptr), stored into v0
  // (through tag) before the move, a non-finite one raising CG_EINVAL
  const double* v0_user;
  double mu, dt, noise_amp;
  unsigned long long seed;
  const double2* nrm;  // (cos, sin) of each cell's director, from k_dir
  const double* xi;    // the step's director noise, from k_dir
  const int* order;    // processing order of the cells (as GeomArgs), or null
  // Beside the repair rounds (tolerant): rings may be rewritten meanwhile; a
  // cell whose ring, neighbours or move look wrong raises nothing and is
  // put on the fix-up list (fix_list, fix_bits, ctl->force_count) instead.
  int tolerant;
  int* fix_list;
  unsigned* fix_bits;
  // Fix-up: only the cells of list[0 .. *list_count), clearing their bits
  const int* list;
  const int* list_count;
  unsigned* list_bits;
};
// The cells whose force the step recomputes after the repair rounds: every
// cell whose ring a round rewrote and every cell of its new ring, added once
// each to the fix-up list (beside the cells the tolerant pass put there).
struct ForceFixArgs {
  int n;
  const int *cnt, *nbr;
  const int* dirty_list;
  const int* dirty_count;
  int* fix_list;
  unsigned* fix_bits;
  Ctl* ctl;
};
void launch_force_fix_list(const ForceFixArgs& a, int blocks, cudaStream_t st);

// Cells of each chunk of kOrderChunk consecutive cells regrouped by ring size:
// a warp of the geometry and force kernels then runs cells with (mostly) the
// same number of ring slots, so its lanes stay active through the slot loop.
// order becomes a permutation of 0..n-1 whatever the ring sizes read (rings
// may be rewritten concurrently; each cell is placed exactly once).
constexpr int kOrderChunk = 1024;
void launch_order(int n, const int* cnt, int* order, cudaStream_t st);

// Director terms of the next move, computed off the critical path: n(theta)
// and the Philox/Box-Muller noise of the step held in the control word.
struct DirArgs {
  int n;
  Ctl* ctl;
  double* theta;
  const int* tag;
  unsigned long long seed;
  double2* nrm;
  double* xi;
  // 1 in a step: first rotate every director by the noise of the previous
  // step, theta <- theta + noise_amp * xi (Eq. 3); 0 when the terms are only
  // refreshed for the current directors
  int advance;
  double noise_amp;
  const double2* tab;  // director table (dir_math.cuh), filled by launch_init_dir_tables
};
// blocks: grid size (grid-stride loop); 0 = one thread per cell
void launch_dir(const DirArgs& a, cudaStream_t st, int blocks = 0);
// Fills the kDirTabEntries-entry director table.
void launch_init_dir_tables(double2* tab, cudaStream_t st);
// cos, sin of n angles and the noise xi(seed, tag[i], step) (FP64 path).
void launch_dir_terms(int n, const double* theta, const int* tag, unsigned long long seed, long long step,
                      const double2* tab, double* cs, double* sn, double* xi, cudaStream_t st);

struct TestArgs {
  int n;
  const Rep* reps;
  const int* rep;
  Ctl* ctl;
  const long long *X, *Y;  // [2][n]
  const int *cnt, *nbr, *tag;
  unsigned* flags;
  int* list;  // list 0
  const int* order;  // processing order of the cells (as GeomArgs), or null
};

struct CellListArgs {
  int n, nbins;
  const Rep* reps;
  const int* rep;
  Ctl* ctl;
  const long long *X, *Y;  // [2][n] grid coordinates
  int *bin_count, *bin_start, *cell_bin, *cell_rank, *ids;
  int* scan_partials;
  int only_if_flagged;  // skip when nothing is flagged
};

struct RepairArgs {
  int n;
  const Rep* reps;
  const int* rep;
  Ctl* ctl;
  const double *x, *y;     // [2][n]
  const long long *X, *Y;  // [2][n]
  const int* tag;
  const int *bin_start, *bin_partials, *ids;
  int *cnt, *nbr;
  int *old_cnt, *old_nbr;
  unsigned* flags;
  const int* list_in;
  int which_in;  // count index of list_in
  int all_cells; // process cells 0..n-1 instead of the list
  // Rounds inside a conditional (while) graph node: the input list is
  // lists[round & 1] with the round counter read from the control word.
  int dyn;
  const int* lists[2];
  cudaGraphConditionalHandle loop;
  // Cells whose ring a per-step round rewrites, each once per step (bitmap
  // dirty_bits, list dirty_list, count in the control word); null: not kept.
  int* dirty_list;
  unsigned* dirty_bits;
};

struct CheckArgs {
  int n;
  Ctl* ctl;
  const int *cnt, *nbr, *old_cnt, *old_nbr;
  unsigned* flags;
  const int* list_in;
  int* list_out;
  int which_in, which_out;
  int last_round;  // raise REPAIR_CAP if anything is flagged
  int all_cells;
  // Rounds inside a conditional (while) graph node (see RepairArgs): the last
  // block counts the round, raises REPAIR_CAP after `cap` rounds with work
  // and asks for another round while cells are left flagged.
  int dyn, cap;
  int* lists[2];
  cudaGraphConditionalHandle loop;
};

// blocks: grid size (grid-stride loop); 0 = one thread per cell (or per list entry bound n)
void launch_geom(const GeomArgs& a, cudaStream_t st, int blocks = 0);
// Single-precision variants (spv_kernels_f32.cu); same arguments.
void launch_geom_f32(const GeomArgs& a, cudaStream_t st, int blocks = 0);
void launch_force_f32(const ForceArgs& a, cudaStream_t st, int blocks = 0);
void launch_dir_f32(const DirArgs& a, cudaStream_t st, int blocks = 0);
// blocks > 0: a grid-stride launch of that many blocks (list mode)
void launch_force(const ForceArgs& a, cudaStream_t st, int blocks = 0);
void launch_begin_topology(Ctl* ctl, int flip, cudaStream_t st);
void launch_test(const TestArgs& a, cudaStream_t st, int blocks = 0);
void launch_cell_list(const CellListArgs& a, cudaStream_t st);
void launch_repair(const RepairArgs& a, int grid_blocks, cudaStream_t st);
// exclusive scan of a.bin_count[0..nbins) into (a.bin_start, a.scan_partials)
void launch_scan(const CellListArgs& a, cudaStream_t st);
void launch_check(const CheckArgs& a, int grid_blocks, cudaStream_t st);

// state preparation and user-order transfers
void launch_snap(int n, const Rep* reps, const int* rep, const double* xin, const double* yin, double* x,
                 double* y, long long* X, long long* Y, Ctl* ctl, cudaStream_t st);
void launch_gather_d(int n, const int* tag, const double* src, double* dst_user, cudaStream_t st);
void launch_check_finite(int n, const double* v, Ctl* ctl, cudaStream_t st);
void launch_scatter_d(int n, const int* tag, const double* src_user, double* dst, cudaStream_t st);
void launch_scatter_i(int n, const int* tag, const int* src_user, int* dst, cudaStream_t st);
// Halo exchange of a decomposed system: pending positions of the cells with
// slot[user index] >= 0 to/from out/in[2 slot], [2 slot + 1] as grid
// coordinates of the larger box (topo_kernels.cu).
void launch_halo_pack(int n, const int* tag, const int* slot, const Rep* reps, const int* rep, const Ctl* ctl,
                      const long long* X2, const long long* Y2, long long* out, cudaStream_t st);
void launch_halo_unpack(int n, const int* tag, const int* slot, const Rep* reps, const int* rep, Ctl* ctl,
                        const long long* in, double* x2, double* y2, long long* X2, long long* Y2, cudaStream_t st);
// positions (x2, y2: [2][n]) of buffer ctl->cur (pending 0) or of the
// pending move, buffer ctl->cur ^ 1 (pending 1), into user order; a null
// destination is skipped
void launch_gather_cur_xy(int n, const int* tag, const double* x2, const double* y2, const Ctl* ctl, int pending,
                          double* dst_x, double* dst_y, cudaStream_t st);
void launch_gather_ring(int n, const int* tag, const int* cnt, const int* nbr, int* cnt_user, int* nbr_user,
                        cudaStream_t st);
void launch_reduce_sum(int n, const double* v, double* out, cudaStream_t st);

// Hilbert re-sort of all per-cell state (sort_kernels.cu)
struct SortArgs {
  int n, nkeys;
  const Rep* reps;
  Ctl* ctl;
  double *x, *y;        // [2][n]; the permuted state goes to the other buffer
  long long *X, *Y;     // [2][n]
  double *theta, *p0, *v0;
  int *tag, *rep, *cnt, *nbr;
  // scratch
  int *key, *rank, *perm;
  int *key_count, *key_start, *key_partials;
  double *theta_alt, *p0_alt, *v0_alt;
  int *tag_alt, *rep_alt, *cnt_alt, *nbr_alt;
  int *nid, *nid_alt;  // noise counters of the cells
};
void launch_sort(const SortArgs& a, cudaStream_t st);

// Backward pass (adjoint_kernels.cu)
struct JvpArgs {
  int n;
  const Rep* reps;
  const int* rep;
  Ctl* ctl;
  const long long *X, *Y;  // [2][n]
  const int *cnt, *nbr;
  const double* p0;
  const double* theta;
  double A0, sqrtA0, KA, KP, dt, dtmu;
  const double *coefA, *coefP;  // loss coefficients instead of 2K(A-A0), 2K(P-P0), or null
  double2* v;                   // tangent / running cotangent per cell
  double *A, *P;                // optional outputs
  double *Adot, *Pdot;          // optional outputs: tangents of A and P along v
  double2 *fs, *fsd, *s, *sd, *w, *wd;  // [CG_RING][n]
  double *gp0, *gv0, *gKA, *gKP;        // per-cell accumulators, or null
  double2 *F, *Hv;                      // optional outputs of k_force_jvp
  int update;                           // v <- v - dt mu H v
};
struct Snapshot {
  double *x, *y, *theta;
  long long *X, *Y;
  int *cnt, *nbr;
  Ctl* ctl;
};
void launch_snapshot(int n, int save, Ctl* ctl, double* x, double* y, long long* X, long long* Y, double* theta,
                     int* cnt, int* nbr, const Snapshot& s, cudaStream_t st);
void launch_geom_jvp(const JvpArgs& a, cudaStream_t st);
void launch_force_jvp(const JvpArgs& a, cudaStream_t st);
void launch_combine_final(int n, const double* gx, const double* gy, const double2* F, double2* g, cudaStream_t st);
void launch_reduce2(int n, const double* a, const double* b, double* out, cudaStream_t st);

// Active vertex model (avm_kernels.cu)
struct AvmBuildArgs {
  int n;
  Ctl* ctl;
  double Lx, Ly;
  const double *x, *y;     // seed positions (user order)
  const int *cnt, *nbr;    // Delaunay rings (user order)
  int *owned, *base_local, *base_partial;
  int *vc, *vn, *cc, *cv;
  double *hx, *hy;         // first position buffer
};
// One periodic axis: the length and the bit patterns of L and L/2.
struct Axis {
  double L;
  unsigned long long L_bits, half_bits;
};
struct AvmArgs {
  int n, V;
  Ctl* ctl;
  double Lx, Ly;
  Axis ax, ay;
  float Lxf, Lyf;           // lengths for the FP32 T1 filter
  double *hx, *hy;         // [2][V]
  int *vc, *vn, *cc, *cv;
  double* theta;
  double *p0, *v0;         // [n] (written only by divisions)
  double* a0;              // [n] preferred areas A0_c
  double* P0;              // [n] preferred perimeters p0_c sqrt(A0_c)
  double KA, KP, mu, dt, noise_amp;
  unsigned long long seed;
  const double2* tab;      // director table (dir_math.cuh)
  double *A, *P, *energy;
  double *ka, *kp;         // [n] K_A (A - A0) and 2 K_P (P - P0) of each cell
  double2* act;            // [n] (v0/3) n(theta) of the step's directors
  double* thn;             // [n] the directors after the step's rotation (k_avm_dir)
  double *Fx, *Fy;
  int move;
  double thr2, t1_len;
  double t2_twice;           // T2: twice the area threshold (0: no T2)
  float t2lo, t2hi;          // FP32 squared lengths certainly below / above thr2
  float2* hf;                // [V] float copies of the current positions
  int t1_cap, apply_blocks;  // T1 pass cap; blocks of the apply kernel (of 128 threads)
  unsigned long long* lock;  // [n] pass-stamped T1 locks
  int* cand_e;               // [3V/2 + n] proposed edges 3v+s (slots), or 3V + c for a T2 of cell slot c
  int* cand_k;               // [3V/2 + n] their priorities: the same ids in tags
  int4* cand;                // [3V/2 + n] their cells (i, j, k, l), or (c, and the three across its edges)
  int4* cand_v;              // [3V/2 + n] of a T1 candidate: the other end v2 and v1's outer neighbours
                             // (v2, Aul, All, Alr) (Fig. 1 naming)
  int* cand_w;               // [3V/2 + n] and v2's other outer neighbour Aur
  const int *vtag, *ctag;    // [V], [n] the tag (API id) of each vertex and cell slot
  unsigned int* done;        // [2] last-block counters (force/move, T1 apply)
  cudaGraphConditionalHandle loop;  // while-node handle of the T1 passes
};
void launch_avm_build(const AvmBuildArgs& a, cudaStream_t st);
// part: 0 both kernels, 1 the per-cell kernel only, 2 the per-vertex kernel only
void launch_avm_move(const AvmArgs& a, cudaStream_t st, int part = 0);
// Director terms of the next step, act = (v0/3) n(theta) and the rotated
// directors thn = theta + sqrt(2 D_r dt) xi (noise counter of ctl->step); in
// the step graph beside the T1 passes, which leave the FP64 pipe idle
void launch_avm_dir(const AvmArgs& a, cudaStream_t st);
void launch_avm_begin_t1(Ctl* ctl, cudaStream_t st);
void launch_avm_t1_pass(const AvmArgs& a, cudaStream_t st);
void launch_avm_forces(const AvmArgs& a, cudaStream_t st);
void launch_avm_validate(const AvmArgs& a, cudaStream_t st);
// P0[c] = p0[c] sqrt(a0[c]) after p0 or A0 change
void launch_avm_p0s(const AvmArgs& a, cudaStream_t st);
// Divisions of a call (cells[k], direction dirs[2k], dirs[2k+1]) with the
// result of doing them in order; the divisions made take cslots[0, 1, ...]
// and vslots[0, 1, ...] in turn.  Conflict-free rounds: launch_avm_divide_begin
// once, then launch_avm_divide_round as the body of a while node (its first
// kernel clears the node's handle, its last sets it while divisions remain).
constexpr int kDivWindow = 1024;  // divisions tried per round
struct DivCtl {
  int count;  // divisions of the call (set by the host)
  int start;  // first pending division
  int end;    // end of the round's prefix of lock holders
  int used;   // divisions made so far (slots taken)
  int round;
  int stop;   // 1: a status was raised; 2: too few free slots (nothing done)
  int free_c, free_v;  // free cell and vertex slots before the call
  unsigned int done;   // last-block counter of the commit kernel
};
struct DivArgs {
  AvmArgs g;
  int* cells;  // the named cells (staged as tags, mapped to slots)
  const double* dirs;
  int *cslots, *vslots;
  int* made;
  unsigned long long* dlock;  // [n] round-stamped locks
  int* flag;                  // [kDivWindow] outcome of the round's dry runs
  DivCtl* dc;
  cudaGraphConditionalHandle loop;
};
// Before the rounds: the named cells (tags) to slots in place, and the first
// count empty cells and 2 count free vertices in increasing tag order into
// cslots and vslots (dc->free_c, free_v: how many there are).  fc/sc/scp and
// fv/sv/svp: scan scratch for n and V flags (bins and partials), left to be
// cleared by the caller.
void launch_avm_divide_slots(const DivArgs& d, const int* cslot, const int* vslot, int* fc, int* sc, int* scp,
                             int* fv, int* sv, int* svp, cudaStream_t st);
void launch_avm_divide_begin(const DivArgs& d, cudaStream_t st);
void launch_avm_divide_round(const DivArgs& d, cudaStream_t st);
void launch_avm_shadow(const AvmArgs& a, cudaStream_t st);
// Storage order of the AVM (Hilbert re-sort of the vertex and cell slots).
// Every slot carries a tag, its id in the network as built (and as the API
// speaks of it); vslot/cslot map tags back to slots.  The *_s arrays receive
// the permuted copies before they are copied back.
struct AvmSortArgs {
  int n, V;
  Ctl* ctl;
  double Lx, Ly;
  int hord_v, hord_c;             // Hilbert grid of side 2^hord for vertices and cells
  int by_tag;                     // 1: key = tag (back to the order as built)
  const double *hx, *hy;          // [2][V]
  double *hx_w, *hy_w;            // the same buffers (written: the permuted copy into the other half)
  int *vc, *vn, *cc, *cv;
  double *theta, *p0, *v0, *a0, *P0;
  int *vtag, *ctag, *vslot, *cslot;
  int *vkey, *vrank, *vperm, *ckey, *crank, *cperm;
  int *kcount_v, *kstart_v, *kpart_v, *kcount_c, *kstart_c, *kpart_c;
  int *vc_s, *vn_s, *cc_s, *cv_s, *vtag_s, *ctag_s;
  double *theta_s, *p0_s, *v0_s, *a0_s, *P0_s;
};
// Re-sorts vertices and cells along Hilbert curves (keys: vertex position;
// a cell's first vertex; freed vertices and empty cells last), or by tag
// (by_tag: every slot back to its tag).  Leaves the positions in the other
// buffer and flips ctl->cur.  Key counts: kcount/kstart [max(keys, V) + 2]
void launch_avm_sort(const AvmSortArgs& a, cudaStream_t st);
// Identity tags (tags[i] = slots[i] = i)
void launch_iota2(int n, int* tags, int* slots, cudaStream_t st);
// Network in tag order (for the API): dst arrays indexed by tag, entries
// renamed to tags (-1 kept)
void launch_avm_topology_by_tag(const AvmArgs& a, const int* vslot, const int* cslot, int* vc_out, int* vn_out,
                                int* cc_out, int* cv_out, cudaStream_t st);
void launch_fill_d(int n, double v, double* out, cudaStream_t st);
void launch_fill_u64(int n, unsigned long long v, unsigned long long* out, cudaStream_t st);

}  // namespace cgk
