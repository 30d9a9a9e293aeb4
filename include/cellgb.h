/* cellgb: GB300-native (sm_103a) self-propelled Voronoi (SPV) model.
 *
 * C ABI of libcellgb.so.  The model and every step follow D. M. Sussman,
 * "cellGPU: massively parallel simulations of dynamic vertex models",
 * arXiv 1702.02939 (cited below as "the paper"):
 *   energy           E = sum_i K_A (A_i - A0)^2 + K_P (P_i - P0_i)^2     Eq. 1
 *   force            F_i = -dE/dr_i (chain rule through the Voronoi
 *                    vertices)                                          Eqs. 2, A6-A16
 *   motion           dr_i/dt = mu F_i + v0_i n(theta_i),
 *                    dtheta_i/dt = eta_i,  <eta eta> = 2 D_r            Eq. 3
 *   topology         Delaunay triangulation of the cell positions in a
 *                    periodic box, tested by the empty-circumcircle
 *                    property after every move and repaired locally     Sec. 2.C.3-4
 *
 * Units and conventions
 *   - Cells live in periodic boxes [0, Lx) x [0, Ly).  Positions are kept on
 *     the dyadic grid 2^-q with q = 50 - ceil(log2(max(Lx, Ly))); box sides
 *     are rounded to that grid at creation.  Moves are rounded to the grid
 *     (error <= 2^-(q+1), about 1e-15 L) so that every topological decision
 *     is exact.
 *   - P0_i = p0_i * sqrt(A0): p0 is the dimensionless target shape index.
 *   - One Euler-Maruyama step: positions move with theta(t), then
 *     theta <- theta + sqrt(2 D_r dt) xi, xi a standard normal from
 *     Philox4x32-10 keyed by (seed) with counter (cell index, step, 0).
 *   - A context may hold several independent systems ("replicas"), each
 *     with its own box, p0 and v0; their cells are concatenated in replica
 *     order and cell indices below always refer to that user order.
 *
 * Memory and ownership
 *   - The caller owns all device memory.  The library needs one device
 *     workspace of cg_workspace_bytes() bytes, aligned to 256 bytes, that
 *     must stay allocated and unused by anyone else until cg_destroy().
 *   - The library owns only the opaque host context.
 *   - Array arguments marked "any" may be host or device pointers (unified
 *     addressing); pinned host memory gives the fastest transfers.
 *   - All work runs on the CUDA stream given at creation.  Calls that return
 *     data synchronize that stream before returning; cg_step() does not.
 *
 * Errors: every call returns CG_OK (0) or a negative CG_E* code.  Device
 * kernels report errors through a status word that cg_sync() and every
 * getter return; once set, it stays set.
 */
#ifndef CELLGB_H
#define CELLGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CG_MAX_RING 16

#define CG_OK 0
#define CG_EINVAL (-1)          /* bad argument or position outside [-L, 2L) */
#define CG_ECUDA (-2)           /* a CUDA runtime call failed */
#define CG_ERING_OVERFLOW (-3)  /* a cell has more than CG_MAX_RING neighbours */
#define CG_EREPAIR_CAP (-4)     /* topology not consistent after repair_cap rounds */
#define CG_ETOPO_INCONSISTENT (-5) /* j in ring(i) but i not in ring(j) during forces */
#define CG_ENONFINITE (-6)      /* a move produced a non-finite position */
#define CG_EBOX_TOO_SMALL (-7)  /* Voronoi cell wider than the search box allows */
#define CG_EDEGENERATE (-8)     /* coincident cells */
#define CG_ECANDIDATES (-9)     /* too many repair candidates in one cell-list ring */
#define CG_ET1_CAP (-10)        /* AVM: T1 candidates left after t1_cap passes */

typedef struct cg_ctx cg_ctx;

/* One independent periodic system. */
typedef struct cg_replica {
  int32_t n;      /* cells, >= 16 */
  double Lx, Ly;  /* box sides */
  double p0;      /* default target shape index of its cells */
  double v0;      /* default self-propulsion speed of its cells */
} cg_replica;

/* Parameters shared by all replicas (Eqs. 1 and 3 of the paper). */
typedef struct cg_params {
  double A0;           /* preferred area */
  double KA, KP;       /* area and perimeter moduli */
  double mu;           /* mobility */
  double Dr;           /* rotational diffusion constant */
  double dt;           /* time step */
  uint64_t seed;       /* Philox key of the director noise */
  int32_t repair_cap;  /* repair rounds per step, >= 1 (default 4) */
  int32_t sort_every;  /* Hilbert re-sort period in steps; 0 = never */
  int32_t precision;   /* 0: FP64 physics (default); 1: FP32 geometry, forces and
                          director terms (positions stay on the exact grid and every
                          topological decision stays exact; no backward pass) */
  int32_t reserved;    /* 0 */
} cg_params;

/* Counters accumulated on the device since creation. */
typedef struct cg_counters {
  int64_t steps;           /* steps taken (the Philox step counter) */
  int64_t flagged_total;   /* cells flagged by the circumcircle test */
  int64_t repaired_total;  /* cell repairs (all rounds) */
  int32_t last_flagged;    /* flagged cells in the last step */
  int32_t last_rounds;     /* repair rounds in the last step */
  int32_t status;          /* device status word */
  int32_t reserved;
  int64_t loop_total;      /* iterations of the step graph's loop node (repair
                              rounds; T1 passes for the AVM) since creation */
} cg_counters;

/* Launch shapes of the step graph.  They change timing only: every result
 * is the same for any valid setting. */
typedef struct cg_launch {
  int32_t repair_blocks_per_sm;  /* repair-round grid = SMs x this (1..64, default 4) */
  int32_t check_blocks_per_sm;   /* consistency-check grid = SMs x this (1..64, default 4) */
  int32_t dir_blocks_per_sm;     /* director branch grid = SMs x this; 0 = one thread per cell
                                    (default 4 in FP64, 2 in FP32) */
  int32_t dir_low_priority;      /* 1: the low-priority branch (directors, next geometry) at the lowest
                                    stream priority, the rest at the highest (default 1) */
  int32_t geom_blocks_per_sm;    /* grid of the geometry pass beside the repair rounds = SMs x this;
                                    0 = one thread per cell (default) */
  int32_t test_blocks_per_sm;    /* grid of the circumcircle test = SMs x this (default 8), a
                                    grid-stride loop over cells; 0 = one thread per cell */
  int32_t dir_beside_geom;       /* 1: the director terms on a branch of their own, beside the
                                    geometry pass (both FP64; one fills the other's idle FP64
                                    cycles); 0: before it on the same branch (default 1 in FP64,
                                    0 in FP32) */
  int32_t ring_order;            /* bit 0: the geometry pass, bit 1: the force pass, bit 2: the
                                    circumcircle test takes the cells regrouped by ring size within
                                    chunks of 1024 cells, so that the lanes of a warp run the same
                                    number of ring slots (0..7; default 5 in FP64, 0 in FP32) */
  int32_t force_beside;          /* 1: the force pass and the pending move run on the geometry
                                    branch beside the repair rounds, and after the rounds only the
                                    cells around rewritten rings are done again (results
                                    unchanged); 0: after the rounds, all cells (default: the
                                    fix-up after the rounds costs more than the overlap gains,
                                    in FP64 and in FP32 at N = 262144) */
} cg_launch;

/* Workspace size for R replicas. */
int cg_workspace_bytes(int32_t R, const cg_replica* reps, size_t* bytes);

/* Creates a context and triangulates every replica from scratch: each cell's
 * Voronoi polygon is built by clipping with cell-list candidates, which is the
 * GPU counterpart of the paper's CPU repair (Sec. 2.C.4) applied to all cells.
 *   x, y, theta : any, n_total doubles each, replica-concatenated user order;
 *                 positions must lie in [-L, 2L) and are wrapped into [0, L).
 *   d_ws        : device workspace of ws_bytes >= cg_workspace_bytes().
 *   stream      : cudaStream_t (may be 0).
 * Synchronizes the stream; on error *out is NULL. */
int cg_create(int32_t R, const cg_replica* reps, const cg_params* params, const double* x, const double* y,
              const double* theta, void* d_ws, size_t ws_bytes, void* stream, cg_ctx** out);

/* Advances every replica by nsteps time steps (Sec. 2.C: geometry, force
 * sets, net force, move and rotate, circumcircle test, local repair).
 * Asynchronous: enqueues work on the stream and returns.  Steps run as a
 * captured CUDA graph without host synchronization. */
int cg_step(cg_ctx* ctx, int64_t nsteps);

/* nsteps steps (as cg_step) with per-step I/O overlapped with the steps'
 * kernels.  Before step k (0-based) the per-cell v0 of that step is taken
 * from v0 + k*v0_stride (n_total doubles, user order; NULL keeps v0) exactly
 * as cg_set_v0 would set it; after step k the positions are written to
 * x + k*out_stride and y + k*out_stride (n_total doubles each, user order;
 * NULL skips).  Strides count doubles; 0 reuses one buffer for every step.
 * Pointers may be host or device.  Device buffers are read and written by
 * the step's kernels in place; host buffers (page-locked for overlap) go
 * through double-buffered staging in the workspace.  The positions after
 * step k are known before step k's kernels start (they are its pending
 * move), so their download runs on a private stream beside step k; in a
 * call of several steps the upload of step k's v0 runs on another private
 * stream beside step k-1.  The results are bit-identical to
 * cg_set_v0, cg_step(1), cg_get_state per step.  Synchronizes before
 * returning and returns the device status (a non-finite v0 sets CG_EINVAL;
 * the steps after it still run). */
int cg_run_io(cg_ctx* ctx, int64_t nsteps, const double* v0, int64_t v0_stride, double* x, double* y,
              int64_t out_stride);

/* Per-phase device time of nsteps ordinary steps run eagerly (not as a
 * graph), timed with CUDA events on the context's stream.  ms_out[k] receives
 * the summed milliseconds of phase k (n_out >= CG_NUM_PHASES):
 *   0 geometry + force sets, 1 net force + move, 2 circumcircle test,
 *   3 cell-list build, 4 repair rounds (repair + consistency check),
 *   5 director terms of the next step (n(theta) and the noise; in the step
 *     graph this runs beside phases 2-4),
 *   6 ring-size grouping of the cells for the geometry pass (in the step
 *     graph this runs at the end of the previous step, beside the forces).
 * The steps advance the state exactly like cg_step(). */
#define CG_NUM_PHASES 7
int cg_profile_step(cg_ctx* ctx, int64_t nsteps, double* ms_out, int32_t n_out);

/* Waits for the stream and returns the device status word. */
int cg_sync(cg_ctx* ctx);

/* State in user order (any pointers, n_total doubles each; NULL to skip). */
int cg_get_state(cg_ctx* ctx, double* x, double* y, double* theta);
/* Replaces the state and triangulates from scratch (as cg_create). */
int cg_set_state(cg_ctx* ctx, const double* x, const double* y, const double* theta);

/* Cell areas and perimeters at the current state (Sec. 2.C.1). */
int cg_get_geometry(cg_ctx* ctx, double* A, double* P);
/* Forces F = -dE/dr at the current state (Eqs. A6-A16); *energy (host, may
 * be NULL) receives E of Eq. 1 summed over all replicas. */
int cg_get_forces(cg_ctx* ctx, double* Fx, double* Fy, double* energy);
/* Delaunay neighbours: cnt[i] and nbr[i*CG_MAX_RING + a] (cell indices, CCW,
 * starting at the smallest index, -1 padded).  int32 arrays, any pointers. */
int cg_get_neighbors(cg_ctx* ctx, int32_t* cnt, int32_t* nbr);

/* Per-cell target shape index and self-propulsion speed (any pointers). */
int cg_set_p0(cg_ctx* ctx, const double* p0);
int cg_set_v0(cg_ctx* ctx, const double* v0);

int cg_get_counters(cg_ctx* ctx, cg_counters* host_out);

/* Director terms of Eq. 3 as the FP64 step evaluates them (Sec. 2.C.3): for
 * n angles theta[i] and noise keys tag[i] (a cell's global index in the
 * concatenated system) writes cos theta[i], sin theta[i] and the standard
 * normal xi(seed, tag[i], step) of the context's seed (Box-Muller on
 * Philox4x32-10).  Device pointers, n elements each; enqueued on the
 * context's stream without synchronizing.  CG_EINVAL for n < 0 or a NULL
 * pointer with n > 0. */
int cg_director_terms(cg_ctx* ctx, int32_t n, const double* d_theta, const int32_t* d_tag, int64_t step,
                      double* d_cos, double* d_sin, double* d_xi);

/* ---- Differentiation (backward pass) ------------------------------------
 * With the director noise replayed from the seed, one step of Eq. 3 is the
 * map r' = r + dt (mu F(r) + v0 n(theta)) whose transposed Jacobian is
 * I - dt mu H, H the Hessian of E (Eq. 1).  The reverse pass below runs
 * g_t = g_{t+1} - dt mu H(r_t) g_{t+1} over a checkpointed run, with H g
 * computed as a forward-mode derivative of the forces (Eqs. A6-A16) on the
 * frozen topology of each step.  Gradients are exact on windows without
 * neighbour changes.  Cell re-sorting is suspended during these calls.
 * They need a second caller-owned device buffer of cg_backward_bytes(). */

/* Size of the backward buffer for a run of nsteps with a checkpoint every
 * ckpt_every steps (one saved state per checkpoint plus one segment). */
int cg_backward_bytes(const cg_ctx* ctx, int64_t nsteps, int32_t ckpt_every, size_t* bytes);
/* Moduli K_A, K_P (Eq. 1); recaptures the step graph.  Synchronizes. */
int cg_set_moduli(cg_ctx* ctx, double KA, double KP);
/* Sets the Philox step counter (the noise of the next step uses it). */
int cg_set_step(cg_ctx* ctx, int64_t step);

/* ------------------------------------------------------------------------
 * Domain decomposition of one large periodic system (Sec. 4 of the paper
 * names it as the way to larger systems; forces reach the next-nearest
 * neighbours, App. A.2 after Eq. A7, so a domain needs a halo of cells around
 * the cells it owns).  A domain is a context of one replica whose box is a
 * frame of the larger box (a strip plus its halo); the host owns the
 * partition, the exchange and the migration of cells between domains.  With
 * the calls below a domain's own cells evolve exactly (bit for bit) as in the
 * undivided system, provided its cells are passed in increasing global index
 * (the order that breaks ties and starts rings) and its halo is wide enough.
 * ------------------------------------------------------------------------ */
/* Noise counters of the cells: ids (host or device, n int32 >= 0, user order)
 * replace the user index as the cell's Philox counter of Eq. 3's director
 * noise (a domain passes its cells' indices in the undivided system).
 * Recomputes the pending move.  Synchronizes. */
int cg_set_noise_ids(cg_ctx* ctx, const int32_t* ids);
/* Makes replica's box (Lx, Ly of cg_create) the frame with origin (x0, y0) of
 * a larger periodic box (Lx_outer, Ly_outer): positions stay in frame
 * coordinates, and the move of Eq. 3 is formed and rounded in the larger
 * box's coordinates (x0 + x, reduced into [0, Lx_outer)), as the undivided
 * system rounds it.  The larger box must have the same position grid
 * (ceil(log2(max side)) equal), the origin must be a grid point inside it
 * and the frame must fit in it; otherwise CG_EINVAL.  A cell whose move
 * leaves the frame is wrapped into it (only halo cells can; their positions
 * are replaced by the halo exchange).  Recomputes the pending move.
 * Synchronizes. */
int cg_set_frame(cg_ctx* ctx, int32_t replica, double x0, double y0, double Lx_outer, double Ly_outer);
/* Halo exchange, asynchronous on the context's stream.  The values exchanged
 * are the pending positions (where the next step starts) as int64 grid
 * coordinates (units of 2^-q) of the larger box of a framed replica (of the
 * replica's own box otherwise).  d_slot: device, n int32 in user order, the
 * cell's place in the message or -1.  cg_halo_pack writes the listed cells to
 * d_out[2 slot], d_out[2 slot + 1]; cg_halo_unpack replaces the listed cells'
 * pending positions with d_in[2 slot], d_in[2 slot + 1] (a value outside the
 * frame sets the device status to CG_EINVAL and leaves the cell unchanged). */
int cg_halo_pack(cg_ctx* ctx, const int32_t* d_slot, int64_t* d_out);
int cg_halo_unpack(cg_ctx* ctx, const int32_t* d_slot, const int64_t* d_in);
/* nsteps steps from the current state, saving checkpoints into d_bw
 * (device, >= cg_backward_bytes, 256-byte aligned).  Synchronizes. */
int cg_run_checkpointed(cg_ctx* ctx, int64_t nsteps, int32_t ckpt_every, void* d_bw, size_t bytes);
/* Reverse pass of the run saved by cg_run_checkpointed (same nsteps,
 * ckpt_every, d_bw).  Inputs (any pointers, n doubles each, user order):
 * cotangents of the final positions (gxT, gyT), areas (gAT) and perimeters
 * (gPT).  Outputs (any pointers or NULL): cotangents of the initial
 * positions (gx0, gy0), per-cell p0 (gp0) and v0 (gv0), and h_gK[2] (host)
 * for (K_A, K_P).  Leaves the context in the final state.  Synchronizes. */
int cg_backward(cg_ctx* ctx, int64_t nsteps, int32_t ckpt_every, void* d_bw, size_t bytes, const double* gxT,
                const double* gyT, const double* gAT, const double* gPT, double* gx0, double* gy0, double* gp0,
                double* gv0, double* h_gK);
/* H v at the current state, and the derivatives of the areas and perimeters
 * along v (Adot, Pdot; may be NULL).  d_bw: a buffer of at least
 * cg_backward_bytes(ctx, 1, 1).  Any pointers, user order.  Synchronizes. */
int cg_hvp(cg_ctx* ctx, const double* vx, const double* vy, double* hvx, double* hvy, double* Adot, double* Pdot,
           void* d_bw, size_t bytes);

/* Total cells of the context. */
int64_t cg_num_cells(const cg_ctx* ctx);

/* ---- Launch shapes and autotuning -------------------------------------- */
int cg_get_launch(const cg_ctx* ctx, cg_launch* out);
/* Sets the launch shapes and recaptures the step graph.  Synchronizes. */
int cg_set_launch(cg_ctx* ctx, const cg_launch* launch);
/* Scratch needed by cg_autotune: a second workspace, the saved state and an
 * optional L2-flush region of flush_bytes. */
int cg_autotune_bytes(const cg_ctx* ctx, size_t flush_bytes, size_t* bytes);
/* Picks the launch shapes by timing candidates (coordinate descent over the
 * fields of cg_launch, two sweeps; the winner is confirmed against the starting shapes
 * in longer trials) on a temporary copy of the context built in d_ws2
 * (device, >= cg_autotune_bytes(ctx, flush_bytes), 256-byte aligned) from the
 * current state, directors, step counter, p0 and v0: each trial restores that
 * state, runs 2 untimed and steps_per_trial timed graph steps (CUDA events).
 * With flush_bytes > 0 (more than the L2 size, e.g. 256 MB) every timed step
 * starts after a write of that many bytes and is timed alone, as a
 * benchmark with a cold L2 times it.  The context itself takes no step; it gets
 * the fastest shapes (graph recaptured).  best (may be NULL) receives them,
 * best_ms the time per step.  Synchronizes. */
int cg_autotune(cg_ctx* ctx, int32_t steps_per_trial, size_t flush_bytes, void* d_ws2, size_t ws2_bytes,
                cg_launch* best, double* best_ms);

/* Allocation-free triangulation, for callers that cannot call cudaMalloc
 * (code running under a fixed device memory pool, inside another runtime's
 * allocator or plugin hooks, or with all device memory reserved up front).
 * The paper has no counterpart: this is a deployment variant of the
 * from-scratch triangulation that cg_create performs.
 *   n, Lx, Ly   : 16 <= n <= CG_NOALLOC_MAX_CELLS cells in a periodic box;
 *                 any other n, or a box needing more than
 *                 4*CG_NOALLOC_MAX_CELLS cell-list bins (a very elongated
 *                 box), returns CG_EINVAL before any GPU work.
 *   d_x, d_y    : device, n doubles each, positions in [-L, 2L); a position
 *                 outside that range returns CG_EINVAL.
 *   d_cnt, d_nbr: device outputs, n and n*CG_MAX_RING int32: the Delaunay
 *                 neighbours of every cell exactly as cg_get_neighbors()
 *                 returns them for the same positions.
 *   stream      : cudaStream_t (may be 0); the call synchronizes it.
 * Scratch lives in a static device array of the library (about 3.7 MB, held
 * by every GPU that loads the library until the process exits); the call
 * makes no device allocation.  All calls share that array: calls whose GPU
 * work overlaps race.  The first call on each device looks the array's address
 * up and should come before any stream capture.  That address is kept for the
 * life of the process: after a cudaDeviceReset() of a device, do not call
 * this function on that device again.  Returns CG_OK or a status code (the
 * outputs are undefined on error). */
#define CG_NOALLOC_MAX_CELLS 16384
int cg_triangulate_noalloc(int32_t n, double Lx, double Ly, const double* d_x, const double* d_y,
                           int32_t* d_cnt, int32_t* d_nbr, void* stream);

/* ------------------------------------------------------------------------
 * Active vertex model (AVM), Sec. 2.D and Eq. 4 of the paper.
 *
 * The degrees of freedom are the 2N vertices of a degree-3 network; the
 * initial network is the Voronoi tessellation of N seed positions (the
 * circumcentres of their exact periodic Delaunay triangulation).  One step:
 * the energy of Eq. 1 per polygon, the vertex force F_v = -dE/dh_v (Eq. A2
 * with Eqs. A4 and A5), the move dh_v = dt (mu F_v + (1/3) sum over the three
 * cells c of v of v0_c n(theta_c)) (Eq. 4), the director rotation
 * theta_c += sqrt(2 D_r dt) xi (Philox4x32-10, counter (c, step)), then T1
 * passes (Fig. 1) until no edge is shorter than the threshold.
 *
 * Layout (all int32 / double, vertex v, cell c; N = the cell slots, i.e.
 * cell_capacity when one is given, V = 2N vertex slots; slots past the
 * network, and those T2s free, hold empty cells and free vertices):
 *   hx, hy [V]        vertex positions in [0, L)
 *   vc [3V], vn [3V]  cells and neighbours of v, counter-clockwise: the edge
 *                     v - vn[3v+k] separates cells vc[3v+k] and vc[3v+k+1]
 *   cc [N], cv [N*CG_MAX_RING]  vertex count and counter-clockwise vertex
 *                     list of each cell (unused slots -1)
 * Vertex ids of the initial network: the Delaunay triangles owned by their
 * smallest cell, in that cell's ring order, numbered in increasing cell.
 *
 * T1 rule: an edge (v, vn[3v+s]) with v < vn[3v+s] and squared length (each
 * product and the sum rounded separately) below t1_threshold^2 is a
 * candidate with id 3v+s; its cells are i = vc[3v+s], k = vc[3v+s+1] (they
 * share the edge), j = vc[3v+s+2] and l (the third cell of the other end).
 * It needs more than 3 vertices on i and k and fewer than CG_MAX_RING on j
 * and l.  In a pass a candidate applies when its id is the smallest among the
 * candidates touching each of i, j, k, l; the edge is rotated by 90 degrees
 * about its midpoint to length t1_length and i, k lose the edge to j, l.
 * After t1_cap passes with transitions a last pass only counts candidates:
 * any left set CG_ET1_CAP.
 *
 * T2 rule (cell removal; Sec. 2.A names T2 transitions, the paper's code has
 * only T1s): with t2_area > 0, a cell with exactly 3 vertices (v0, v1, v2 its
 * list) and d < 2 t2_area, d = px1 py2 - px2 py1 with p the minimum-image
 * offsets from v0 (each product and the difference rounded separately), is a
 * candidate with id 3V + c in the same passes as the T1s; its cells are c and
 * the three across its edges, which must be distinct with more than 3
 * vertices each (the three outer vertices distinct too); the same lock rule.
 * It keeps the smallest of the three vertex ids at v0 + (p1 + p2)/3 (wrapped),
 * joined to the three outer vertices; the other two are freed (their vc, vn
 * entries -1, positions left as they were) and the cell is emptied (cc = 0,
 * cv = -1).  Freed vertices and empty cells take no part in forces, moves or
 * transitions (an empty cell's A, P are 0; its director still turns).  The
 * preferred perimeter of cell c is P0_c = p0_c sqrt(A0_c) with per-cell
 * preferred areas A0_c (cg_avm_set_a0; all A0 at creation): a cell set to
 * die gets a small A0_c.
 * ------------------------------------------------------------------------ */
typedef struct cg_avm_ctx cg_avm_ctx;

typedef struct cg_avm_params {
  double A0;            /* preferred area */
  double KA, KP;        /* area and perimeter moduli */
  double mu;            /* mobility */
  double Dr;            /* rotational diffusion constant */
  double dt;            /* time step */
  double t1_threshold;  /* edges shorter than this undergo a T1 transition (0: none) */
  double t1_length;     /* length of the rotated edge; 0 = 1.5 t1_threshold */
  uint64_t seed;        /* Philox key of the director noise */
  int32_t t1_cap;       /* T1 passes with transitions per step; 0 = 16 */
  int32_t cell_capacity; /* cell slots, >= N (0: N); divisions fill empty cell
                            slots and free vertex slots, lowest first */
  double t2_area;       /* triangular cells with area below this are removed (T2); 0: none */
  int32_t sort_every;   /* Hilbert re-sort of the vertex and cell storage at creation and every
                           sort_every steps (Sec. 2.B); 0: never.  Results are the same either way */
} cg_avm_params;

/* Workspace size for an N-cell network in an Lx x Ly box. */
int cg_avm_workspace_bytes(int32_t n, double Lx, double Ly, size_t* bytes);
/* The same with room for `capacity` cells (N <= capacity <= 2^26): every
 * per-cell array then has `capacity` entries and every per-vertex array
 * 2 capacity (slots past the network: empty cells, free vertices). */
int cg_avm_workspace_bytes_capacity(int32_t n, int32_t capacity, double Lx, double Ly, size_t* bytes);
/* Builds the Voronoi network of the seeds x, y (n doubles each, host or
 * device, in [-L, 2L), snapped to the position grid as cg_create does) with
 * directors theta, per-cell shape index p0 and speed v0.  d_ws: device,
 * >= cg_avm_workspace_bytes, 256-byte aligned, the caller's until
 * cg_avm_destroy.  stream: cudaStream_t (may be 0).  Synchronizes. */
int cg_avm_create(int32_t n, double Lx, double Ly, double p0, double v0, const cg_avm_params* params,
                  const double* x, const double* y, const double* theta, void* d_ws, size_t ws_bytes, void* stream,
                  cg_avm_ctx** out);
/* Enqueues nsteps steps (one CUDA graph launch each); does not synchronize. */
int cg_avm_step(cg_avm_ctx* ctx, int64_t nsteps);
/* Device time of nsteps ordinary steps run eagerly (not as a graph), timed
 * with CUDA events on the context's stream; the T1 pass control is read back
 * by the host after each pass.  ms_out (n_out >= CG_AVM_NUM_PHASES) receives:
 *   [0] summed ms of the per-cell kernel (geometry, force coefficients),
 *   [1] of the per-vertex kernel (forces, move), [2] of the T1 passes,
 *   [3] the number of T1 passes run, [4] ms of the next step's director
 *   terms (activity and rotation; beside the T1 passes in the step graph).
 * The steps advance the state exactly like cg_avm_step(). */
#define CG_AVM_NUM_PHASES 5
int cg_avm_profile_step(cg_avm_ctx* ctx, int64_t nsteps, double* ms_out, int32_t n_out);
/* Waits for the stream and returns the device status. */
int cg_avm_sync(cg_avm_ctx* ctx);
/* Vertex positions [V] and directors [N]; any pointer may be NULL.  Host or
 * device pointers.  Synchronizes. */
int cg_avm_get_state(cg_avm_ctx* ctx, double* hx, double* hy, double* theta);
/* Network (layout above); any pointer may be NULL.  Synchronizes. */
int cg_avm_get_topology(cg_avm_ctx* ctx, int32_t* vc, int32_t* vn, int32_t* cc, int32_t* cv);
/* Replaces positions (required) and, where not NULL, directors and network
 * arrays, which must describe a valid network of the same N (cell slots).
 * Synchronizes. */
int cg_avm_set_state(cg_avm_ctx* ctx, const double* hx, const double* hy, const double* theta, const int32_t* vc,
                     const int32_t* vn, const int32_t* cc, const int32_t* cv);
/* Per-cell p0, v0 and A0 [N] as they stand (divisions copy them to the new
 * cells); any pointer may be NULL.  Host or device pointers.  Synchronizes. */
int cg_avm_get_cell_params(cg_avm_ctx* ctx, double* p0, double* v0, double* a0);
/* Sets the Philox step counter (the director noise of the next step uses it);
 * with cg_avm_get_state/_topology/_cell_params it resumes a run.
 * Synchronizes. */
int cg_avm_set_step(cg_avm_ctx* ctx, int64_t step);
/* Polygon areas and perimeters [N] of the current state.  Synchronizes. */
int cg_avm_get_geometry(cg_avm_ctx* ctx, double* A, double* P);
/* Vertex forces [V] and, if energy != NULL, the total energy of Eq. 1.
 * Synchronizes. */
int cg_avm_get_forces(cg_avm_ctx* ctx, double* Fx, double* Fy, double* energy);
/* Transition passes (T1, and T2 when t2_area > 0) on the current state,
 * without a move.  Synchronizes. */
int cg_avm_t1(cg_avm_ctx* ctx);
/* Per-cell shape index and speed, N doubles (host or device).  Synchronizes. */
int cg_avm_set_p0(cg_avm_ctx* ctx, const double* p0);
int cg_avm_set_v0(cg_avm_ctx* ctx, const double* v0);
/* Cell divisions (Sec. 2.A lists division among the features vertex models
 * add; the paper's code has none), made one after the other: division k cuts
 * cell cells[k] along the direction (dirs[2k], dirs[2k+1]) through the mean
 * of its vertices.  With p the minimum-image offsets of its vertices from
 * the first one, m their mean (sum in list order, then / count), q = p - m
 * and s = u x q, an edge a -> a+1 is cut where s changes sign (s > 0 against
 * s <= 0) at X = q_a + t (q_{a+1} - q_a), t = s_a / (s_a - s_{a+1}) clamped
 * to [1/16, 15/16]; the cut with the smallest u.X > 0 gives new vertex A
 * (edge a1), the one with the largest u.X < 0 new vertex B (edge a2); every
 * product, sum and quotient is rounded on its own.  The cell keeps A,
 * v_{a1+1} .. v_{a2}, B; the lowest empty cell slot (cc = 0: never used, or
 * emptied by a T2) takes B, v_{a2+1} .. v_{a1}, A and copies the cell's
 * director, p0, v0 and A0; A and B take the two lowest free vertex slots
 * (vc = -1); the cells across the cut edges gain them.  A division
 * with a missing cut, or that would give a cell more than CG_MAX_RING
 * vertices, is not made (made[k] = 0).  cells [count] int32 and dirs
 * [2 count] doubles: host or device; made [count] (NULL to skip) and
 * *n_made (host, may be NULL) receive the outcome.  CG_EINVAL when fewer
 * than count cell slots (2 count vertex slots) are free, a cell index is
 * out of range or a direction is not finite.  Synchronizes. */
int cg_avm_divide(cg_avm_ctx* ctx, int32_t count, const int32_t* cells, const double* dirs, int32_t* made,
                  int32_t* n_made);
/* Per-cell preferred areas A0_c >= 0 (Eq. 1), N doubles (host or device);
 * a negative or non-finite entry returns CG_EINVAL.  Synchronizes. */
int cg_avm_set_a0(cg_avm_ctx* ctx, const double* a0);
/* Counters: steps, repaired_total = T1 transitions made, flagged_total = T2
 * transitions made, last_rounds = transition passes that ran (all since
 * creation), status. */
int cg_avm_get_counters(cg_avm_ctx* ctx, cg_counters* host_out);
/* Releases the host context (the workspace stays the caller's). */
int cg_avm_destroy(cg_avm_ctx* ctx);
const char* cg_avm_last_error(const cg_avm_ctx* ctx);
/* Storage order (Sec. 2.B: spatially close vertices and cells close in
 * memory).  The ids of this API (vertex and cell ids, the entries of vc, vn,
 * cv, the order of every per-vertex and per-cell array, the cells of
 * cg_avm_divide) are tags fixed when a vertex or cell slot comes into being;
 * where each one is stored is the context's business.  Every rule above that
 * depends on ids (T1 and T2 priorities, the end a T1 edge is taken from, the
 * vertex a T2 keeps, the director noise counter, the slots divisions fill)
 * uses the tags, so results do not depend on the storage order.
 * cg_avm_sort re-sorts now: vertices along a Hilbert curve of their
 * positions, cells along one of their first vertices', freed vertices and
 * empty cells last.  Enqueued on the context's stream; synchronizes. */
int cg_avm_sort(cg_avm_ctx* ctx);
/* The tag held by each vertex slot [V] and cell slot [N] (host or device
 * pointers, either may be NULL): a diagnostic of the storage order.
 * Synchronizes. */
int cg_avm_get_tags(cg_avm_ctx* ctx, int32_t* vtag, int32_t* ctag);

/* Releases the host context (the workspace stays the caller's). */
int cg_destroy(cg_ctx* ctx);

/* Static description of a status code. */
const char* cg_status_string(int status);
/* Last error message of a context (static lifetime within the context). */
const char* cg_last_error(const cg_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* CELLGB_H */
