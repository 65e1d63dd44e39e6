/*
 * bfgpu.h -- C ABI of the GB300 (sm_103a) library for the generalized
 * Bellman-Ford method of symbolic optimal control
 * (Weber, Kreuzer, Knoll, arXiv 2001.06231).
 *
 * The library solves optimal control problems (X, U, F, G, g) of Def. ocp
 * (Sec. III-C) whose system (X, U, F) is a discrete abstraction of a sampled
 * system (Def. abstraction, Sec. V-A/V-B): X is a uniform grid of
 * hyper-rectangular cells, U a finite input set, and F(x,u) an integer box of
 * cells (the cells that meet a box over-approximation of the attainable set).
 * It computes the value function V of Eq. (valuefunction) and a controller mu
 * realizing it with Algorithm 1 (generalized Bellman-Ford-Yen), on one GPU.
 *
 * Conventions shared by every call
 *   - Cells: D <= 4 dimensions, n[d] cells each (n[d] <= 16383), cell index
 *     c = i0 + n0*(i1 + n1*(i2 + n2*i3)) (dim 0 fastest).  A periodic
 *     dimension wraps (index n[d] is index 0).
 *   - Boxes (external layout): int16 [C][U][2][D] -- lo[0..D-1] then
 *     hi[0..D-1].  F(x,u) = { y : lo_d <= y_d <= hi_d for all d }; on a
 *     periodic dim hi may exceed n-1 (at most lo + n - 1) and indices wrap.
 *     lo[0] == BF_BLOCKED marks a pair whose image leaves the grid: its
 *     successor is the overflow set of the cover (Sec. V-B), value +inf.
 *   - Costs: G is double [C][U]: the running cost g(x,y,u) = G(x,u) for every
 *     successor y (Eq. cost with g independent of y).  +inf is allowed (an
 *     unusable input); NaN, -inf and finite |G| > 2^64 are rejected.  -0.0 is
 *     read as +0.0.  The terminal cost of Eq. (cost) is 0 on target cells and
 *     +inf elsewhere, or an explicit double [C] array (bf_solve_opts).
 *   - Avoid cells: g(x,.,.) = g(.,x,.) = +inf and terminal +inf, so V = +inf
 *     there and any box touching one yields +inf.
 *   - Output: V double [C]; mu uint8 [C] with BF_HANDOVER (0xFF) meaning
 *     "mu(x) = U", i.e. hand over control (Ex. ex:algorithm); iters = number
 *     of passes of Algorithm 1's while-loop; status BF_CONVERGED (F1 empty:
 *     V is the value function, Thm. BellmanFord), BF_NEG_CYCLE (the |X| cap
 *     of the while-loop was reached: negative-cycle test) or BF_ITER_CAP
 *     (a smaller caller cap was reached).
 *   - Rounds are synchronous (Jacobi): every relaxation of a pass reads V as
 *     it stood when the pass began; mu(x) changes only on a strict decrease
 *     and takes the lowest input index among equal minima.  V, mu, iters and
 *     status are therefore deterministic.
 *   - Pointers: unless stated otherwise, an array argument may be host memory
 *     or device memory of the current device (detected with
 *     cudaPointerGetAttributes).  The caller owns every buffer it passes and
 *     keeps it alive until the call returns; library-owned objects
 *     (abstractions, servers) are freed only by abs_free / bf_serve_close.
 *   - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *     Calls returning results in host memory synchronize that stream.
 *   - Errors: every int-returning call returns BF_OK (0) or a negative
 *     BF_ERR_* code and sets a thread-local message (bf_last_error).  No C++
 *     exception crosses this boundary.
 */
#ifndef BFGPU_H
#define BFGPU_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define BF_API __attribute__((visibility("default")))
#else
#define BF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define BF_OK 0
#define BF_ERR_INVALID (-1)      /* bad argument, malformed box, NaN cost   */
#define BF_ERR_OOM (-2)          /* device allocation failed / over budget  */
#define BF_ERR_CUDA (-3)         /* a CUDA runtime call failed              */
#define BF_ERR_TIMEOUT (-4)      /* a bounded device wait gave up           */
#define BF_ERR_UNSUPPORTED (-5)  /* valid but not supported by this build   */

#define BF_CONVERGED 0
#define BF_NEG_CYCLE 1
#define BF_ITER_CAP 2

#define BF_HANDOVER 0xFF
#define BF_BLOCKED (-32768)

/* Built-in sampled systems (Sec. V, Eq. ode).  Parameters in bf_dynamics.param:
 *   BF_DYN_LINEAR2D   double integrator x0' = x1, x1' = u0; exact linear flow
 *                     of the cell corners (no parameters).
 *   BF_DYN_UNICYCLE3D x' = v cos th, y' = v sin th, th' = w; u = (v, w);
 *                     param[0] = disturbance bound (added to every component).
 *   BF_DYN_FIRE4D     x' = V cos psi + param[0], y' = V sin psi,
 *                     psi' = (param[1] / V) tan(phi), V' = a; u = (phi, a);
 *                     param[2], param[3] = lower / upper speed bound used in
 *                     the Jacobian bound; param[4] = disturbance bound.
 * UNICYCLE3D and FIRE4D boxes are centre +- growth bound: the classical RK4
 * scheme (rk4_substeps equal steps) applied to x' = f(x,u) from the cell
 * centre and to r' = L r + w from r(0) = eta/2 (Sec. V-B, box
 * over-approximation of attainable sets).  Cells meeting [a, b] on dim d are
 * floor((a - lo_d)/eta_d) .. floor((b - lo_d)/eta_d). */
#define BF_DYN_LINEAR2D 1
#define BF_DYN_UNICYCLE3D 2
#define BF_DYN_FIRE4D 3

/* Storage mode of an abstraction (Sec. IV-B, memory control): STORED keeps the
 * image of F in device memory; RECOMPUTE keeps only the dynamics and
 * regenerates each box inside the relaxation kernel (bit-identical boxes,
 * 4*D*C*U fewer bytes, far more FP64 work). */
#define BF_MODE_STORED 0
#define BF_MODE_RECOMPUTE 1
#define BF_MODE_HYBRID 2       /* records of the first K inputs stored, the
                                  rest regenerated (abs_build_hybrid)       */

typedef struct {
    int32_t ndim;          /* D, 1..4                                   */
    int32_t n[4];          /* cells per dimension                       */
    double lo[4], hi[4];   /* grid extent: cell k of dim d spans
                              [lo + k*eta, lo + (k+1)*eta], eta=(hi-lo)/n */
    uint8_t periodic[4];   /* nonzero: the dimension wraps              */
} bf_grid;

typedef struct {
    int32_t ninputs;       /* |U'|, 1..254                              */
    int32_t udim;          /* components per input                      */
    const double *u;       /* host, row-major [ninputs][udim]           */
} bf_inputs;

typedef struct {
    int32_t kind;          /* BF_DYN_*                                  */
    int32_t rk4_substeps;  /* RK4 steps per sampling period (>= 1)      */
    double param[8];
} bf_dynamics;

typedef struct bf_abstraction bf_abstraction;   /* opaque, device-resident */

/* abs_build -- discrete abstraction of the sampled system (dyn, tau) on grid
 * with the given inputs (Def. abstraction, Sec. V-B).  Writes, per (cell,
 * input), the int16 successor box on the device, then the predecessor index
 * (a per-cell bounding box of pred(y) = {x : y in F(x,u) for some u}, a
 * superset of Eq. pred, which Sec. V-B allows).  mode = BF_MODE_STORED or
 * BF_MODE_RECOMPUTE.  On success *out owns all device memory (abs_free).
 * Errors: BF_ERR_INVALID (grid/inputs/dyn out of range), BF_ERR_OOM,
 * BF_ERR_CUDA. */
BF_API int abs_build(const bf_dynamics *dyn, const bf_grid *grid, const bf_inputs *inputs,
              double tau, int32_t mode, void *stream, bf_abstraction **out);

/* abs_build_hybrid -- the memory regulation of Sec. IV-B between the two modes
 * above: store the images of F while memory allows, recompute the rest.  The
 * box records of the first K inputs are stored, K the most inputs whose
 * compact records (4 bytes per (cell, input) for D <= 2, 8 for D >= 3) fit
 * in box_budget bytes; the boxes of the other inputs are regenerated inside
 * the relaxation kernel.  K = U gives a stored-mode abstraction, K = 0 (or a
 * system whose boxes do not fit the compact records) a recompute-mode one;
 * otherwise the mode is BF_MODE_HYBRID.  (The transitions of the other
 * inputs that the next round needs can be kept per solve: the frontier cache
 * of bf_solve_opts.)  Boxes, and so every result, are bit-identical to the
 * other modes.  The predecessor index and the inputs
 * are not counted in box_budget.  Errors: as abs_build, and BF_ERR_INVALID
 * for a negative budget. */
BF_API int abs_build_hybrid(const bf_dynamics *dyn, const bf_grid *grid, const bf_inputs *inputs,
              double tau, int64_t box_budget, void *stream, bf_abstraction **out);

/* abs_stored_inputs -- K, the inputs whose box records are stored (U in
 * stored mode, 0 in recompute mode).  Errors: BF_ERR_INVALID on NULL. */
BF_API int abs_stored_inputs(const bf_abstraction *abs, int32_t *nstored);

/* abs_from_boxes -- abstraction from caller-supplied boxes in the external
 * layout int16 [C][U][2][D] (host or device).  Every box is validated on the
 * device (0 <= lo <= hi <= n-1, or hi <= lo + n - 1 on a periodic dim, or
 * blocked); any malformed box gives BF_ERR_INVALID.  Always STORED mode. */
BF_API int abs_from_boxes(const bf_grid *grid, int32_t ninputs, const int16_t *boxes,
                   void *stream, bf_abstraction **out);

/* abs_export_boxes -- write the abstraction's boxes to out (int16
 * [C][U][2][D], host or device).  In RECOMPUTE mode the boxes are generated
 * by the same device code the solver uses. */
BF_API int abs_export_boxes(const bf_abstraction *abs, int16_t *out, void *stream);

/* abs_export_pred -- write the predecessor index to out (int16 [C][2][D]):
 * offsets lo then hi, x in pred(y) only if y + lo <= x <= y + hi per dim (on a
 * periodic dim the offsets are taken mod n).  lo[0] > hi[0] = empty. */
BF_API int abs_export_pred(const bf_abstraction *abs, int16_t *out, void *stream);

/* abs_info -- sizes of an abstraction; any out pointer may be NULL.
 * box_record_bytes: bytes per stored (cell, input) box -- 4 or 8 for the
 * compact relative records (per dim an 8-bit offset from the cell and an
 * 8-bit width; used whenever every box fits), 4*D for 16-bit absolute
 * records, 0 in RECOMPUTE mode. */
BF_API int abs_info(const bf_abstraction *abs, int64_t *ncells, int32_t *ninputs,
             int32_t *ndim, int32_t *mode, int64_t *device_bytes, int32_t *box_record_bytes);

/* abs_shape_info -- the plane shape table of an abstraction (stored compact
 * records on a grid of 2+ dims whose dims 0 and 1 are not periodic).  A plane
 * is the set of cells with equal coordinates on dims >= 2; for dynamics that
 * do not depend on the coordinates of dims 0 and 1 (Def. abstraction, built
 * from one flow for every cell: the unicycle and fire models) all non-blocked
 * boxes of a plane and input have the same relative record.  *nplanes = the
 * number of planes (0: no table), *mismatch = the non-blocked boxes whose
 * record differs from their plane's entry (they are gathered cell by cell).
 * Either out pointer may be NULL. */
BF_API int abs_shape_info(const bf_abstraction *abs, int64_t *nplanes, int64_t *mismatch);

/* abs_free -- release an abstraction (NULL is a no-op).  The caller must not
 * free it while a solve on it is running. */
BF_API void abs_free(bf_abstraction *abs);

/* Pass schedules (bf_solve_opts.schedule).
 * BF_SCHED_JACOBI (default): every relaxation of a pass reads W as it stood at
 *   the start of the pass; V, mu, the pass count and every per-pass frontier
 *   are deterministic (and equal to the CPU oracle's).
 * BF_SCHED_INPLACE: a decrease of W(x) is written at once, so relaxations later
 *   in the same pass may read it -- the in-place writes of Alg. 1's for-loop,
 *   whose processing order the paper leaves open (Sec. IV-A).  Every update is
 *   W <- min(W, G + max W) with a monotone operator, so a run that stops with
 *   F1 empty reaches the same V (the greatest fixed point below the terminal
 *   cost), usually in fewer passes; mu is a controller realizing V (Thm. 2's
 *   construction) but not necessarily the Jacobi one, and the pass count,
 *   trace and exact-F1 counts depend on the order warps run in. */
#define BF_SCHED_JACOBI 0
#define BF_SCHED_AUTO 0
#define BF_SCHED_INPLACE 1

#define BF_FLAG_HOST_LOOP 1    /* drive passes from the host (one sync per pass) */
#define BF_FLAG_COUNT_EXACT 2  /* also count |F1| of Algorithm 1 with the exact
                                  pred of Eq. (pred) (extra gather per pair)    */
#define BF_FLAG_TIME_KERNELS 4 /* host-driven passes with a CUDA event pair
                                  around every relax and propagate launch       */

/* Statistics of one bf_solve call (all optional outputs). */
typedef struct {
    int64_t kernel_launches;   /* kernels of this library the call launched      */
    int64_t relaxed_cells;     /* sum over passes of cells relaxed (the frontier
                                  flagged through predecessor bounding boxes:
                                  a superset of the exact F1)                    */
    int64_t executed_pairs;    /* relaxed_cells * U                              */
    int64_t exact_f1_cells;    /* sum over passes of |F1| with exact pred (only
                                  with BF_FLAG_COUNT_EXACT, else -1)             */
    int64_t changed_cells;     /* sum over passes of cells whose V decreased    */
    int64_t relax_launches;    /* relax kernels launched                         */
    double relax_ms;           /* summed relax kernel time (BF_FLAG_TIME_KERNELS) */
    double propagate_ms;       /* summed time of the pass kernel after relax
                                  (commit, compaction; the predecessor marking
                                  of Alg. 1's F2 line runs inside relax)        */
} bf_solve_stats;

typedef struct {
    int64_t max_iters;         /* 0 -> |X| (the paper's cap); else min(., |X|) */
    int32_t schedule;          /* BF_SCHED_*                                    */
    int32_t flags;             /* BF_FLAG_*                                     */
    const double *terminal;    /* optional [C] terminal cost (host or device);
                                  NULL -> 0 on target cells, +inf elsewhere     */
    int64_t *trace;            /* optional host [trace_cap][4]: per pass cells
                                  relaxed, cells changed, relax chunks (32
                                  frontier cells each), and exact |F1|
                                  (BF_FLAG_COUNT_EXACT, else -1)                  */
    int64_t trace_cap;
    bf_solve_stats *stats;     /* optional output                               */
    /* Optional successor class (Sec. VI-A, g2: a running cost that depends on
     * the successor): g(x,y,u) = G_class(x,u) when succ_class[y] != 0, G(x,u)
     * otherwise.  Both host or device; NULL succ_class = no class.  G_class
     * follows G's layout and rules ([C][U] double). */
    const uint8_t *succ_class; /* [C]                                           */
    const double *G_class;     /* [C][U]                                        */
    /* Frontier cache (Sec. IV-B memory regulation: after each round keep only
     * the transitions the next round needs), for abstractions whose boxes are
     * regenerated (recompute mode, or the inputs a hybrid abstraction does not
     * store): the regenerated records of the first frontier_cache cells of each
     * pass's frontier are kept for the next pass, where the cells still in the
     * frontier read them instead of regenerating them; the others are dropped.
     * Device memory in the handle's workspace: 8 C + 16 (U - K) frontier_cache
     * bytes.  0: no cache (stored-mode abstractions never use one). */
    int64_t frontier_cache;
} bf_solve_opts;

/* bf_solve -- Algorithm 1 (Sec. IV-A) on the abstraction with running cost G
 * ([C][U] double), target ([C] uint8, nonzero = terminal cost 0; ignored when
 * opts->terminal is set) and avoid ([C] uint8 or NULL).  Writes V ([C]
 * double), mu ([C] uint8), *iters and *status (host pointers for the last
 * two).  V and mu may be host or device.  opts may be NULL.  One solve at a
 * time per abstraction handle (they share its workspace).
 * Errors: BF_ERR_INVALID (NaN / -inf / too large costs, bad sizes),
 * BF_ERR_OOM, BF_ERR_CUDA. */
BF_API int bf_solve(const bf_abstraction *abs, const double *G, const uint8_t *target,
             const uint8_t *avoid, const bf_solve_opts *opts, double *V, uint8_t *mu,
             int64_t *iters, int32_t *status, void *stream);

/* bf_tune -- pick the pass schedule of this abstraction's solves by timing
 * (one schedule dimension at a time, keeping the others at the best found so
 * far, over two rounds):
 * the slice target (inputs of a small frontier's chunks split over warps when
 * the frontier has fewer chunks than slice_target x warps; 0 = never),
 * whether relax marks the next frontier itself or a propagate launch does,
 * the relax grid (one or half a wave) and, on grids of 2 or more dims,
 * whether boxes at least 3 cells wide on dims 0 and 1 read a table of 3 x 3
 * window maxima (fewer gathers, more table upkeep per changed cell; not
 * with a successor class) and, where the abstraction has a plane shape table
 * (stored compact records on 2+ dims, dims 0 and 1 not periodic: the cells
 * with equal coordinates on dims >= 2 share each input's relative box), whether
 * a warp whose cells lie on one plane reads that plane's precomputed lookup
 * offsets instead of decoding each box, and whether the next frontier is
 * marked from the planes' predecessor templates (the rows of pred(y) of Eq.
 * (pred) for every cell y of a plane, when every box of a plane and input is
 * the plane's entry) instead of the per-cell bounding boxes of pred, and
 * (with the lookup lists) whether relax takes two inputs per iteration,
 * runs one block per SM more (occupancy) and reads the per-cell input masks
 * (cell_masks), on grids of 3+ dims with the 3 x 3 windows along which dim >= 2
 * a plane-pair table halves the lookups (pair_dim), whether (with the
 * templates) the next frontier is kept per input (input_frontier), and
 * from which frontier size (share of the cells) a pass relaxes by tiles
 * staged in shared memory (dense_pct; abstractions with a plane shape table
 * and an even dim 0 of at most 256 cells); two whole schedules of the
 * pair-queue relax are timed before the descent starts from the best.  Each
 * candidate is solved five times (one warm, four timed) on the given inputs (G, target, avoid and the
 * optional terminal / succ_class / G_class / max_iters of opts; flags, trace
 * and stats are ignored); the fastest stays in force for later bf_solve calls
 * on the handle.  Results never depend on the schedule.  Errors: as bf_solve. */
typedef struct {
    int32_t slice_target;
    int32_t fuse_mark;         /* 1: relax marks the next frontier                */
    int32_t relax_blocks;
    int32_t candidates;        /* schedules timed (the default included)          */
    double best_ms;            /* mean solve time of the chosen schedule          */
    double default_ms;         /* the same for the default schedule               */
    int32_t window33;          /* 1: the 3 x 3 window table is used               */
    int32_t plane_lists;       /* 1: warps whose cells share a plane read that
                                  plane's precomputed lookup lists              */
    int32_t templates;         /* 1: the next frontier is marked from the
                                  planes' predecessor templates                 */
    int32_t pair_inputs;       /* 1: with plane lookup lists, relax takes two
                                  inputs per iteration (both gathers in flight) */
    int32_t dense_pct;         /* passes whose F1 holds at least this percentage
                                  of the cells relax by tiles: a block per plane
                                  and band of rows, the window-table cells of its
                                  boxes copied to shared memory by TMA; 0: never */
    int32_t occupancy;         /* 1: the plane relax kernel runs one block per SM
                                  more than its registers want (some spills)    */
    int32_t cell_masks;        /* 1 or 2: with plane lookup lists, relax reads
                                  one 8-byte word per cell saying which inputs
                                  have the plane's record (their lists apply)
                                  and which another (their records are read);
                                  no record is read for the first kind and no
                                  cost for blocked pairs.  1: the inputs in
                                  turn, pair_inputs ? 4 : 2 per iteration; 2:
                                  the pairs queued over the lanes, input by
                                  input, pair_inputs ? 2 : 1 per lane and round
                                  (only the pairs a cell holds cost work)       */
    int32_t pair_dim;          /* 2 .. D - 1: with the 3 x 3 window table, a
                                  second table holds the maximum of two of its
                                  entries one step apart on this dim, and boxes
                                  spanning 2+ planes on it read that (half the
                                  lookups along it, more table upkeep per
                                  changed cell); 0: none                        */
    int32_t input_frontier;    /* 1: with the predecessor templates, the next
                                  frontier is kept per input (one bitmap per
                                  input, marked from per-input templates) and
                                  relax with cell_masks takes up only the pairs
                                  (x, u) whose own box holds a cell changed in
                                  the previous pass: a pair whose box did not
                                  change cannot lower W(x), so results are the
                                  same                                          */
} bf_tune_result;

BF_API int bf_tune(const bf_abstraction *abs, const double *G, const uint8_t *target,
             const uint8_t *avoid, const bf_solve_opts *opts, bf_tune_result *out, void *stream);

/* bf_set_schedule -- put a pass schedule in force without timing (a schedule
 * bf_tune printed earlier, or a fixed one): slice_target 0..4, fuse_mark,
 * relax_blocks (<= 0 or above one wave: one wave), window33, plane_lists,
 * templates, pair_inputs, occupancy, cell_masks, pair_dim (0 or 2 .. D - 1;
 * without effect unless window33 and plane_lists are on), input_frontier
 * (without effect unless templates are on and U <= 32) and dense_pct
 * (0..100; ignored where the tile form does not apply) of *sched are read, the
 * rest ignored; window33 has no effect on
 * 1-D grids or solves with a successor class, plane_lists none on
 * abstractions without a plane shape table or solves with a successor class,
 * templates none on abstractions without templates.  Results never depend on the schedule.  Returns BF_OK,
 * BF_ERR_INVALID (NULL argument, slice_target or pair_dim out of range) or BF_ERR_CUDA /
 * BF_ERR_OOM (the handle's solve workspace could not be set up). */
BF_API int bf_set_schedule(const bf_abstraction *abs, const bf_tune_result *sched, void *stream);

/* bf_solve_batch -- n independent instances of bf_solve (possibly on
 * different abstractions of uneven size), advanced together: every device
 * step relaxes the frontiers of all unfinished instances in one launch.
 * Arrays of n pointers (host arrays of pointers; the pointed-to buffers as in
 * bf_solve).  avoid[i] may be NULL; terminal may be NULL or hold NULLs.
 * Results are identical to n separate bf_solve calls. */
BF_API int bf_solve_batch(int32_t n, const bf_abstraction *const *abs, const double *const *G,
                   const uint8_t *const *target, const uint8_t *const *avoid,
                   const double *const *terminal, int64_t max_iters,
                   double *const *V, uint8_t *const *mu, int64_t *iters, int32_t *status,
                   void *stream);

/* bf_tune_batch -- pick the batched form's schedule by timing whole
 * bf_solve_batch calls on these instances (arguments as bf_solve_batch, no
 * result arrays): whether relax marks the next frontier itself, the 3 x 3
 * window table, the plane lookup lists, the predecessor templates, two
 * inputs per relax iteration and the relax by cell masks with the pairs queued
 * over the lanes (one at a time, keeping the others at the best so far, two
 * rounds; each candidate solved three times).  The fastest schedule
 * is stored in every given abstraction and used by later bf_solve_batch calls
 * and by the server's engine (a group of instances that share a dimension and
 * storage form takes the schedule of its first instance).  In *out: fuse_mark
 * (-1: by predecessor-box size, the default), window33, plane_lists,
 * templates, pair_inputs, cell_masks (0 or 2), candidates, best_ms and
 * default_ms; the other fields are 0.  Results never depend on the schedule.  Errors: as bf_solve_batch. */
BF_API int bf_tune_batch(int32_t n, const bf_abstraction *const *abs, const double *const *G,
                  const uint8_t *const *target, const uint8_t *const *avoid,
                  const double *const *terminal, int64_t max_iters, bf_tune_result *out, void *stream);

/* bf_set_batch_schedule -- put a batched-form schedule in force on an
 * abstraction without timing: fuse_mark (-1: relax marks when the
 * predecessor boxes are small, 0: a propagate launch, 1: relax marks),
 * window33, plane_lists, templates, pair_inputs and cell_masks (nonzero: the
 * pair-queue relax) of *sched are read.  The
 * handle is modified; it must not be in use by a running batch or server.
 * Results never depend on the schedule.  Returns BF_OK or BF_ERR_INVALID. */
BF_API int bf_set_batch_schedule(bf_abstraction *abs, const bf_tune_result *sched);

/* Server: continuous batching of solve requests (the served form of the
 * solver).  A server owns one engine thread and one stream.  Requests are
 * admitted in arrival order while the device-memory budget and the slot count
 * allow; the engine advances every admitted request together (a bounded
 * number of passes per engine step, as in bf_solve_batch), and between steps
 * retires finished requests (results copied to the request's host buffers)
 * and admits waiting ones, so requests that arrive while others are on the
 * GPU join them.  Each result is identical to a solo bf_solve.
 *
 * A request names either a resident abstraction (abs, kept alive by the
 * caller) or a system (dyn, grid, inputs, tau); the server keeps the
 * abstractions it builds resident and reuses them for later requests with
 * the same system (compared field by field).  A new abstraction is built in
 * STORED mode when its boxes fit the remaining budget, else in HYBRID mode
 * with the records of as many inputs as the rest of the budget holds (see
 * abs_build_hybrid), else in RECOMPUTE mode (the memory control of
 * Sec. IV-B); bf_result.mode reports which. */
typedef struct bf_server bf_server;

typedef struct {
    const bf_abstraction *abs;   /* resident abstraction, or NULL: use dyn/grid/inputs/tau */
    const bf_dynamics *dyn;      /* system of the request when abs == NULL (copied)      */
    const bf_grid *grid;
    const bf_inputs *inputs;
    double tau;
    const double *G;             /* host [C][U], copied at submit                         */
    const uint8_t *target;       /* host [C] or NULL when terminal is given               */
    const uint8_t *avoid;        /* host [C] or NULL                                      */
    const double *terminal;      /* host [C] or NULL                                      */
    int64_t max_iters;
    double *V;                   /* host [C] destination, written before done = 1        */
    uint8_t *mu;                 /* host [C] destination                                  */
    int32_t flags;               /* BF_REQ_*                                              */
} bf_request;

/* The caller keeps G, target, avoid and terminal unchanged and alive until the
 * request is done, so bf_serve_submit does not copy them (pinned host buffers
 * then go to the device by DMA without an extra host copy). */
#define BF_REQ_BORROW_INPUTS 1

typedef struct {
    int32_t done;                /* 1 when V/mu/iters/status are final                    */
    int32_t status;              /* BF_CONVERGED / BF_NEG_CYCLE / BF_ITER_CAP             */
    int64_t iters;
    int32_t error;               /* BF_OK or the error of this request                    */
    int32_t mode;                /* storage mode of the abstraction used                  */
    double submit_s, admit_s, finish_s;   /* steady-clock seconds                         */
} bf_result;

/* bf_serve_open -- start a server.  hbm_budget: device bytes the server may
 * use for the abstractions it builds plus per-request state; max_active: most
 * requests on the device at once; passes_per_step: passes per engine step (0
 * -> 8).  Errors: BF_ERR_INVALID, BF_ERR_CUDA. */
BF_API int bf_serve_open(size_t hbm_budget, int32_t max_active, int32_t passes_per_step,
                         bf_server **out);
/* bf_serve_submit -- enqueue a request (host inputs copied); *id identifies
 * it.  A request that can never fit the budget completes with BF_ERR_OOM. */
BF_API int bf_serve_submit(bf_server *srv, const bf_request *req, uint64_t *id);
/* bf_serve_poll -- state of request id; wait != 0 blocks until it is done.
 * A done request is forgotten after it was polled done once. */
BF_API int bf_serve_poll(bf_server *srv, uint64_t id, int32_t wait, bf_result *out);
/* bf_serve_close -- finish every submitted request, stop the engine thread,
 * free the server and the abstractions it built. */
BF_API void bf_serve_close(bf_server *srv);

/* bf_last_error -- message of the last failed call on this thread. */
BF_API const char *bf_last_error(void);

/* bf_solve_noalloc -- the same solve as bf_solve, for callers that must not
 * have the library allocate device memory.  The paper has no counterpart: it
 * exists for host programs that hand out all device memory themselves (a
 * fixed budget carved up at start-up, a memory pool they own, a long-running
 * loop that may not call cudaMalloc/cudaFree once it runs), where a solver
 * that allocates its own workspace, or that stages host arrays through
 * temporary device buffers, cannot be used.
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine.  Its working
 * state (values, frontier bitmap and lists, the transposed cost array,
 * counters) lives in one file-scope device array of BF_NOALLOC_SCRATCH_BYTES
 * bytes that every GPU which loads the library holds until the process
 * exits.  An instance needing more than that (about 40 + 8*U bytes per cell:
 * four int64 value and window arrays, two int32 cell lists, the frontier
 * bitmap and the transposed FP64 costs) is rejected with BF_ERR_INVALID and a
 * message giving the size it would need.
 *
 * Every array argument must be device memory of the current device (host
 * pointers are rejected with BF_ERR_INVALID, since copying them would need a
 * staging buffer): G [C][U], target [C] (ignored when terminal != NULL),
 * avoid [C] or NULL, terminal [C] or NULL, V [C] and mu [C] as outputs.
 * iters and status are host pointers.  max_iters as in bf_solve_opts.
 * Results are identical to bf_solve.
 *
 * The first call on a device looks up the device address of the scratch
 * array (cudaGetSymbolAddress) and caches it for the life of the process;
 * make that first call before any stream capture, and do not call it on a
 * device after cudaDeviceReset there (the cached address would be stale).
 * The call drives the passes from the host: it reads the pass counters back
 * and synchronizes the stream before it returns.  All calls share the one
 * array and it keeps the last call's contents (each call clears what must
 * start at zero), so calls that may overlap on the GPU -- on different
 * streams, or from different host threads -- race and must be serialized by
 * the caller. */
#define BF_NOALLOC_SCRATCH_BYTES (32u << 20)
BF_API int bf_solve_noalloc(const bf_abstraction *abs, const double *G, const uint8_t *target,
                            const uint8_t *avoid, const double *terminal, int64_t max_iters,
                            double *V, uint8_t *mu, int64_t *iters, int32_t *status, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* BFGPU_H */
