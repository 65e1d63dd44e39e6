// solve_core.cuh -- per-warp / per-block device routines of Algorithm 1
// (Sec. IV-A), shared by the single solve (solve.cu), the batched engine
// (batch.cu, serve.cu) and the allocation-free solve (noalloc.cu).
//
// State of one instance (InstView):
//   Vkey        int64 [C]  W as order-preserving keys (bf_internal.cuh)
//   M2, M3      int64 [C]  window maxima along dim 0: M2(y) = max(V(y), V(y+1)),
//                          M3(y) = max(V(y..y+2)) (wrapping on a periodic dim 0),
//                          equal to V's windows at the start of every pass
//   M33         int64 [C]  (single solve) max of V over y0..y0+2 x y1..y1+2 on
//                          dims 0-1 (wrapping on periodic dims), same refresh
//   M33P        int64 [C]  (single solve, optional) max(M33(y), M33(y + e_z)) for
//                          one dim z >= 2 (the plane-pair dim; wrapping on a
//                          periodic z, M33(y) alone on a non-periodic z's last
//                          index), same refresh
//   fbits       u32 [S]    upcoming frontier F2, one bit per cell
//   cells       i32 [C]    current frontier F1 as a compacted cell list
//   chg         i32 [C]    cells whose W decreased in the current pass
//
// One pass of the while-loop (single solve: two kernels; batched engine and
// scratch solve: three, with propagate on its own):
//   relax      warp per 32 cells of F1 (lanes = cells): for u = 0..U-1,
//              d = G(x,u) + max_{y in F(x,u)} V(y) (one FP64 add, max on keys),
//              lowest u among the smallest d; if d < W(x): Vnew(x), mu(x) and
//              append x to chg.  V and the tables are read-only here, so the
//              pass is synchronous (Jacobi).  The same warp then sets the bits
//              of its changed cells' predecessor boxes in fbits (F2 = union of
//              pred of the changed cells), one box per run of cells along a
//              dim-0 row.
//   propagate  (three-kernel form) warp per changed cell y: commit W(y) =
//              Vnew(y) and mark as above from the changed list.
//   compact    block per 256 bitmap words: F2's bits -> the cell list of the
//              next pass (ordered within a block; bits cleared on the way);
//              threads also commit W = Vnew on the changed cells (two-kernel
//              form) and refresh the window maxima around them; the last block
//              closes the pass (trace, i += 1, loop condition F1 != empty and
//              i < cap).
//
// Box gather.  For a pair whose box spans w0 cells along dim 0, one row of
// the box is max over [lo0, lo0 + w0): one table lookup for w0 <= 3 (V, M2 or
// M3) and ceil(w0 / 3) overlapping M3 lookups beyond.  When all lanes of a
// warp hold boxes of the same shape relative to their cells (true for
// dynamics invariant under translation along the grid, such as the built-in
// systems), every lookup is one warp load at a lane-independent offset from
// each lane's cell and the loops are warp-uniform.  Other warps walk each
// lane's box cell by cell.
//
// Plane relax forms (abstractions with a plane shape table): the lists of the
// plane a warp's cells lie on are staged in shared memory; relax_plane reads
// every record, relax_plane_m the per-cell input masks (inputs in turn), and
// relax_plane_q queues the (lane, input) pairs the lists serve over the lanes,
// so that with the per-input frontier (one bitmap per input, marked from
// per-input templates) only pairs whose box holds a changed cell cost work.
#pragma once
#include <type_traits>

#include "bf_internal.cuh"
#include "dynamics.cuh"

namespace bfk {

struct Counters {
    int ncur;                 // cells of the current frontier F1 (in `cells`)
    int nnext;                // cells compacted for the next pass
    int nchg;                 // cells changed in the current pass
    int err;                  // nonzero: invalid input seen during set-up
    long long round;          // passes completed (i of Algorithm 1)
    long long cap;            // |X| or the caller's smaller cap
    long long relaxed;        // cells relaxed in the current pass
    long long total_relaxed;  // summed over passes
    long long exact;          // cells of the exact F1 in the current pass (counting mode)
    long long total_exact;
    long long pairs;          // (cell, input) pairs the masked relax took up in the current pass
    long long total_pairs;
    long long total_changed;
    unsigned blocks_done;     // blocks of the running compact launch that finished
    int done;                 // loop condition became false
    int status;               // BF_CONVERGED / BF_NEG_CYCLE / BF_ITER_CAP
    int fault;                // nonzero: a kernel gave up waiting for its copies (tile relax)
    int ubuf;                 // per-input frontier: the buffer holding the current frontier
};

struct InstView {
    GridDesc g;
    DynDesc dd;
    int box_fmt;                // kBoxWide / kBoxCompact / kBoxRecompute / kBoxHybrid
    int nstored;                // hybrid: inputs u < nstored have compact records
    const void* boxes;          // [U][C] records (wide or compact) or NULL
    const double* inputs;       // [U][udim] (recompute mode)
    const double* rk;           // [keys][U][kRkEntry] shared RK4 parts (recompute mode) or NULL
    const short* pred;          // [C][2D] predecessor offsets
    // plane lookup lists (compact records, grids of 2+ dims): per (plane,
    // input) the record every non-blocked pair of the plane shares and the
    // offsets of its box's table lookups (plane_offsets), or NULL
    const unsigned long long* shape;   // [P][U]
    const int* poffs;                  // [P][U][kPlaneEnt]
    // per cell: bit u (u < 32) = the pair (c, u) has a box and its record is
    // the plane's entry; bit 32 + u = a box with another record; or NULL
    const unsigned long long* fmask;   // [C]
    // predecessor templates per target plane (marking), or NULL: bounding boxes
    const int* tptr;                   // [2 P + 1] (entries without the flag first)
    const int4* tent;
    const double* Gint;         // [U][C] running cost, +inf on avoid cells
    long long* Vkey;            // [C]
    long long* Vnew;            // [C]
    long long* M2;              // [C]
    long long* M3;              // [C]
    long long* M33;             // [C] max of V over 3 x 3 cells on dims 0-1, or NULL
    long long* M33P;            // [C] max of M33 over two planes along dim pz, or NULL
    int pz;                     // plane-pair dim (2 .. D - 1) of M33P, 0: none
    unsigned char* mu;          // [C]
    unsigned* fbits;            // [S]
    // per-input frontier (per-input templates, U <= 32): one bitmap per input
    // (the pairs (x, u) whose box holds a changed cell) in two buffers, the
    // current frontier in buffer ctr->ubuf (relax reads it), the upcoming one
    // in the other (marking sets it, compact takes its cells and clears the
    // current one for the pass after); NULL: the cell frontier fbits, every
    // input of a frontier cell
    const int* uptr;            // [2 P + 1] per-input templates, as tptr
    const int4* uent;
    unsigned* ubits;            // [2][U][S]
    long long nwords;           // S
    int* cells;                 // [C]
    int* chg;                   // [C]
    Counters* ctr;
    long long* trace;           // [trace_cap][4] or NULL
    long long trace_cap;
    int* stamp;                 // [C] pass that last changed the cell (counting mode) or NULL
    // frontier cache (recompute / hybrid modes): the records of the inputs u >=
    // nstored of the first fc_cap cells of each pass's frontier list, in two
    // buffers [U - nstored][fc_cap] used by alternate passes, and per cell a tag
    // ((pass + 2) << 32 | position) of the pass and place that wrote them
    unsigned long long* fc[2];
    long long* fc_tag;          // [C]
    long long fc_cap;           // 0: no cache
    unsigned* f1bits;           // [S] the current frontier F1 as a bitmap (tile relax) or NULL
    long long dense_min;        // passes with at least this many F1 cells take the tile relax
                                // (the list relax returns at once), else the list relax
    // input slices (small frontiers): per (chunk, slice) lane candidates and
    // per chunk arrival counters; NULL -> one warp per chunk over all inputs
    long long* cand_key;        // [slice_cap]
    int* cand_u;                // [slice_cap] input (0xFFFF: none) | exact flag << 16
    int* slice_cnt;             // [slice_cap / 32], zero between passes
    long long slice_cap;
    int slice_target;           // see kSliceTarget
    int inplace;                // BF_SCHED_INPLACE: a decrease is written to Vkey at once
    // successor class (running cost Gc(x,u) for successors y in the class):
    // NULL rmask = none.  VN / VR hold V off / on the class (kKeyMin elsewhere),
    // M2 / M3 then hold VN's windows and M2R / M3R VR's.
    const unsigned char* rmask; // [C]
    const double* GRint;        // [U][C] class running cost, +inf on avoid cells
    long long* VN;
    long long* VR;
    long long* M2R;
    long long* M3R;
};

// Plane lookup list entry: int 0 = L | table << 8 (L = 0: no list, the
// lanes take the general gather; table 0..4 = V, M2, M3, M33, M33P), ints
// 4 .. 4 + L4 - 1 the offsets of the L lookups from the cell, L4 = L rounded
// up to 4 (padded with the first).
constexpr int kPlaneEnt = 4 + 28;
constexpr int kPlaneMaxLook = 28;

// Slices: a pass whose frontier has fewer than slice_target x (warps of the
// relax grid) chunks splits the inputs of each chunk over several warps
// (slice_target 0: never).  kSliceTarget is the default, kSliceTargetMax the
// largest a workspace's buffers hold.
constexpr int kSliceTarget = 2;
constexpr int kSliceTargetMax = 4;

// Host: the abstraction part of a view (grid, dynamics, boxes, pred).
inline void view_from_abs(InstView& v, const bf_abstraction* a) {
    v.g = a->g;
    v.dd.kind = a->dyn.kind;
    v.dd.substeps = a->dyn.rk4_substeps;
    v.dd.udim = a->udim;
    v.dd.tau = a->tau;
    for (int i = 0; i < 8; ++i) v.dd.p[i] = a->dyn.param[i];
    for (int d = 0; d < 4; ++d) {
        v.dd.glo[d] = d < a->g.D ? a->glo[d] : 0.0;
        v.dd.eta[d] = d < a->g.D ? (a->ghi[d] - a->glo[d]) / (double)a->g.n[d] : 1.0;
    }
    v.box_fmt = a->box_fmt;
    v.nstored = a->nstored;
    v.boxes = a->d_boxes;
    v.inputs = a->d_inputs;
    v.rk = a->d_rk;
    v.pred = a->d_pred;
    v.shape = a->d_shape;
    v.poffs = nullptr;            // set by the solve that built the lists
    v.fmask = nullptr;            // set by the solve when it relaxes by cell masks
    v.M33P = nullptr;             // set by the solve that keeps the plane-pair table
    v.pz = 0;
    v.tptr = nullptr;             // set by the solve when it marks with templates
    v.tent = nullptr;
}

// ---------------------------------------------------------------------------
// set-up (lines 1-9 of Algorithm 1), shared by every solve entry point
// ---------------------------------------------------------------------------

// -0 -> +0; NaN, -inf and |finite| > 2^64 are errors.
__device__ __forceinline__ bool clean_cost(double v, double& out) {
    if (v != v) return false;
    if (v == -__longlong_as_double(0x7FF0000000000000LL)) return false;
    if (v != __longlong_as_double(0x7FF0000000000000LL) && fabs(v) > 18446744073709551616.0) return false;
    out = (v == 0.0) ? 0.0 : v;
    return true;
}

// Gint[u][c] = clean(G[c][u]), +inf on avoid cells (grid-stride over cells).
// Lanes take consecutive cells of one input: the writes are coalesced and the
// strided reads of a warp's 32 x U block are served from L1 across the u loop.
__device__ __forceinline__ void init_costs_body(long long C, int U, const double* __restrict__ G,
                                                const unsigned char* __restrict__ avoid, double* Gint,
                                                Counters* ctr) {
    const double inf = __longlong_as_double(0x7FF0000000000000LL);
    bool bad = false;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < C;
         c += (long long)gridDim.x * blockDim.x) {
        const bool av = avoid && avoid[c];
        for (int u = 0; u < U; ++u) {
            double v;
            if (!clean_cost(__ldg(G + c * U + u), v)) bad = true;
            Gint[(long long)u * C + c] = av ? inf : v;
        }
    }
    if (bad) atomicOr(&ctr->err, 1);
}

// Lines 1-9 of Algorithm 1: W = terminal cost (0 on target, +inf elsewhere,
// or the caller's array), mu = U (hand over); the cells with finite W go to
// the changed list so that the first propagate builds F1 from their preds.
// stamp (counting mode) or NULL.
__device__ __forceinline__ void init_values_body(long long C, const double* __restrict__ terminal,
                                                 const unsigned char* __restrict__ target,
                                                 const unsigned char* __restrict__ avoid, long long* Vkey,
                                                 long long* Vnew, unsigned char* mu, int* chg, int* stamp,
                                                 Counters* ctr) {
    const double inf = __longlong_as_double(0x7FF0000000000000LL);
    bool bad = false;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long start = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    // uniform trip count per warp so the ballot in warp_append is safe
    const long long rounds = (C + stride - 1) / stride;
    for (long long it = 0; it < rounds; ++it) {
        const long long c = start + it * stride;
        bool finite = false;
        if (c < C) {
            double t;
            if (terminal) {
                if (!clean_cost(terminal[c], t)) { bad = true; t = inf; }
            } else {
                t = (target && target[c]) ? 0.0 : inf;
            }
            if (avoid && avoid[c]) t = inf;
            const long long k = key_of(t);
            Vkey[c] = k;
            Vnew[c] = k;
            mu[c] = kHandover;
            finite = k != kKeyInf;
            if (stamp) stamp[c] = finite ? -1 : -2;   // -1: "changed" before pass 0
        }
        const int slot = warp_append(finite, &ctr->nchg);
        if (finite) chg[slot] = (int)c;
    }
    if (bad) atomicOr(&ctr->err, 1);
}

// ---------------------------------------------------------------------------
// compact relative box records
// ---------------------------------------------------------------------------
// Byte 2d = lower corner minus the cell's coordinate on dim d (int8; on a
// periodic dim reduced to [-n/2, n/2)); byte 2d+1 = width on dim d (1..127).
// A width byte of 0 on dim 0 marks a blocked pair; bit 7 of that byte marks a
// box that wraps around a periodic dim for this cell (gathered cell by cell).
// D <= 2: 4-byte records, D >= 3: 8-byte records.
template <int D>
using compact_t = typename std::conditional<(D <= 2), unsigned, unsigned long long>::type;

__device__ __forceinline__ int rec_byte(unsigned long long r, int k) { return (int)((r >> (8 * k)) & 0xFF); }
__device__ __forceinline__ int rec_sbyte(unsigned long long r, int k) {
    return (int)(signed char)((r >> (8 * k)) & 0xFF);
}

__device__ __forceinline__ unsigned long long shfl_u64(unsigned long long x, int src) {
    const unsigned lo = __shfl_sync(0xFFFFFFFFu, (unsigned)x, src);
    const unsigned hi = __shfl_sync(0xFFFFFFFFu, (unsigned)(x >> 32), src);
    return ((unsigned long long)hi << 32) | lo;
}

// Absolute box of a compact record (slow path; needs the cell's coordinates).
template <int D>
__device__ __forceinline__ Box<D> decode_compact(unsigned long long r, const GridDesc& g, long long c) {
    Box<D> b;
    int k[4];
    cell_coords(g, c, k);
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const int w = rec_byte(r, 2 * d + 1) & 0x7F;
        int lo = k[d] + rec_sbyte(r, 2 * d);
        if (g.periodic[d]) {
            if (lo < 0) lo += g.n[d];
            else if (lo >= g.n[d]) lo -= g.n[d];
        }
        b.lo[d] = lo;
        b.hi[d] = lo + w - 1;
    }
    return b;
}

// ---------------------------------------------------------------------------
// gathers
// ---------------------------------------------------------------------------

// Max of V over the box of relative record r for the lanes with `mine` set.
// Those lanes share r and, when r wraps a periodic dim, the coordinates of
// their cells on the periodic dims, so every lookup (row x piece) lies at the
// same offset from each lane's cell; lc is one of their cells.  Rows along
// dim 0 are read from the window tables (V, M2, M3: one lookup covers up to 3
// cells), so a box takes ceil(w0/3) x w1 x w2 x w3 lookups.  Lane e computes
// the offset of lookup e once and the warp walks the offsets broadcast by
// shuffle, four loads in flight.  Must be called by all 32 lanes.
template <int D, bool CLS = false>
__device__ __forceinline__ long long box_max_rows(const InstView& v, long long c, bool mine,
                                                  unsigned long long r, long long lc, long long* mcls = nullptr) {
    const GridDesc& g = v.g;
    const int lane = threadIdx.x & 31;
    int w[4] = {1, 1, 1, 1}, rel[4] = {0, 0, 0, 0}, k[4] = {0, 0, 0, 0}, lo[4] = {0, 0, 0, 0};
#pragma unroll
    for (int d = 0; d < D; ++d) {
        w[d] = rec_byte(r, 2 * d + 1) & 0x7F;
        rel[d] = rec_sbyte(r, 2 * d);
    }
    const bool wrap = (rec_byte(r, 1) & 0x80) != 0;
    if (wrap) {
        cell_coords(g, lc, k);
#pragma unroll
        for (int d = 1; d < D; ++d) {
            int l = k[d] + rel[d];
            if (g.periodic[d]) {
                if (l < 0) l += g.n[d];
                else if (l >= g.n[d]) l -= g.n[d];
            }
            lo[d] = l;
        }
    }
    // successor classes: V off the class in VN / M2 / M3, on it in VR / M2R / M3R.
    // A box at least 3 cells wide on dims 0 and 1 reads 3 x 3 windows (M33):
    // ceil(w0/3) x ceil(w1/3) lookups per dims >= 2 place instead of ceil(w0/3) x w1.
    bool use33 = false;
    if constexpr (!CLS && D >= 2) use33 = v.M33 != nullptr && w[0] >= 3 && w[1] >= 3;
    const long long* tab = use33 ? v.M33 : (w[0] == 1 ? (CLS ? v.VN : v.Vkey) : (w[0] == 2 ? v.M2 : v.M3));
    const int np = w[0] < 3 ? 1 : (w[0] + 2) / 3;            // lookups per row
    const int n1 = use33 ? (w[1] + 2) / 3 : w[1];            // lookups along dim 1
    const int total = np * n1 * w[2] * w[3];
    // lookup e = q + np (j1 + n1 (j2 + w2 j3)); below 2^23 lookups (every box
    // of a real system) its digits come from multiply-high quotients
    const bool quick = (unsigned)total < kSmallDivMax;
    const unsigned inv_q = kRecip.m[np], inv_1 = kRecip.m[n1], inv_2 = kRecip.m[w[2]];
    const long long* p = tab + (mine ? c + rel[0] : 0);
    long long m0 = kKeyMin, m1 = kKeyMin;
    const long long* pr = nullptr;
    long long r0 = kKeyMin, r1 = kKeyMin;
    if constexpr (CLS) pr = (w[0] == 1 ? v.VR : (w[0] == 2 ? v.M2R : v.M3R)) + (mine ? c + rel[0] : 0);
    for (int e0 = 0; e0 < total; e0 += 32) {
        int off = 0;
        const int e = e0 + lane;
        if (e < total) {
            int q, j[4] = {0, 0, 0, 0};
            if (quick) {
                const unsigned t1 = small_div((unsigned)e, inv_q);
                q = e - (int)(t1 * np);
                if constexpr (D == 2) {
                    j[1] = (int)t1;
                } else if constexpr (D >= 3) {
                    const unsigned t2 = small_div(t1, inv_1);
                    j[1] = (int)(t1 - t2 * n1);
                    if constexpr (D == 3) {
                        j[2] = (int)t2;
                    } else {
                        const unsigned t3 = small_div(t2, inv_2);
                        j[2] = (int)(t2 - t3 * w[2]);
                        j[3] = (int)t3;
                    }
                }
            } else {
                int t = e;
                q = t % np;
                t /= np;
                j[1] = t % n1;
                t /= n1;
                j[2] = t % w[2];
                j[3] = t / w[2];
            }
            if (use33) j[1] = min(3 * j[1], w[1] - 3);         // window rows j1 .. j1 + 2
            off = w[0] < 3 ? 0 : min(3 * q, w[0] - 3);
#pragma unroll
            for (int d = 1; d < D; ++d) {
                int dl = rel[d] + j[d];
                if (wrap && g.periodic[d]) {
                    int x = lo[d] + j[d];
                    if (x >= g.n[d]) x -= g.n[d];
                    dl = x - k[d];
                }
                off += dl * (int)g.stride[d];
            }
        }
        const int n = min(32, total - e0);
        int kk = 0;
        for (; kk + 4 <= n; kk += 4) {
            const int o0 = __shfl_sync(0xFFFFFFFFu, off, kk), o1 = __shfl_sync(0xFFFFFFFFu, off, kk + 1);
            const int o2 = __shfl_sync(0xFFFFFFFFu, off, kk + 2), o3 = __shfl_sync(0xFFFFFFFFu, off, kk + 3);
            if (mine) {
                const long long a0 = __ldg(p + o0), a1 = __ldg(p + o1), a2 = __ldg(p + o2), a3 = __ldg(p + o3);
                m0 = max(m0, max(a0, a2));
                m1 = max(m1, max(a1, a3));
                if constexpr (CLS) {
                    const long long b0 = __ldg(pr + o0), b1 = __ldg(pr + o1), b2 = __ldg(pr + o2), b3 = __ldg(pr + o3);
                    r0 = max(r0, max(b0, b2));
                    r1 = max(r1, max(b1, b3));
                }
            }
        }
        for (; kk < n; ++kk) {
            const int o = __shfl_sync(0xFFFFFFFFu, off, kk);
            if (mine) {
                m0 = max(m0, __ldg(p + o));
                if constexpr (CLS) r0 = max(r0, __ldg(pr + o));
            }
        }
    }
    if constexpr (CLS) *mcls = max(r0, r1);
    return max(m0, m1);
}

// Plane of cell x: its coordinates on dims >= 2 as one index (0 for D = 2).
template <int D>
__device__ __forceinline__ int plane_of_cell(const GridDesc& g, long long x) {
    if constexpr (D <= 2) return 0;
    else return (int)grid_div(g, 1, grid_div(g, 0, (unsigned)x));
}

// Lookup list of record r on plane p (the lookups box_max_rows makes for a
// lane of that plane, as offsets from the cell); the table is M33 when m33
// and the box is at least 3 cells wide on dims 0 and 1, else V / M2 / M3 by
// the width on dim 0.  With a plane-pair dim pz (2 .. D - 1; 0: none) a box
// that reads M33 and spans at least 2 planes on dim pz reads M33P instead, at
// ceil(w_pz / 2) positions along pz (the last one shifted back to end on the
// box's last plane: the windows may overlap, the maximum is the same).  Dims
// 0 and 1 are not periodic here; periodic dims >= 2 wrap with the plane's
// coordinates.
template <int D>
__device__ __forceinline__ void plane_offsets(const GridDesc& g, unsigned long long r, int p, bool m33, int pz,
                                              int* out) {
    out[0] = 0;
    if ((rec_byte(r, 1) & 0x7F) == 0) return;                 // no pair of the plane
    int w[4] = {1, 1, 1, 1}, rel[4] = {0, 0, 0, 0}, k[4] = {0, 0, 0, 0};
#pragma unroll
    for (int d = 0; d < D; ++d) {
        w[d] = rec_byte(r, 2 * d + 1) & 0x7F;
        rel[d] = rec_sbyte(r, 2 * d);
    }
    if (D >= 3) { k[2] = p % g.n[2]; k[3] = p / g.n[2]; }
    const bool use33 = m33 && D >= 2 && w[0] >= 3 && w[1] >= 3;
    const bool usep = use33 && pz >= 2 && pz < D && w[pz] >= 2;
    const int tab = usep ? 4 : (use33 ? 3 : (w[0] == 1 ? 0 : (w[0] == 2 ? 1 : 2)));
    const int np = w[0] < 3 ? 1 : (w[0] + 2) / 3;
    const int n1 = use33 ? (w[1] + 2) / 3 : w[1];
    // positions along dims 2 and 3 (steps of 2 along the pair dim)
    int n23[4] = {1, 1, 1, 1};
    for (int d = 2; d < D; ++d) n23[d] = (usep && d == pz) ? (w[d] + 1) / 2 : w[d];
    const long long L = (long long)np * n1 * n23[2] * n23[3];
    if (L > kPlaneMaxLook) return;
    int lo[4] = {0, 0, 0, 0};
#pragma unroll
    for (int d = 2; d < D; ++d) {
        int x = k[d] + rel[d];
        if (g.periodic[d]) x = ((x % g.n[d]) + g.n[d]) % g.n[d];
        lo[d] = x;
    }
    int i = 0;
    for (int j3 = 0; j3 < n23[3]; ++j3)
        for (int j2 = 0; j2 < n23[2]; ++j2)
            for (int j1 = 0; j1 < n1; ++j1)
                for (int q = 0; q < np; ++q) {
                    int off = rel[0] + (w[0] < 3 ? 0 : min(3 * q, w[0] - 3));
                    off += (rel[1] + (use33 ? min(3 * j1, w[1] - 3) : j1)) * (int)g.stride[1];
                    int j[4] = {0, 0, j2, j3};
                    if (usep) j[pz] = min(2 * j[pz], w[pz] - 2);
#pragma unroll
                    for (int d = 2; d < D; ++d) {
                        int x = lo[d] + j[d];
                        if (g.periodic[d] && x >= g.n[d]) x -= g.n[d];
                        off += (x - k[d]) * (int)g.stride[d];
                    }
                    out[4 + i++] = off;
                }
    for (; i & 3; ++i) out[4 + i] = out[4];
    out[0] = (int)L | (tab << 8);
}

// Does the box hold a cell whose stamp equals `want` (counting mode)?
template <int D>
__device__ __forceinline__ bool box_has_stamp(const int* __restrict__ stamp, const GridDesc& g,
                                              const Box<D>& b, int want) {
    int len[D];
    int total = 1;
#pragma unroll
    for (int d = 0; d < D; ++d) { len[d] = b.hi[d] - b.lo[d] + 1; total *= len[d]; }
    for (int t = 0; t < total; ++t) {
        int r = t;
        long long y = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int k = r % len[d];
            r /= len[d];
            y += (long long)wrap_idx(b.lo[d] + k, g.n[d], g.periodic[d]) * g.stride[d];
        }
        if (stamp[y] == want) return true;
    }
    return false;
}

// ---------------------------------------------------------------------------
// propagate
// ---------------------------------------------------------------------------

// Set the bits `mask` of word wd of the upcoming frontier.  The atomicOr's
// result is not used, so it is a reduction the warp does not wait for (no
// read of the word first: the predecessor boxes of neighbouring changed cells
// overlap, and a read that finds the bits set still costs an L2 round trip).
__device__ __forceinline__ void mark_word(unsigned* fbits, int wd, unsigned mask) {
    atomicOr(&fbits[wd], mask);
}

__device__ __forceinline__ unsigned bit_range(int s, int e) {
    return (e == 31 ? 0xFFFFFFFFu : ((1u << (e + 1)) - 1u)) & ~((1u << s) - 1u);
}

// Set the bits of the box lo[d] .. lo[d] + len[d] - 1 (wrapping on periodic
// dims; rows = product of len[1..D-1]) in fbits; lanes take the rows.
template <int D>
__device__ __forceinline__ void mark_box_rows(const InstView& v, const int* lo, const int* len, int rows) {
    const int lane = threadIdx.x & 31;
    const GridDesc& g = v.g;
    const int n0 = g.n[0];
    const int a0 = lo[0], e0 = lo[0] + len[0] - 1;
    const int e1 = min(e0, n0 - 1);
    const bool wrap = e0 >= n0;                                   // periodic dim 0: the part past n0 - 1 wraps
    // row r = j1 + len1 (j2 + len2 j3): multiply-high quotients for the usual sizes
    const bool quick = (unsigned)rows < kSmallDivMax && len[1] < 256 && (D < 4 || len[2] < 256);
    const unsigned m1 = kRecip.m[min(len[1], 255)], m2 = kRecip.m[min(len[2], 255)];
    for (int r = lane; r < rows; r += 32) {
        int j[4] = {0, 0, 0, 0};
        const unsigned t = (unsigned)r;
        if constexpr (D == 2) {
            j[1] = (int)t;
        } else if constexpr (D == 3) {
            j[2] = (int)(quick ? small_div(t, m1) : t / (unsigned)len[1]);
            j[1] = (int)(t - (unsigned)j[2] * (unsigned)len[1]);
        } else if constexpr (D == 4) {
            const unsigned t2 = quick ? small_div(t, m1) : t / (unsigned)len[1];
            j[1] = (int)(t - t2 * (unsigned)len[1]);
            j[3] = (int)(quick ? small_div(t2, m2) : t2 / (unsigned)len[2]);
            j[2] = (int)(t2 - (unsigned)j[3] * (unsigned)len[2]);
        }
        int rowbase = 0;
#pragma unroll
        for (int d = 1; d < D; ++d) {
            int xd = lo[d] + j[d];
            if (g.periodic[d] && xd >= g.n[d]) xd -= g.n[d];
            rowbase += xd * (int)g.stride[d];
        }
        for (int part = 0; part < (wrap ? 2 : 1); ++part) {
            const int a = rowbase + (part ? 0 : a0);
            const int b = rowbase + (part ? e0 - n0 : e1);
            for (int wd = a >> 5; wd <= (b >> 5); ++wd) {
                const int lo_b = max(a, wd << 5), hi_b = min(b, (wd << 5) + 31);
                mark_word(v.fbits, wd, bit_range(lo_b & 31, hi_b & 31));
            }
        }
    }
}

// Set the bits of pred of the run of changed cells y0 .. y0 + L - 1 on row y1
// of plane p from p's predecessor template (dims 0 and 1 not periodic): per
// entry (q, d1, lo, hi) the cells y0 + lo .. y0 + L - 1 + hi of row y1 + d1 of
// plane q, clipped to the grid.  skip_cov: the warp already marked the run
// y0 .. y0 + L - 1 on row y1 - 1 of the same plane, which covered every entry
// whose flag says row d1 + 1 spans its range.  Lanes take entries.
__device__ __forceinline__ void mark_template(const InstView& v, int p, int y0, int L, int y1, bool skip_cov) {
    const int lane = threadIdx.x & 31;
    const int n0 = v.g.n[0], n1 = v.g.n[1];
    const bool per_input = v.ubits != nullptr;       // rows by input into that input's bitmap
    const int* tp = per_input ? v.uptr : v.tptr;
    const int4* te = per_input ? v.uent : v.tent;
    // the flagged entries (row d1 + 1 spans the same range) come last
    const int b = __ldg(tp + 2 * p), e = __ldg(tp + 2 * p + (skip_cov ? 1 : 2));
    unsigned* ub = per_input ? v.ubits + (long long)(v.ctr->ubuf ^ 1) * v.g.U * v.nwords : v.fbits;
    for (int i = b + lane; i < e; i += 32) {
        const int4 t = __ldg(te + i);
        unsigned* bits = per_input ? ub + (long long)(t.w >> 8) * v.nwords : ub;
        const int r = y1 + t.y;
        if (r < 0 || r >= n1) continue;
        const int lo = (int)(short)(t.z & 0xFFFF), hi = t.z >> 16;
        const int a = max(0, y0 + lo), z = min(n0 - 1, y0 + L - 1 + hi);
        if (a > z) continue;
        const int base = (t.x * n1 + r) * n0;
        const int ca = base + a, cz = base + z;
        for (int wd = ca >> 5; wd <= (cz >> 5); ++wd) {
            const int lo_b = max(ca, wd << 5), hi_b = min(cz, (wd << 5) + 31);
            mark_word(bits, wd, bit_range(lo_b & 31, hi_b & 31));
        }
    }
}

// Changed cells that follow each other along a dim-0 row, in consecutive
// places of the changed list, form a run.  propagate_entry(i) commits
// chg[i]; when chg[i] starts a run, it also sets the bits of the bounding box
// of the run's predecessor boxes in fbits -- their union, for dynamics
// invariant under translation; a superset otherwise, which relaxes a few
// extra cells and changes no result, since a cell none of whose boxes holds a
// changed cell cannot decrease.  Lanes take the rows (dim-0 runs) of the box.
// Called by a whole warp.
template <int D>
__device__ __forceinline__ void propagate_entry(const InstView& v, int i, int nchg, bool commit) {
    const int lane = threadIdx.x & 31;
    const GridDesc& g = v.g;
    const int n0 = g.n[0];
    const int y0 = v.chg[i];
    if (commit && lane == 0) {
        v.Vkey[y0] = v.Vnew[y0];
        if (v.stamp) v.stamp[y0] = (int)v.ctr->round;
    }
    const int k0 = y0 - (int)grid_div(g, 0, (unsigned)y0) * n0;
    if (i > 0 && k0 != 0 && v.chg[i - 1] == y0 - 1) return;     // inside a run
    if (v.tent) {
        // the run's length, 32 places at a time
        int L = 0;
        for (int off = 0;; off += 32) {
            const int idx = i + off + lane;
            const int y = idx < nchg ? v.chg[idx] : -1;
            const bool in = y >= 0 && y == y0 + off + lane && k0 + off + lane < n0;
            const unsigned inm = __ballot_sync(0xFFFFFFFFu, in);
            const unsigned runm = ~inm ? (inm & ((1u << (__ffs(~inm) - 1)) - 1u)) : inm;
            L += __popc(runm);
            if (runm != 0xFFFFFFFFu) break;
        }
        const unsigned rq = grid_div(g, 0, (unsigned)y0);
        const int y1 = (int)(rq - grid_div(g, 1, rq) * (unsigned)g.n[1]);
        // the run's cells one dim-1 row down all changed in this pass (W not
        // yet committed: Vnew != Vkey): the runs holding them mark every row
        // a covered template entry would (dims 0 and 1 are not periodic here)
        bool cov = false;
        if (!commit && !v.inplace && y1 > 0) {
            bool all = true;
            for (int off = 0; off < L; off += 32) {
                bool ok = true;
                if (off + lane < L) {
                    const long long yb = (long long)y0 + off + lane - n0;
                    ok = v.Vnew[yb] != v.Vkey[yb];
                }
                all = __all_sync(0xFFFFFFFFu, ok) && all;
            }
            cov = all;
        }
        mark_template(v, plane_of_cell<D>(g, y0), k0, L, y1, cov);
        return;
    }
    // gather the run 32 places at a time; per lane min / max of the box ends
    int mn[D], mx[D];
#pragma unroll
    for (int d = 0; d < D; ++d) { mn[d] = 0x7FFFFFFF; mx[d] = (int)0x80000000; }
    int kh[4];
    cell_coords(g, y0, kh);
    for (int off = 0;; off += 32) {
        const int idx = i + off + lane;
        const int y = idx < nchg ? v.chg[idx] : -1;
        // lane l is in the run when chg[i + off + l] == y0 + off + l on y0's row
        const bool in = y >= 0 && y == y0 + off + lane && k0 + off + lane < n0;
        const unsigned inm = __ballot_sync(0xFFFFFFFFu, in);
        const unsigned runm = ~inm ? (inm & ((1u << (__ffs(~inm) - 1)) - 1u)) : inm;   // prefix of lanes in the run
        if ((runm >> lane) & 1) {
            const short* q = v.pred + (long long)y * (2 * D);
            const int ql0 = q[0], qh0 = q[D];
            if (ql0 <= qh0) {
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    const int base = d == 0 ? off + lane : 0;
                    mn[d] = min(mn[d], base + (int)q[d]);
                    mx[d] = max(mx[d], base + (int)q[D + d]);
                }
            }
        }
        if (runm != 0xFFFFFFFFu) break;
    }
    int lo[4] = {0, 0, 0, 0}, len[4] = {1, 1, 1, 1};
    int rows = 1;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const int n = g.n[d];
        const int a = __reduce_min_sync(0xFFFFFFFFu, mn[d]);
        const int b = __reduce_max_sync(0xFFFFFFFFu, mx[d]);
        if (a > b) return;                                        // no predecessor in the run
        int s = kh[d] + a;
        int len_d = b - a + 1;
        if (g.periodic[d]) {                      // s in [-n/2, 3n/2): offsets are kept in [-n/2, n/2)
            if (len_d >= n) { s = 0; len_d = n; }
            else if (s < 0) s += n;
            else if (s >= n) s -= n;
        }
        lo[d] = s;
        len[d] = len_d;
        if (d > 0) rows *= len_d;
    }
    mark_box_rows<D>(v, lo, len, rows);
}

// Set the bits of the predecessor boxes of the changed lanes' cells y in
// fbits (whole warp; relax calls it right after deciding its cells, so the
// frontier of the next pass is built while the pass runs).  Changed cells
// that follow each other along a dim-0 row in consecutive lanes form a run,
// which marks the bounding box of its cells' predecessor boxes (the same
// superset argument as propagate_entry).
template <int D>
__device__ __forceinline__ void mark_changed(const InstView& v, int y, bool changed) {
    const int lane = threadIdx.x & 31;
    const GridDesc& g = v.g;
    int ql[D], qh[D];
    int ky[4] = {0, 0, 0, 0};
    bool has = false;
#pragma unroll
    for (int d = 0; d < D; ++d) { ql[d] = 0; qh[d] = -1; }
    if (changed) {
        const short* q = v.pred + (long long)y * (2 * D);
#pragma unroll
        for (int d = 0; d < D; ++d) { ql[d] = q[d]; qh[d] = q[D + d]; }
        has = ql[0] <= qh[0];                    // else y has no predecessor
        if (has) cell_coords(g, y, ky);
    }
    const int yprev = __shfl_up_sync(0xFFFFFFFFu, y, 1);
    const int hprev = __shfl_up_sync(0xFFFFFFFFu, has ? 1 : 0, 1);
    const bool cont = has && lane > 0 && hprev && y == yprev + 1 && ky[0] != 0;
    const unsigned contm = __ballot_sync(0xFFFFFFFFu, cont);
    unsigned heads = __ballot_sync(0xFFFFFFFFu, has && !cont);
    if constexpr (D >= 2) {
        if (v.tent) {
            // predecessor templates: per run its plane, row and x range; a run
            // on the next dim-1 row of the previous run's plane with the same x
            // range skips the template rows that run already marked
            const int pl = has ? plane_of_cell<D>(g, y) : 0;
            int pp = -1, px = -1, pL = -1, py1 = -1;
            while (heads) {
                const int h = __ffs(heads) - 1;
                heads &= heads - 1;
                const unsigned above = h < 31 ? (contm >> (h + 1)) : 0u;
                const int L = __ffs(~above);                        // lanes h .. h + L - 1
                const int x0 = __shfl_sync(0xFFFFFFFFu, ky[0], h);
                const int y1 = __shfl_sync(0xFFFFFFFFu, ky[1], h);
                const int p = __shfl_sync(0xFFFFFFFFu, pl, h);
                const bool cov = p == pp && x0 == px && L == pL && y1 == py1 + 1;
                mark_template(v, p, x0, L, y1, cov);
                pp = p; px = x0; pL = L; py1 = y1;
            }
            return;
        }
    }
    // the previous run's box: when this run's box is the same box moved up by
    // one cell on dim 1 (and no wider on dim 0), the previous box -- marked by
    // this warp -- holds all of it but its top row on dim 1
    int plo[4] = {0, 0, 0, 0}, plen[4] = {0, 0, 0, 0};
    bool prev = false;
    while (heads) {
        const int h = __ffs(heads) - 1;
        heads &= heads - 1;
        const unsigned above = h < 31 ? (contm >> (h + 1)) : 0u;
        const int last = h + __ffs(~above) - 1;          // the run is lanes h..last
        const bool in = lane >= h && lane <= last;
        int lo[4] = {0, 0, 0, 0}, len[4] = {1, 1, 1, 1};
        int rows = 1, rows2 = 1;                          // rows2: product of len[2..D-1]
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int n = g.n[d];
            const int base = d == 0 ? ky[0] : 0;
            const int mn = __reduce_min_sync(0xFFFFFFFFu, in ? base + ql[d] : 0x7FFFFFFF);
            const int mx = __reduce_max_sync(0xFFFFFFFFu, in ? base + qh[d] : (int)0x80000000);
            int s = mn + (d == 0 ? 0 : __shfl_sync(0xFFFFFFFFu, ky[d], h));
            int len_d = mx - mn + 1;
            if (g.periodic[d]) {                  // s in [-n/2, 3n/2): offsets are kept in [-n/2, n/2)
                if (len_d >= n) { s = 0; len_d = n; }
                else if (s < 0) s += n;
                else if (s >= n) s -= n;
            }
            lo[d] = s;
            len[d] = len_d;
            if (d > 0) rows *= len_d;
            if (d > 1) rows2 *= len_d;
        }
        if constexpr (D >= 2) {
            bool covered = prev && !g.periodic[0] && plo[0] <= lo[0] && plo[0] + plen[0] >= lo[0] + len[0] &&
                           plen[1] == len[1] && len[1] < g.n[1];
            int up = plo[1] + 1;
            if (g.periodic[1] && up >= g.n[1]) up -= g.n[1];
            covered = covered && up == lo[1];
#pragma unroll
            for (int d = 2; d < D; ++d) covered = covered && plo[d] == lo[d] && plen[d] == len[d];
#pragma unroll
            for (int d = 0; d < 4; ++d) { plo[d] = lo[d]; plen[d] = len[d]; }
            prev = true;
            if (covered) {                                    // only the top row on dim 1
                int top = lo[1] + len[1] - 1;
                if (g.periodic[1] && top >= g.n[1]) top -= g.n[1];
                lo[1] = top;
                rows = rows2;
                len[1] = 1;
            }
        }
        mark_box_rows<D>(v, lo, len, rows);
    }
}

// ---------------------------------------------------------------------------
// relax
// ---------------------------------------------------------------------------

// Per-lane view of the pair (x, u): validity, the relative record of its box
// and the absolute box when needed.
template <int D>
struct PairShape {
    bool valid;               // the lane holds a cell and the pair is not blocked
    bool slow;                // gathered cell by cell: the box has no relative
                              // record or wraps a periodic dim 0
    bool have_box;            // b holds the absolute box
    unsigned long long sig;   // relative record (compact form)
    int wkey;                 // wrapping boxes: the cell's place on the periodic dims
    Box<D> b;
};

// Place of a cell on the periodic dims >= 1 (lanes with equal keys see a
// wrapping relative box at equal offsets).
__device__ __forceinline__ int wrap_key(const GridDesc& g, const int* k) {
    int key = 1;
#pragma unroll
    for (int d = 1; d < 4; ++d)
        if (d < g.D && g.periodic[d]) key += k[d] * (int)g.stride[d];
    return key;
}

// A lane's place in the frontier cache: hit = its cell's records of the
// previous pass are at old_pos of the old buffer; pos = where this pass keeps
// them (pos >= fc_cap: not kept).
struct FcLane {
    bool hit;
    long long old_pos;
    long long pos;
};
constexpr unsigned long long kNoRecord = ~0ull;   // a box the compact record cannot hold

// k: the cell's coordinates (only read for wrapping boxes and non-compact
// formats).
template <int D, int FMT>
__device__ __forceinline__ void pair_shape(const InstView& v, long long c, const int* k, int u, bool act,
                                           PairShape<D>& s, const FcLane* fl = nullptr) {
    const GridDesc& g = v.g;
    s.valid = false;
    s.slow = false;
    s.have_box = false;
    s.sig = 0;
    s.wkey = 0;
    if (!act) return;
    bool from_cache = false;
    unsigned long long r = 0;
    if constexpr (FMT == kBoxRecompute || FMT == kBoxHybrid) {
        if (fl && u >= v.nstored) {
            const long long slot = (long long)(u - v.nstored) * v.fc_cap;
            if (fl->hit) {
                r = v.fc[(v.ctr->round + 1) & 1][slot + fl->old_pos];
                from_cache = r != kNoRecord;
            }
            if (from_cache && fl->pos < v.fc_cap) v.fc[v.ctr->round & 1][slot + fl->pos] = r;   // carried over
        }
    }
    if (FMT == kBoxCompact || (FMT == kBoxHybrid && u < v.nstored) || from_cache) {
        if (!from_cache)
            r = (unsigned long long)__ldcs(reinterpret_cast<const compact_t<D>*>(v.boxes) + (long long)u * g.C + c);
        const int f0 = rec_byte(r, 1);
        if ((f0 & 0x7F) == 0) return;                 // blocked
        s.valid = true;
        s.sig = r;
        if (f0 & 0x80) {
            s.wkey = wrap_key(g, k);
            if (g.periodic[0]) {
                const int l0 = k[0] + rec_sbyte(r, 0);
                s.slow = l0 < 0 || l0 + (f0 & 0x7F) > g.n[0];
            }
        }
    } else {
        Box<D> b;
        if constexpr (FMT == kBoxRecompute || FMT == kBoxHybrid) {
            // systems blind to dims 0-1: the abstraction keeps the RK4 work shared
            // by each (dims >= 2 coordinates, input); bit-identical to make_box
            if (D >= 3 && v.rk)
                b = box_from_shared<D>(v.dd, g, k, v.rk + ((long long)rk_key<D>(g, k) * g.U + u) * kRkEntry);
            else
                b = make_box<D>(v.dd, g, v.inputs, c, u);
        } else {
            b = load_box<D>(v.boxes, (long long)u * g.C + c);
        }
        if (b.lo[0] == kBlocked) {
            if constexpr (FMT == kBoxRecompute || FMT == kBoxHybrid)
                if (fl && u >= v.nstored && fl->pos < v.fc_cap)
                    v.fc[v.ctr->round & 1][(long long)(u - v.nstored) * v.fc_cap + fl->pos] = 0ull;
            return;
        }
        s.valid = true;
        s.have_box = true;
        s.b = b;
        // the relative record of the box, as the builder encodes it
        unsigned long long rec = 0;
        bool wrap = false, bad = false;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int n = g.n[d];
            const int w = b.hi[d] - b.lo[d] + 1;
            int rel = b.lo[d] - k[d];
            if (g.periodic[d]) {
                rel %= n;
                if (rel < 0) rel += n;
                if (rel >= n - n / 2) rel -= n;
                const bool wd = (k[d] + rel < 0) || (k[d] + rel + w > n);
                wrap |= wd;
                bad |= d == 0 && wd;
            }
            bad |= w > 127 || w < 1 || rel < -128 || rel > 127;
            rec |= (unsigned long long)(unsigned char)(signed char)rel << (16 * d);
            rec |= (unsigned long long)(w & 0x7F) << (16 * d + 8);
        }
        if (wrap) {
            rec |= 0x80ull << 8;
            s.wkey = wrap_key(g, k);
        }
        s.sig = rec;
        s.slow = bad;
        if constexpr (FMT == kBoxRecompute || FMT == kBoxHybrid)
            if (fl && u >= v.nstored && fl->pos < v.fc_cap)
                v.fc[v.ctr->round & 1][(long long)(u - v.nstored) * v.fc_cap + fl->pos] = bad ? kNoRecord : rec;
    }
}

// Relax the inputs u0 <= u < u1 of the lane's cell c: best (the key to beat,
// on entry W(c)) and bu (-1, or the lowest input reaching best) are updated
// on strict decrease; in counting mode in_exact is set when a box holds a
// cell changed in the previous pass.
template <int D, int FMT, bool COUNT, bool CLS = false>
__device__ __forceinline__ void relax_inputs(const InstView& v, long long c, bool act, int u0, int u1,
                                             long long round, long long& best, int& bu, bool& in_exact,
                                             const FcLane* fl = nullptr) {
    const int lane = threadIdx.x & 31;
    const GridDesc& g = v.g;
    int k[4] = {0, 0, 0, 0};
    if (FMT != kBoxCompact || (g.periodic[0] | g.periodic[1] | g.periodic[2] | g.periodic[3])) cell_coords(g, c, k);
    // the next input's record and cost are loaded while this one is gathered
    PairShape<D> nx;
    pair_shape<D, FMT>(v, c, k, u0, act, nx, fl);
    double ngv = nx.valid ? __ldcs(v.Gint + (long long)u0 * g.C + c) : 0.0;
    double ngr = 0.0;
    if constexpr (CLS) ngr = nx.valid ? __ldcs(v.GRint + (long long)u0 * g.C + c) : 0.0;
    for (int u = u0; u < u1; ++u) {
        PairShape<D> s = nx;
        const double gv = ngv;
        const double gr = ngr;
        if (u + 1 < u1) {
            pair_shape<D, FMT>(v, c, k, u + 1, act, nx, fl);
            ngv = nx.valid ? __ldcs(v.Gint + (long long)(u + 1) * g.C + c) : 0.0;
            if constexpr (CLS) ngr = nx.valid ? __ldcs(v.GRint + (long long)(u + 1) * g.C + c) : 0.0;
        }
        const unsigned vmask = __ballot_sync(0xFFFFFFFFu, s.valid);
        if (!vmask) continue;
        long long m = kKeyMin, mr = kKeyMin;
        unsigned todo = __ballot_sync(0xFFFFFFFFu, s.valid && !s.slow);
        if (vmask & ~todo) {                                  // boxes without a relative record
            if (s.valid && s.slow) {
                if (!s.have_box) {
                    s.b = decode_compact<D>(s.sig, g, c);
                    s.have_box = true;
                }
                if constexpr (CLS) {
                    m = box_max<D>(v.VN, g, s.b);
                    mr = box_max<D>(v.VR, g, s.b);
                } else {
                    m = box_max<D>(v.Vkey, g, s.b);
                }
            }
        }
        while (todo) {                                        // one row gather per group of equal boxes
            const int leader = __ffs(todo) - 1;
            const unsigned long long lsig = shfl_u64(s.sig, leader);
            const int lkey = __shfl_sync(0xFFFFFFFFu, s.wkey, leader);
            const long long lc = __shfl_sync(0xFFFFFFFFu, (int)c, leader);
            const bool mine = ((todo >> lane) & 1) && s.sig == lsig && s.wkey == lkey;
            todo &= ~__ballot_sync(0xFFFFFFFFu, mine);
            long long mmr = kKeyMin;
            const long long mm = box_max_rows<D, CLS>(v, c, mine, lsig, lc, &mmr);
            if (mine) { m = mm; mr = mmr; }
        }
        if constexpr (COUNT) {
            if (s.valid && !in_exact) {
                if (!s.have_box) {
                    s.b = decode_compact<D>(s.sig, g, c);
                    s.have_box = true;
                }
                in_exact = box_has_stamp<D>(v.stamp, g, s.b, (int)round - 1);
            }
        }
        if constexpr (CLS) {
            // sup over the box of g(x,y,u) + V(y): G off the class, Gc on it; a part
            // without cells holds the neutral kKeyMin; fl(g + .) is monotone, so
            // each part's sup is g + its max
            if (!s.valid || m == kKeyInf || mr == kKeyInf) continue;
            long long dk = kKeyMin;
            if (m != kKeyMin) dk = key_of(gv + val_of(m));
            if (mr != kKeyMin) dk = max(dk, key_of(gr + val_of(mr)));
            if (dk < best) { best = dk; bu = u; }
        } else {
            if (!s.valid || m == kKeyInf) continue;          // +inf + G = +inf
            const long long dk = key_of(gv + val_of(m));     // the one FP64 add
            if (dk < best) { best = dk; bu = u; }
        }
    }
}

// Plane kernel (compact records with a plane shape table, at most
// kPlaneUMax inputs): per warp a shared-memory copy of the lookup lists of the
// plane its lanes are on, for the inputs the warp relaxes.
constexpr int kPlaneUMax = 32;
struct PlaneStage {
    int ent[kPlaneUMax][kPlaneEnt];
    unsigned long long rec[kPlaneUMax];
    const long long* tab[kPlaneUMax];    // the table each list reads
};

// The table of list header code t (bits 8.. of the header).
__device__ __forceinline__ const long long* plane_table(const InstView& v, int t) {
    return t == 4 ? v.M33P : (t == 3 ? v.M33 : (t == 2 ? v.M3 : (t == 1 ? v.M2 : v.Vkey)));
}

// Copy the lists, records and list tables of plane p, inputs u0 .. u1 - 1,
// into st (whole warp).
__device__ __forceinline__ void stage_plane(const InstView& v, int p, int u0, int u1, PlaneStage& st) {
    const int lane = threadIdx.x & 31;
    const int n = u1 - u0;
    const int* lists = v.poffs + ((long long)p * v.g.U + u0) * kPlaneEnt;
    const int4* src = reinterpret_cast<const int4*>(lists);
    int4* dst = reinterpret_cast<int4*>(&st.ent[0][0]);
    for (int i = lane; i < n * (kPlaneEnt / 4); i += 32) dst[i] = __ldg(src + i);
    for (int i = lane; i < n; i += 32) {
        st.rec[i] = __ldg(v.shape + (long long)p * v.g.U + u0 + i);
        st.tab[i] = plane_table(v, __ldg(lists + (long long)i * kPlaneEnt) >> 8);
    }
    __syncwarp();
}

// Max over the boxes of the lanes with `mine` set from a staged list.
__device__ __forceinline__ long long plane_gather_s(const InstView& v, long long c, bool mine, const int* ent,
                                                    int hdr) {
    const int L4 = ((hdr & 0xFF) + 3) & ~3;
    const long long* base = plane_table(v, hdr >> 8) + c;
    const int4* o4 = reinterpret_cast<const int4*>(ent + 4);
    long long m0 = kKeyMin, m1 = kKeyMin, m2 = kKeyMin, m3 = kKeyMin;
    for (int i = 0; i < L4; i += 4) {
        const int4 o = o4[i >> 2];
        if (mine) {
            const long long a0 = __ldg(base + o.x), a1 = __ldg(base + o.y);
            const long long a2 = __ldg(base + o.z), a3 = __ldg(base + o.w);
            m0 = max(m0, a0);
            m1 = max(m1, a1);
            m2 = max(m2, a2);
            m3 = max(m3, a3);
        }
    }
    return max(max(m0, m1), max(m2, m3));
}

// Maxima over the boxes of two inputs' lists at once (all loads of a round
// of four lookups per list are in flight before either max is taken).
__device__ __forceinline__ void plane_gather2(const InstView& v, long long c, bool ma, const int* ea, int ha, bool mb,
                                              const int* eb, int hb, long long& ra, long long& rb) {
    const int La = ((ha & 0xFF) + 3) & ~3, Lb = ((hb & 0xFF) + 3) & ~3;
    const long long* pa = plane_table(v, ha >> 8) + c;
    const long long* pb = plane_table(v, hb >> 8) + c;
    const int4* oa4 = reinterpret_cast<const int4*>(ea + 4);
    const int4* ob4 = reinterpret_cast<const int4*>(eb + 4);
    long long xa = kKeyMin, ya = kKeyMin, xb = kKeyMin, yb = kKeyMin;
    const int L = La > Lb ? La : Lb;
    for (int i = 0; i < L; i += 4) {
        long long a0 = kKeyMin, a1 = kKeyMin, a2 = kKeyMin, a3 = kKeyMin;
        long long b0 = kKeyMin, b1 = kKeyMin, b2 = kKeyMin, b3 = kKeyMin;
        if (i < La) {
            const int4 o = oa4[i >> 2];
            if (ma) {
                a0 = __ldg(pa + o.x); a1 = __ldg(pa + o.y);
                a2 = __ldg(pa + o.z); a3 = __ldg(pa + o.w);
            }
        }
        if (i < Lb) {
            const int4 o = ob4[i >> 2];
            if (mb) {
                b0 = __ldg(pb + o.x); b1 = __ldg(pb + o.y);
                b2 = __ldg(pb + o.z); b3 = __ldg(pb + o.w);
            }
        }
        xa = max(xa, max(a0, a1));
        ya = max(ya, max(a2, a3));
        xb = max(xb, max(b0, b1));
        yb = max(yb, max(b2, b3));
    }
    ra = max(xa, ya);
    rb = max(xb, yb);
}

// The box maximum of input u for the lanes of a plane group: the staged list
// (lanes whose record is the plane's entry), a warp gather of the shared
// record when its list is too long, or (other records) the box cell by cell.
template <int D>
__device__ __forceinline__ long long plane_box_max(const InstView& v, long long c, bool valid, unsigned long long r,
                                                   const int* ent, int hdr, unsigned long long sr) {
    const bool match = valid && r == sr;
    long long m = kKeyMin;
    if ((hdr & 0xFF) != 0) {
        if (__any_sync(0xFFFFFFFFu, match)) m = plane_gather_s(v, c, match, ent, hdr);
    } else {
        // a list longer than kPlaneMaxLook: one warp gather of the shared record
        const unsigned mm = __ballot_sync(0xFFFFFFFFu, match);
        if (mm) {
            const long long lc = __shfl_sync(0xFFFFFFFFu, (int)c, __ffs(mm) - 1);
            const long long x = box_max_rows<D>(v, c, match, sr, lc);
            if (match) m = x;
        }
    }
    if (valid && !match) m = box_max<D>(v.Vkey, v.g, decode_compact<D>(r, v.g, c));
    return m;
}

// relax_inputs for a warp whose active lanes' cells lie on planes with
// lookup lists: lanes are taken plane by plane (a run of 32 frontier cells
// usually lies on one); a lane whose record is its plane's entry (every
// non-blocked lane, for dynamics invariant along dims 0 and 1) reads the
// staged list; any other lane decodes its box and walks it cell by cell.
// PAIR: inputs go two at a time, the lookups of both in flight together (the
// comparison still takes them in input order: lowest input among equal
// minima).
template <int D, bool COUNT, bool PAIR>
__device__ __forceinline__ void relax_plane(const InstView& v, long long c, bool act, int u0, int u1,
                                            long long round, long long& best, int& bu, bool& in_exact,
                                            PlaneStage& st) {
    const GridDesc& g = v.g;
    const int pl = act ? plane_of_cell<D>(g, c) : -1;
    unsigned pend = __ballot_sync(0xFFFFFFFFu, act);
    const compact_t<D>* rp = reinterpret_cast<const compact_t<D>*>(v.boxes) + c;
    const double* gp = v.Gint + c;
    while (pend) {
        const int p = __shfl_sync(0xFFFFFFFFu, pl, __ffs(pend) - 1);
        const bool grp = act && pl == p;
        pend &= ~__ballot_sync(0xFFFFFFFFu, grp);
        stage_plane(v, p, u0, u1, st);
        if constexpr (!PAIR) {
            // one input at a time; the next input's record and cost are loaded
            // while this one is gathered
            unsigned long long nr = grp ? (unsigned long long)__ldcs(rp + (long long)u0 * g.C) : 0ull;
            double ng = grp ? __ldcs(gp + (long long)u0 * g.C) : 0.0;
            for (int u = u0; u < u1; ++u) {
                const unsigned long long r = nr;
                const double gv = ng;
                if (u + 1 < u1 && grp) {
                    nr = (unsigned long long)__ldcs(rp + (long long)(u + 1) * g.C);
                    ng = __ldcs(gp + (long long)(u + 1) * g.C);
                }
                const bool valid = grp && (rec_byte(r, 1) & 0x7F) != 0;
                if (!__any_sync(0xFFFFFFFFu, valid)) continue;
                const long long m = plane_box_max<D>(v, c, valid, r, st.ent[u - u0], st.ent[u - u0][0],
                                                     st.rec[u - u0]);
                if constexpr (COUNT) {
                    if (valid && !in_exact)
                        in_exact = box_has_stamp<D>(v.stamp, g, decode_compact<D>(r, g, c), (int)round - 1);
                }
                if (!valid || m == kKeyInf) continue;            // +inf + G = +inf
                const long long dk = key_of(gv + val_of(m));     // the one FP64 add
                if (dk < best) { best = dk; bu = u; }
            }
            __syncwarp();                                        // before the stage is overwritten
            continue;
        }
        // the next pair's records and costs are loaded while this pair is gathered
        unsigned long long nr0 = 0ull, nr1 = 0ull;
        double ng0 = 0.0, ng1 = 0.0;
        if (grp) {
            nr0 = (unsigned long long)__ldcs(rp + (long long)u0 * g.C);
            ng0 = __ldcs(gp + (long long)u0 * g.C);
            if (u0 + 1 < u1) {
                nr1 = (unsigned long long)__ldcs(rp + (long long)(u0 + 1) * g.C);
                ng1 = __ldcs(gp + (long long)(u0 + 1) * g.C);
            }
        }
        for (int u = u0; u < u1; u += 2) {
            const bool two = u + 1 < u1;
            const unsigned long long r0 = nr0, r1 = nr1;
            const double g0 = ng0, g1 = ng1;
            if (grp) {
                if (u + 2 < u1) {
                    nr0 = (unsigned long long)__ldcs(rp + (long long)(u + 2) * g.C);
                    ng0 = __ldcs(gp + (long long)(u + 2) * g.C);
                }
                if (u + 3 < u1) {
                    nr1 = (unsigned long long)__ldcs(rp + (long long)(u + 3) * g.C);
                    ng1 = __ldcs(gp + (long long)(u + 3) * g.C);
                }
            }
            const bool v0 = grp && (rec_byte(r0, 1) & 0x7F) != 0;
            const bool v1 = two && grp && (rec_byte(r1, 1) & 0x7F) != 0;
            if (!__any_sync(0xFFFFFFFFu, v0 || v1)) continue;
            const int* e0 = st.ent[u - u0];
            const int* e1 = st.ent[two ? u + 1 - u0 : u - u0];
            const int h0 = e0[0], h1 = two ? e1[0] : 0;
            const unsigned long long s0 = st.rec[u - u0], s1 = two ? st.rec[u + 1 - u0] : 0ull;
            long long m0 = kKeyMin, m1 = kKeyMin;
            const bool f0 = v0 && r0 == s0, f1 = v1 && r1 == s1;
            if ((h0 & 0xFF) != 0 && (h1 & 0xFF) != 0 &&
                __all_sync(0xFFFFFFFFu, f0 == v0 && f1 == v1)) {
                plane_gather2(v, c, f0, e0, h0, f1, e1, h1, m0, m1);
            } else {
                m0 = plane_box_max<D>(v, c, v0, r0, e0, h0, s0);
                if (two) m1 = plane_box_max<D>(v, c, v1, r1, e1, h1, s1);
            }
            if constexpr (COUNT) {
                if (v0 && !in_exact)
                    in_exact = box_has_stamp<D>(v.stamp, g, decode_compact<D>(r0, g, c), (int)round - 1);
                if (v1 && !in_exact)
                    in_exact = box_has_stamp<D>(v.stamp, g, decode_compact<D>(r1, g, c), (int)round - 1);
            }
            if (v0 && m0 != kKeyInf) {                       // +inf + G = +inf
                const long long dk = key_of(g0 + val_of(m0));   // the one FP64 add
                if (dk < best) { best = dk; bu = u; }
            }
            if (v1 && m1 != kKeyInf) {
                const long long dk = key_of(g1 + val_of(m1));
                if (dk < best) { best = dk; bu = u + 1; }
            }
        }
        __syncwarp();                                        // before the stage is overwritten
    }
}

// The inputs u0 <= u < u1 whose pair (c, u) is in the current per-input frontier.
__device__ __forceinline__ unsigned input_frontier(const InstView& v, long long c, int u0, int u1) {
    const unsigned* ub = v.ubits + (long long)v.ctr->ubuf * v.g.U * v.nwords + (c >> 5);
    const int b = (int)(c & 31);
    unsigned m = 0u;
#pragma unroll 4
    for (int u = u0; u < u1; ++u) m |= ((__ldcg(ub + (long long)u * v.nwords) >> b) & 1u) << u;
    return m;
}

// relax_plane driven by the cell masks (fmask): per lane one 8-byte word says
// which inputs have a box with the plane's record (the staged list applies)
// and which have another record; only those pairs load their cost, and only
// the second kind its record.  The inputs some lane of the plane group
// relaxes go K at a time in increasing order with the lookups of all K in
// flight (two per list per step) and the next K costs loaded meanwhile; the
// comparison takes them in input order (lowest input among equal minima).
template <int D, int K>
__device__ __forceinline__ void relax_plane_m(const InstView& v, long long c, bool act, long long pos, int u0,
                                              int u1, long long& best, int& bu, PlaneStage& st) {
    const GridDesc& g = v.g;
    const int pl = act ? plane_of_cell<D>(g, c) : -1;
    const unsigned long long msk = act ? __ldcs(v.fmask + c) : 0ull;
    unsigned range = (u1 >= 32 ? 0xFFFFFFFFu : ((1u << u1) - 1u)) & ~((1u << u0) - 1u);
    // per-input frontier: only the pairs whose box holds a changed cell
    if (v.ubits && act) range &= input_frontier(v, c, u0, u1);
    {
        const unsigned taken = act ? (unsigned)__popc(range) : 0u;
        const unsigned tw = __reduce_add_sync(0xFFFFFFFFu, taken);
        if ((threadIdx.x & 31) == 0 && tw) atomicAdd((unsigned long long*)&v.ctr->pairs, (unsigned long long)tw);
    }
    const double* gp = v.Gint + c;
    unsigned pend = __ballot_sync(0xFFFFFFFFu, act);
    while (pend) {
        const int p = __shfl_sync(0xFFFFFFFFu, pl, __ffs(pend) - 1);
        const bool grp = act && pl == p;
        pend &= ~__ballot_sync(0xFFFFFFFFu, grp);
        const unsigned fast = grp ? (unsigned)msk & range : 0u;
        const unsigned slow = grp ? (unsigned)(msk >> 32) & range : 0u;
        const unsigned mine = fast | slow;
        unsigned todo = __reduce_or_sync(0xFFFFFFFFu, mine);
        if (!todo) continue;
        stage_plane(v, p, u0, u1, st);
        int un[K];
        double gn[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            un[j] = todo ? __ffs(todo) - 1 : -1;
            todo &= todo - 1u;
            gn[j] = (un[j] >= 0 && ((mine >> un[j]) & 1u)) ? __ldcs(gp + (long long)un[j] * g.C) : 0.0;
        }
        while (un[0] >= 0) {
            int uc[K];
            double gc[K];
#pragma unroll
            for (int j = 0; j < K; ++j) {
                uc[j] = un[j];
                gc[j] = gn[j];
            }
#pragma unroll
            for (int j = 0; j < K; ++j) {
                un[j] = todo ? __ffs(todo) - 1 : -1;
                todo &= todo - 1u;
                gn[j] = (un[j] >= 0 && ((mine >> un[j]) & 1u)) ? __ldcs(gp + (long long)un[j] * g.C) : 0.0;
            }
            // lookups of the K staged lists (warp-uniform lengths)
            long long m[K];
            int L[K];
            bool f[K];
            const int* off[K];
            const long long* tb[K];
            int Lmax = 0;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                m[j] = kKeyMin;
                const int e = uc[j] >= 0 ? uc[j] - u0 : 0;
                L[j] = uc[j] >= 0 ? (st.ent[e][0] & 0xFF) : 0;
                f[j] = uc[j] >= 0 && ((fast >> uc[j]) & 1u) && L[j] != 0;
                off[j] = &st.ent[e][4];
                tb[j] = st.tab[e] + c;
                Lmax = L[j] > Lmax ? L[j] : Lmax;
            }
            for (int i = 0; i < Lmax; i += 2) {
                long long a[K], b[K];
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    a[j] = kKeyMin;
                    b[j] = kKeyMin;
                    if (i < L[j]) {
                        // entries past L up to L rounded to 4 repeat the first
                        const int2 o = *reinterpret_cast<const int2*>(off[j] + i);
                        if (f[j]) {
                            a[j] = __ldg(tb[j] + o.x);
                            b[j] = __ldg(tb[j] + o.y);
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < K; ++j) m[j] = max(m[j], max(a[j], b[j]));
            }
            // the rare lanes: another record (box walk) or a list too long
            // for the stage (one warp gather of the plane's record)
#pragma unroll
            for (int j = 0; j < K; ++j) {
                if (uc[j] < 0) continue;
                const bool sj = (slow >> uc[j]) & 1u;
                const bool lj = ((fast >> uc[j]) & 1u) && L[j] == 0;
                if (!__any_sync(0xFFFFFFFFu, sj || lj)) continue;
                const unsigned lm = __ballot_sync(0xFFFFFFFFu, lj);
                if (lm) {
                    const long long lc = __shfl_sync(0xFFFFFFFFu, (int)c, __ffs(lm) - 1);
                    const long long x = box_max_rows<D>(v, c, lj, st.rec[uc[j] - u0], lc);
                    if (lj) m[j] = x;
                }
                if (sj) {
                    const unsigned long long r =
                        (unsigned long long)__ldcs(reinterpret_cast<const compact_t<D>*>(v.boxes) + c +
                                                   (long long)uc[j] * g.C);
                    m[j] = box_max<D>(v.Vkey, g, decode_compact<D>(r, g, c));
                }
            }
#pragma unroll
            for (int j = 0; j < K; ++j) {
                if (uc[j] < 0 || !((mine >> uc[j]) & 1u) || m[j] == kKeyInf) continue;   // +inf + G = +inf
                const long long dk = key_of(gc[j] + val_of(m[j]));                       // the one FP64 add
                if (dk < best) { best = dk; bu = uc[j]; }
            }
        }
        __syncwarp();                                        // before the stage is overwritten
    }
}

// Stage of the pair-queue relax (relax_plane_q), per warp: the lists,
// records and list tables of the plane (inputs u0 .. u1 - 1 at rows u - u0),
// the queue of (lane, input) pairs and the candidate of every pair.
template <int UM>
struct PairStage {
    int ent[UM][kPlaneEnt];
    unsigned long long rec[UM];
    const long long* tab[UM];
    long long cand[UM][32];            // [input - u0][lane]
    unsigned short pairs[UM * 32];     // lane | input << 8, input-major
    int plane, su0, su1;               // what ent / rec / tab hold (plane -1: nothing)
    unsigned longm;                    // inputs whose list did not fit (header 0)
};

// relax_plane_m with the pairs spread over the lanes: the (lane, input) pairs
// the staged lists serve (the lane's record is the plane's entry and the
// per-input frontier, if any, holds the pair) go into a queue, input by
// input; each round the 32 lanes take R pairs each -- consecutive cells of
// one input, so the cost loads and the lookups stay coalesced -- and store
// their candidates; pairs with another record, or a list too long for the
// stage, walk their boxes on their own lanes.  Each lane then takes its
// candidates in input order (strict decrease: the lowest input among equal
// minima), so only the pairs a lane holds cost work, however sparse.
template <int D, int UM, int R>
__device__ __forceinline__ void relax_plane_q(const InstView& v, long long c, bool act, long long pos, int u0,
                                              int u1, long long& best, int& bu, PairStage<UM>& st,
                                              long long& taken) {
    const int lane = threadIdx.x & 31;
    const GridDesc& g = v.g;
    const int pl = act ? plane_of_cell<D>(g, c) : -1;
    const unsigned long long msk = act ? __ldcs(v.fmask + c) : 0ull;
    unsigned range = (u1 >= 32 ? 0xFFFFFFFFu : ((1u << u1) - 1u)) & ~((1u << u0) - 1u);
    if (v.ubits && act) range &= input_frontier(v, c, u0, u1);
    taken += act ? __popc(range) : 0;
    const int ci = (int)c;
    const long long C = g.C;
    const unsigned lt = (1u << lane) - 1u;
    unsigned pend = __ballot_sync(0xFFFFFFFFu, act);
    while (pend) {
        const int p = __shfl_sync(0xFFFFFFFFu, pl, __ffs(pend) - 1);
        const bool grp = act && pl == p;
        pend &= ~__ballot_sync(0xFFFFFFFFu, grp);
        const unsigned fast = grp ? (unsigned)msk & range : 0u;
        const unsigned slow = grp ? (unsigned)(msk >> 32) & range : 0u;
        if (!__any_sync(0xFFFFFFFFu, (fast | slow) != 0u)) continue;
        // stage the plane's lists (rows u - u0), unless the stage holds them
        const int n = u1 - u0;
        if (st.plane != p || st.su0 != u0 || st.su1 != u1) {
            __syncwarp();
            if (lane == 0) { st.plane = p; st.su0 = u0; st.su1 = u1; }
            const int* lists = v.poffs + ((long long)p * g.U + u0) * kPlaneEnt;
            const int4* src = reinterpret_cast<const int4*>(lists);
            int4* dst = reinterpret_cast<int4*>(&st.ent[0][0]);
            for (int i = lane; i < n * (kPlaneEnt / 4); i += 32) dst[i] = __ldg(src + i);
            int hdr = 1;
            for (int i = lane; i < n; i += 32) {
                st.rec[i] = __ldg(v.shape + (long long)p * g.U + u0 + i);
                hdr = __ldg(lists + (long long)i * kPlaneEnt);
                st.tab[i] = plane_table(v, hdr >> 8);
            }
            // inputs whose list did not fit (header 0 on a plane entry with a box)
            const unsigned lm = __ballot_sync(0xFFFFFFFFu, lane < n && (hdr & 0xFF) == 0) << u0;
            if (lane == 0) st.longm = lm;
        }
        __syncwarp();
        const unsigned longm = st.longm;
        const unsigned fl = fast & ~longm;
        const unsigned walk = slow | (fast & longm);
        // queue the list pairs input by input
        int np = 0;
        unsigned todo = __reduce_or_sync(0xFFFFFFFFu, fl);
        while (todo) {
            const int u = __ffs(todo) - 1;
            todo &= todo - 1u;
            const bool has = (fl >> u) & 1u;
            const unsigned b = __ballot_sync(0xFFFFFFFFu, has);
            if (has) st.pairs[np + __popc(b & lt)] = (unsigned short)(lane | (u << 8));
            np += __popc(b);
        }
        __syncwarp();
        for (int k0 = 0; k0 < np; k0 += 32 * R) {
            int s[R], e[R], L[R];
            bool h[R];
            double gv[R];
            const long long* tb[R];
            long long m[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int k = k0 + r * 32 + lane;
                h[r] = k < np;
                const unsigned q = h[r] ? st.pairs[k] : 0u;
                s[r] = (int)(q & 31u);
                const int u = (int)(q >> 8);
                const int cs = __shfl_sync(0xFFFFFFFFu, ci, s[r]);
                e[r] = h[r] ? u - u0 : 0;
                L[r] = h[r] ? (st.ent[e[r]][0] & 0xFF) : 0;
                tb[r] = st.tab[e[r]] + cs;
                gv[r] = h[r] ? __ldcs(v.Gint + (long long)u * C + cs) : 0.0;
                m[r] = kKeyMin;
            }
            int Lm = 0;
#pragma unroll
            for (int r = 0; r < R; ++r) Lm = L[r] > Lm ? L[r] : Lm;
            for (int i = 0; i < Lm; i += 2) {
                long long a[R], b[R];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    a[r] = kKeyMin;
                    b[r] = kKeyMin;
                    if (i < L[r]) {
                        // entries past L up to L rounded to 4 repeat the first
                        const int2 o = *reinterpret_cast<const int2*>(&st.ent[e[r]][4 + i]);
                        a[r] = __ldg(tb[r] + o.x);
                        b[r] = __ldg(tb[r] + o.y);
                    }
                }
#pragma unroll
                for (int r = 0; r < R; ++r) m[r] = max(m[r], max(a[r], b[r]));
            }
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (h[r])    // +inf + G = +inf: no candidate
                    st.cand[e[r]][s[r]] = m[r] == kKeyInf ? kKeyInf : key_of(gv[r] + val_of(m[r]));   // the one FP64 add
        }
        // the rare pairs: another record, or a list too long for the stage
        for (unsigned wk = walk; wk; wk &= wk - 1u) {
            const int u = __ffs(wk) - 1;
            const unsigned long long r =
                ((fast >> u) & 1u) ? st.rec[u - u0]
                                   : (unsigned long long)__ldcs(reinterpret_cast<const compact_t<D>*>(v.boxes) + c +
                                                                (long long)u * C);
            const long long mm = box_max<D>(v.Vkey, g, decode_compact<D>(r, g, c));
            const double gw = __ldcs(v.Gint + (long long)u * C + c);
            st.cand[u - u0][lane] = mm == kKeyInf ? kKeyInf : key_of(gw + val_of(mm));
        }
        __syncwarp();
        for (unsigned mine = fl | walk; mine; mine &= mine - 1u) {
            const int u = __ffs(mine) - 1;
            const long long dk = st.cand[u - u0][lane];
            if (dk < best) { best = dk; bu = u; }
        }
        __syncwarp();                                        // before the stage is overwritten
    }
}

// Write the result of a relaxed cell: Vnew, mu and the changed list; with
// MARK also the predecessor boxes of the changed cells into the next frontier.
template <int D, bool COUNT, bool MARK>
__device__ __forceinline__ void commit_cell(const InstView& v, long long c, long long best, int bu, bool in_exact,
                                            int* exact) {
    const bool changed = bu >= 0;
    if (changed) {
        v.Vnew[c] = best;
        if (v.inplace) v.Vkey[c] = best;         // visible to the rest of this pass
        v.mu[c] = (unsigned char)bu;
    }
    const int slot = warp_append(changed, &v.ctr->nchg);
    if (changed) v.chg[slot] = (int)c;
    if constexpr (COUNT) *exact += __popc(__ballot_sync(0xFFFFFFFFu, in_exact));
    if constexpr (MARK) mark_changed<D>(v, changed ? (int)c : -1, changed);
}

// The frontier-cache place of a lane's cell at frontier position pos.
__device__ __forceinline__ FcLane fc_lane(const InstView& v, long long c, bool act, long long pos, long long round) {
    FcLane f;
    f.pos = act ? pos : v.fc_cap;
    f.hit = false;
    f.old_pos = 0;
    if (act) {
        const long long t = v.fc_tag[c];
        f.hit = (t >> 32) == round + 1 && (t & 0xFFFFFFFFll) < v.fc_cap;
        f.old_pos = t & 0xFFFFFFFFll;
    }
    return f;
}

// Relax cells[first + lane] for lane < count (count <= 32) over all inputs.
// Returns the number of cells relaxed; in counting mode adds the cells of the
// exact F1 (some box holds a cell changed in the previous pass) to *exact.
// MARK: also set the next frontier's bits (no separate propagate launch).
template <int D, int FMT, bool COUNT, bool MARK = false, bool CLS = false, int PLANE = 0, int UM = 16>
__device__ __forceinline__ int relax_chunk(const InstView& v, int first, int count, long long round, int* exact,
                                           void* stv = nullptr, long long* taken = nullptr) {
    PlaneStage* st = reinterpret_cast<PlaneStage*>(stv);
    const int lane = threadIdx.x & 31;
    const bool act = lane < count;
    const long long c = act ? v.cells[first + lane] : 0;
    long long best = act ? v.Vkey[c] : 0;
    int bu = -1;
    bool in_exact = false;
    if constexpr (PLANE >= 5) {
        relax_plane_q<D, UM, PLANE == 6 ? 2 : 1>(v, c, act, first + lane, 0, v.g.U, best, bu,
                                                 *reinterpret_cast<PairStage<UM>*>(stv), *taken);
    } else if constexpr (PLANE >= 3) {
        relax_plane_m<D, PLANE == 4 ? 4 : 2>(v, c, act, first + lane, 0, v.g.U, best, bu, *st);
    } else if constexpr (PLANE != 0) {
        relax_plane<D, COUNT, PLANE == 2>(v, c, act, 0, v.g.U, round, best, bu, in_exact, *st);
    } else if ((FMT == kBoxRecompute || FMT == kBoxHybrid) && v.fc_cap > 0) {
        FcLane fl = fc_lane(v, c, act, first + lane, round);
        relax_inputs<D, FMT, COUNT, CLS>(v, c, act, 0, v.g.U, round, best, bu, in_exact, &fl);
        if (act && fl.pos < v.fc_cap) v.fc_tag[c] = ((round + 2) << 32) | fl.pos;
    } else {
        relax_inputs<D, FMT, COUNT, CLS>(v, c, act, 0, v.g.U, round, best, bu, in_exact);
    }
    commit_cell<D, COUNT, MARK>(v, c, best, bu, in_exact, exact);
    return count < 32 ? count : 32;
}

// Relax slice sl (inputs sl*q .. sl*q+q-1) of chunk ch, one of S slices.  Each
// slice leaves its lanes' candidates in cand_key / cand_u; the warp that
// completes the chunk (arrival counter) takes, slice by slice, the strictly
// smaller candidate -- the same lowest input among the smallest values as one
// warp going through all inputs -- commits the cells and resets the counter.
// Returns the cells relaxed (counted by the completing warp).
template <int D, int FMT, bool COUNT, bool MARK = false, bool CLS = false, int PLANE = 0, int UM = 16>
__device__ __forceinline__ int relax_slice(const InstView& v, int ncur, int ch, int sl, int S, int q, long long round,
                                           int* exact, void* stv = nullptr, long long* taken = nullptr) {
    PlaneStage* st = reinterpret_cast<PlaneStage*>(stv);
    const int lane = threadIdx.x & 31;
    const int first = ch << 5;
    const int count = ncur - first;
    const bool act = lane < count;
    const long long c = act ? v.cells[first + lane] : 0;
    long long best = act ? v.Vkey[c] : 0;
    int bu = -1;
    bool in_exact = false;
    const int u0 = sl * q;
    const int u1 = min(v.g.U, u0 + q);
    FcLane fl;
    const bool fc = (FMT == kBoxRecompute || FMT == kBoxHybrid) && v.fc_cap > 0;
    if constexpr (PLANE >= 5) {
        relax_plane_q<D, UM, PLANE == 6 ? 2 : 1>(v, c, act, first + lane, u0, u1, best, bu,
                                                 *reinterpret_cast<PairStage<UM>*>(stv), *taken);
    } else if constexpr (PLANE >= 3) {
        relax_plane_m<D, PLANE == 4 ? 4 : 2>(v, c, act, first + lane, u0, u1, best, bu, *st);
    } else if constexpr (PLANE != 0) {
        relax_plane<D, COUNT, PLANE == 2>(v, c, act, u0, u1, round, best, bu, in_exact, *st);
    } else if (fc) {
        fl = fc_lane(v, c, act, first + lane, round);
        relax_inputs<D, FMT, COUNT, CLS>(v, c, act, u0, u1, round, best, bu, in_exact, &fl);
    } else {
        relax_inputs<D, FMT, COUNT, CLS>(v, c, act, u0, u1, round, best, bu, in_exact);
    }
    const long long base = (long long)ch * S * 32 + lane;
    v.cand_key[base + (long long)sl * 32] = best;
    v.cand_u[base + (long long)sl * 32] = (bu < 0 ? 0xFFFF : bu) | (in_exact ? 1 << 16 : 0);
    __threadfence();
    __syncwarp();
    int prev = 0;
    if (lane == 0) prev = atomicAdd(v.slice_cnt + ch, 1);
    prev = __shfl_sync(0xFFFFFFFFu, prev, 0);
    if (prev != S - 1) return 0;
    __threadfence();
    long long b = 0;
    int bb = -1;
    bool ex = false;
    for (int t = 0; t < S; ++t) {
        const int cu = __ldcg(v.cand_u + base + (long long)t * 32);
        ex |= (cu >> 16) != 0;
        if ((cu & 0xFFFF) == 0xFFFF) continue;        // no decrease in this slice
        const long long ck = __ldcg(v.cand_key + base + (long long)t * 32);
        if (bb < 0 || ck < b) { b = ck; bb = cu & 0xFFFF; }
    }
    if (lane == 0) v.slice_cnt[ch] = 0;
    // every slice has read this cell's tag: the completing warp writes the new one
    if (fc && act && first + lane < v.fc_cap) v.fc_tag[c] = ((round + 2) << 32) | (first + lane);
    commit_cell<D, COUNT, MARK>(v, c, act ? b : 0, act ? bb : -1, act && ex, exact);
    return count < 32 ? count : 32;
}

// One relax launch of the single solve (whole grid): warps take the chunks
// of 32 frontier cells, or (small frontiers) (chunk, input slice) items.
template <int D, int FMT, bool COUNT, bool MARK, bool CLS, int PLANE = 0, int UM = 16>
__device__ __forceinline__ void relax_pass(const InstView& v) {
    Counters* k = v.ctr;
    if (k->done) return;
    if (!COUNT && v.f1bits && k->ncur >= v.dense_min) return;   // the tile relax takes this pass
    const long long round = k->round;
    const int ncur = k->ncur;
    const int nchunks = (ncur + 31) >> 5;
    const int wpb = blockDim.x >> 5;
    const int nwarps = gridDim.x * wpb;
    const int U = v.g.U;
    long long relaxed = 0;
    int exact = 0;
    // small frontier: split each chunk's inputs over S warps
    int S = 1, q = U;
    if (v.cand_key && v.slice_target > 0 && nchunks > 0 && nchunks < v.slice_target * nwarps) {
        S = min(U, (v.slice_target * nwarps + nchunks - 1) / nchunks);
        q = (U + S - 1) / S;
        S = (U + q - 1) / q;
        if ((long long)nchunks * S * 32 > v.slice_cap) { S = 1; q = U; }
    }
    const int gw = blockIdx.x * wpb + (threadIdx.x >> 5);
    void* st = nullptr;
    if constexpr (PLANE >= 5) {
        extern __shared__ __align__(16) unsigned char plane_smem[];
        PairStage<UM>* ps = reinterpret_cast<PairStage<UM>*>(plane_smem) + (threadIdx.x >> 5);
        if ((threadIdx.x & 31) == 0) ps->plane = -1;                // nothing staged yet
        __syncwarp();
        st = ps;
    } else if constexpr (PLANE != 0) {
        extern __shared__ __align__(16) unsigned char plane_smem[];
        st = reinterpret_cast<PlaneStage*>(plane_smem) + (threadIdx.x >> 5);
    }
    long long taken = 0;
    if (S == 1) {
        for (int ch = gw; ch < nchunks; ch += nwarps)
            relaxed += relax_chunk<D, FMT, COUNT, MARK, CLS, PLANE, UM>(v, ch << 5, ncur - (ch << 5), round,
                                                                        &exact, st, &taken);
    } else {
        const int items = nchunks * S;
        for (int it = gw; it < items; it += nwarps) {
            const int ch = it / S;
            relaxed += relax_slice<D, FMT, COUNT, MARK, CLS, PLANE, UM>(v, ncur, ch, it - ch * S, S, q, round,
                                                                        &exact, st, &taken);
        }
    }
    if constexpr (PLANE >= 5) {
        const unsigned long long tw = __reduce_add_sync(0xFFFFFFFFu, (unsigned)taken);
        if ((threadIdx.x & 31) == 0 && tw) atomicAdd((unsigned long long*)&k->pairs, tw);
    }
    if ((threadIdx.x & 31) == 0) {
        if (relaxed) atomicAdd((unsigned long long*)&k->relaxed, (unsigned long long)relaxed);
        if (COUNT && exact) atomicAdd((unsigned long long*)&k->exact, (unsigned long long)exact);
    }
}

// ---------------------------------------------------------------------------
// window tables
// ---------------------------------------------------------------------------

// Recompute M2 and M3 at cell e from the values at the end of the pass (Vnew,
// equal to V on every cell not changed in it; entries past a non-periodic
// row end take the max over the part inside the row; boxes never read them).
__device__ __forceinline__ void table_entry(const InstView& v, long long e) {
    const GridDesc& g = v.g;
    const int n0 = g.n[0];
    const long long row = (long long)grid_div(g, 0, (unsigned)e) * n0;
    const int x = (int)(e - row);
    const bool cls = v.rmask != nullptr;
    const long long m = v.Vnew[e];
    const bool in = cls && v.rmask[e];
    long long m2 = (cls && in) ? kKeyMin : m, m3 = m2;
    long long r2 = in ? m : kKeyMin, r3 = r2;
    if (cls) {
        v.VN[e] = m2;
        v.VR[e] = r2;
    }
    for (int j = 1; j < 3; ++j) {
        int xj = x + j;
        if (xj >= n0) {
            if (!g.periodic[0]) break;
            xj -= n0;
        }
        const long long val = v.Vnew[row + xj];
        const bool inj = cls && v.rmask[row + xj];
        const long long vn = inj ? kKeyMin : val;
        if (j == 1) m2 = max(m2, vn);
        m3 = max(m3, vn);
        if (cls) {
            const long long vr = inj ? val : kKeyMin;
            if (j == 1) r2 = max(r2, vr);
            r3 = max(r3, vr);
        }
    }
    v.M2[e] = m2;
    v.M3[e] = m3;
    if (cls) {
        v.M2R[e] = r2;
        v.M3R[e] = r3;
    }
}

// Refresh the entries whose window holds the changed cell y (e = y-2 .. y,
// inside its row or wrapping on a periodic dim 0).
// Recompute M33 at cell e from Vnew: the max over cells e0 .. e0 + 2 on dim
// 0 and e1 .. e1 + 2 on dim 1 (wrapping on periodic dims; the part inside the
// grid past a non-periodic edge, where no box reads it).
// base: cell (0, 0) of the entry's dims-0/1 plane; x0, x1: its coordinates.
__device__ __forceinline__ void table33_at(const InstView& v, long long base, int x0, int x1) {
    const GridDesc& g = v.g;
    const int n0 = g.n[0], n1 = g.n[1];
    long long m = kKeyMin;
    for (int b = 0; b < 3 && b < n1; ++b) {
        int r = x1 + b;
        if (r >= n1) {
            if (!g.periodic[1]) break;
            r -= n1;
        }
        const long long* row = v.Vnew + base + (long long)r * n0;
        for (int a = 0; a < 3 && a < n0; ++a) {
            int c = x0 + a;
            if (c >= n0) {
                if (!g.periodic[0]) break;
                c -= n0;
            }
            m = max(m, row[c]);
        }
    }
    v.M33[base + (long long)x1 * n0 + x0] = m;
}

__device__ __forceinline__ void table33_entry(const InstView& v, long long e) {
    const GridDesc& g = v.g;
    const int n0 = g.n[0], n1 = g.n[1];
    const long long rowq = (long long)grid_div(g, 0, (unsigned)e);
    const int x0 = (int)(e - rowq * n0);
    const int x1 = (int)(rowq - (long long)grid_div(g, 1, (unsigned)rowq) * n1);
    table33_at(v, e - x0 - (long long)x1 * n0, x0, x1);
}

// The nine 3 x 3 window maxima of Vnew holding cell (x, x1) of the dims-0/1
// plane whose cell (0, 0) is base: out[b][a] = the window starting at
// (x - a, x1 - b).  Vnew is read once over the 5 x 5 block around the cell
// (cells outside a non-periodic edge count as kKeyMin, periodic dims wrap):
// 3-cell row windows first, then 3-row column windows.
__device__ __forceinline__ void windows33(const InstView& v, long long base, int x, int x1, long long out[3][3],
                                          long long* row2 = nullptr) {
    const GridDesc& g = v.g;
    const int n0 = g.n[0], n1 = g.n[1];
    long long w3[5][3];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        int r = x1 - 2 + i;
        bool rin = true;
        if (r < 0) { if (g.periodic[1]) r += n1; else rin = false; }
        else if (r >= n1) { if (g.periodic[1]) r -= n1; else rin = false; }
        if (rin && (r < 0 || r >= n1)) r = ((r % n1) + n1) % n1;   // n1 < 3 on a periodic dim
        long long cv[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            int c = x - 2 + k;
            bool cin = rin;
            if (c < 0) { if (g.periodic[0]) c += n0; else cin = false; }
            else if (c >= n0) { if (g.periodic[0]) c -= n0; else cin = false; }
            if (cin && (c < 0 || c >= n0)) c = ((c % n0) + n0) % n0;
            cv[k] = cin ? v.Vnew[base + (long long)r * n0 + c] : kKeyMin;
        }
        if (row2 && i == 2)
#pragma unroll
            for (int k = 0; k < 5; ++k) row2[k] = cv[k];
#pragma unroll
        for (int a = 0; a < 3; ++a) w3[i][a] = max(cv[2 - a], max(cv[3 - a], cv[4 - a]));
    }
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) out[b][a] = max(w3[2 - b][a], max(w3[3 - b][a], w3[4 - b][a]));
}

// Write max(p[b][a], q[b][a]) to the window entries starting at (x - a,
// x1 - b) of the plane at base (those inside a non-periodic edge).
__device__ __forceinline__ void write33(const InstView& v, long long* t, long long base, int x, int x1,
                                        const long long p[3][3], const long long q[3][3]) {
    const GridDesc& g = v.g;
    const int n0 = g.n[0], n1 = g.n[1];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        int r = x1 - b;
        if (r < 0) {
            if (!g.periodic[1]) break;
            r += n1;
            if (r < 0) break;                     // n1 < 3: the entry repeats
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int c = x - a;
            if (c < 0) {
                if (!g.periodic[0]) break;
                c += n0;
                if (c < 0) break;
            }
            t[base + (long long)r * n0 + c] = max(p[b][a], q[b][a]);
        }
    }
}

// M33P at cell e from M33 (set-up, after every M33 entry is in place).
__device__ __forceinline__ void table33p_entry(const InstView& v, long long e) {
    const GridDesc& g = v.g;
    const int z = v.pz;
    const long long sz = g.stride[z];
    const int kz = (int)((e / sz) % g.n[z]);
    long long m = v.M33[e];
    if (kz + 1 < g.n[z]) m = max(m, v.M33[e + sz]);
    else if (g.periodic[z]) m = max(m, v.M33[e - (long long)kz * sz]);
    v.M33P[e] = m;
}

__device__ __forceinline__ void refresh_tables(const InstView& v, long long y) {
    const GridDesc& g = v.g;
    const int n0 = g.n[0];
    const long long rq = (long long)grid_div(g, 0, (unsigned)y);
    const long long row = rq * n0;
    const int x = (int)(y - row);
    if (!v.M33 || v.rmask) {
        for (int j = 0; j < 3 && j < n0; ++j) {
            int xe = x - j;
            if (xe < 0) {
                if (!g.periodic[0]) break;
                xe += n0;
            }
            table_entry(v, row + xe);
        }
    }
    if (v.M33) {
        const int n1 = g.n[1];
        const int x1 = (int)(rq - (long long)grid_div(g, 1, (unsigned)rq) * n1);
        const long long base = row - (long long)x1 * n0;
        long long mid[3][3], r2[5];
        windows33(v, base, x, x1, mid, r2);
        // M2 / M3 at x - j from y's row of the block (cells x - 2 .. x + 2)
        for (int j = 0; j < 3 && j < n0; ++j) {
            int xe = x - j;
            if (xe < 0) {
                if (!g.periodic[0]) break;
                xe += n0;
            }
            const long long a = r2[2 - j], b = r2[3 - j], c3 = r2[4 - j];
            v.M2[row + xe] = max(a, b);
            v.M3[row + xe] = max(a, max(b, c3));
        }
        write33(v, v.M33, base, x, x1, mid, mid);
        if (v.M33P) {
            // the pair entries holding y's plane: (plane z, z + 1) and (z - 1, z)
            const int z = v.pz;
            const long long sz = g.stride[z];
            const int nz = g.n[z];
            const int kz = (int)((y / sz) % nz);
            long long nb[3][3];
            int zp = kz + 1;
            if (zp >= nz) zp = g.periodic[z] ? zp - nz : -1;
            if (zp >= 0) windows33(v, base + (long long)(zp - kz) * sz, x, x1, nb);
            write33(v, v.M33P, base, x, x1, mid, zp >= 0 ? nb : mid);
            int zm = kz - 1;
            if (zm < 0) zm = g.periodic[z] ? zm + nz : -1;
            if (zm >= 0 && zm != kz) {
                windows33(v, base + (long long)(zm - kz) * sz, x, x1, nb);
                write33(v, v.M33P, base + (long long)(zm - kz) * sz, x, x1, nb, mid);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// compaction of the upcoming frontier (whole block)
// ---------------------------------------------------------------------------

// Words [w_begin, min(w_end, w_begin + blockDim.x)) of fbits: their set bits
// become consecutive entries of `cells` (in cell order within the block) and
// the words are cleared.  One atomicAdd on nnext per block.
__device__ __forceinline__ void compact_words(const InstView& v, int w_begin, int w_end) {
    __shared__ int warp_sum[32];
    __shared__ int block_base;
    const int t = threadIdx.x;
    const int lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
    const int wd = w_begin + t;
    unsigned bits = 0;
    if (wd < w_end) {
        if (v.ubits) {
            // per-input frontier: a cell is in the upcoming frontier when some
            // input's bit is set; the current buffer (read by this pass's
            // relax) is cleared for the pass after next
            const int U = v.g.U;
            const int cur = v.ctr->ubuf;
            const unsigned* nx = v.ubits + (long long)(cur ^ 1) * U * v.nwords + wd;
            unsigned* cu = v.ubits + (long long)cur * U * v.nwords + wd;
#pragma unroll 4
            for (int u = 0; u < U; ++u) {
                bits |= nx[(long long)u * v.nwords];
                cu[(long long)u * v.nwords] = 0u;
            }
        } else {
            bits = v.fbits[wd];
            if (bits) v.fbits[wd] = 0u;
        }
        if (v.f1bits) v.f1bits[wd] = bits;
    }
    const int cnt = __popc(bits);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += x;
    }
    if (lane == 31) warp_sum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int s = lane < nw ? warp_sum[lane] : 0;
        int si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xFFFFFFFFu, si, o);
            if (lane >= o) si += x;
        }
        if (lane < nw) warp_sum[lane] = si - s;          // exclusive per warp
        if (lane == 31) block_base = si > 0 ? atomicAdd(&v.ctr->nnext, si) : 0;
    }
    __syncthreads();
    int pos = block_base + warp_sum[wid] + incl - cnt;
    const long long cbase = (long long)wd << 5;
    while (bits) {
        const int b = __ffs(bits) - 1;
        bits &= bits - 1;
        v.cells[pos++] = (int)(cbase + b);
    }
    __syncthreads();                                      // before warp_sum / block_base are reused
}

// ---------------------------------------------------------------------------
// pass end
// ---------------------------------------------------------------------------

// Close a pass (one thread): trace, counters, loop condition.  The next
// frontier holds nnext cells.
__device__ __forceinline__ int finish_pass(const InstView& v) {
    Counters* k = v.ctr;
    const long long r = k->round;
    if (v.trace && r < v.trace_cap) {
        long long* t = v.trace + r * 4;
        t[0] = k->relaxed;
        t[1] = k->nchg;
        t[2] = (k->ncur + 31) / 32;
        t[3] = v.stamp ? k->exact : -1;
    }
    k->total_relaxed += k->relaxed;
    k->total_exact += k->exact;
    k->total_pairs += k->pairs;
    k->pairs = 0;
    k->total_changed += k->nchg;
    k->relaxed = 0;
    k->exact = 0;
    k->nchg = 0;
    k->round = r + 1;
    const int next = k->nnext;
    k->ncur = next;
    k->nnext = 0;
    if (v.ubits) k->ubuf ^= 1;
    const int cont = (next > 0 && r + 1 < k->cap) ? 1 : 0;
    if (!cont) {
        k->done = 1;
        k->status = next == 0 ? BF_CONVERGED : (r + 1 >= v.g.C ? BF_NEG_CYCLE : BF_ITER_CAP);
    }
    return cont;
}

// After the set-up's compaction: F1 holds nnext cells; decide whether to loop.
__device__ __forceinline__ int start_loop(const InstView& v) {
    Counters* k = v.ctr;
    k->nchg = 0;
    k->ncur = k->nnext;
    k->nnext = 0;
    if (v.ubits) k->ubuf ^= 1;
    const int cont = (k->err == 0 && k->ncur > 0 && k->cap > 0) ? 1 : 0;
    if (!cont) {
        k->done = 1;
        k->status = k->ncur == 0 ? BF_CONVERGED : BF_ITER_CAP;
    }
    return cont;
}

// Last-block detection: true in exactly one thread (thread 0 of the last
// block of the grid to arrive), after the writes of every block are visible
// to it.  The counter is reset for the next launch.
__device__ __forceinline__ bool last_block_done(unsigned* counter) {
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
        if (last) {
            __threadfence();
            *counter = 0u;
        }
    }
    __syncthreads();
    return last && threadIdx.x == 0;
}

}  // namespace bfk
