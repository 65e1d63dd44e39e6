// solve_core.cuh -- per-warp / per-block device routines of Algorithm 1
// (Sec. IV-A), shared by the single solve (solve.cu), the batched engine
// (batch.cu, serve.cu) and the allocation-free solve (noalloc.cu).
//
// State of one instance (InstView):
//   Vkey        int64 [C]  W as order-preserving keys (bf_internal.cuh)
//   M2, M3      int64 [C]  window maxima along dim 0: M2(y) = max(V(y), V(y+1)),
//                          M3(y) = max(V(y..y+2)) (wrapping on a periodic dim 0),
//                          equal to V's windows at the start of every pass
//   fbits       u32 [S]    upcoming frontier F2, one bit per cell
//   cells       i32 [C]    current frontier F1 as a compacted cell list
//   chg         i32 [C]    cells whose W decreased in the current pass
//
// One pass of the while-loop is three kernels:
//   relax      warp per 32 cells of F1 (lanes = cells): for u = 0..U-1,
//              d = G(x,u) + max_{y in F(x,u)} V(y) (one FP64 add, max on keys),
//              lowest u among the smallest d; if d < W(x): Vnew(x), mu(x) and
//              append x to chg.  V and the tables are read-only here, so the
//              pass is synchronous (Jacobi).
//   propagate  warp per changed cell y: commit W(y) = Vnew(y), set the bits of
//              y's predecessor box in fbits (F2 = union of pred of the
//              changed cells).
//   compact    block per 256 bitmap words: F2's bits -> the cell list of the
//              next pass (ordered within a block; bits cleared on the way);
//              threads also refresh the window maxima around every changed
//              cell; the last block closes the pass (trace, i += 1, loop
//              condition F1 != empty and i < cap).
//
// Box gather.  For a pair whose box spans w0 cells along dim 0, one row of
// the box is max over [lo0, lo0 + w0): one table lookup for w0 <= 3 (V, M2 or
// M3) and ceil(w0 / 3) overlapping M3 lookups beyond.  When all lanes of a
// warp hold boxes of the same shape relative to their cells (true for
// dynamics invariant under translation along the grid, such as the built-in
// systems), every lookup is one warp load at a lane-independent offset from
// each lane's cell and the loops are warp-uniform.  Other warps walk each
// lane's box cell by cell.
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
    long long total_changed;
    unsigned blocks_done;     // blocks of the running compact launch that finished
    int done;                 // loop condition became false
    int status;               // BF_CONVERGED / BF_NEG_CYCLE / BF_ITER_CAP
    int pad;
};

struct InstView {
    GridDesc g;
    DynDesc dd;
    int box_fmt;                // kBoxWide / kBoxCompact / kBoxRecompute
    const void* boxes;          // [U][C] records (wide or compact) or NULL
    const double* inputs;       // [U][udim] (recompute mode)
    const short* pred;          // [C][2D] predecessor offsets
    const double* Gint;         // [U][C] running cost, +inf on avoid cells
    long long* Vkey;            // [C]
    long long* Vnew;            // [C]
    long long* M2;              // [C]
    long long* M3;              // [C]
    unsigned char* mu;          // [C]
    unsigned* fbits;            // [S]
    int* cells;                 // [C]
    int* chg;                   // [C]
    Counters* ctr;
    long long* trace;           // [trace_cap][4] or NULL
    long long trace_cap;
    int* stamp;                 // [C] pass that last changed the cell (counting mode) or NULL
};

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
    v.boxes = a->d_boxes;
    v.inputs = a->d_inputs;
    v.pred = a->d_pred;
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

// Max of V over the box with the window tables, for a warp whose valid lanes
// share the box shape: lower corner at c + base, widths w0..w3.  The lookups
// (row x piece) are enumerated with warp-uniform counters, 8 per round so
// that 8 loads are in flight.
template <int D>
__device__ __forceinline__ long long box_max_rows(const InstView& v, long long c, bool valid, int base, int w0,
                                                  int w1, int w2, int w3) {
    const GridDesc& g = v.g;
    const long long* tab = w0 == 1 ? v.Vkey : (w0 == 2 ? v.M2 : v.M3);
    const int np = w0 < 3 ? 1 : (w0 + 2) / 3;            // lookups per row
    const int total = np * w1 * w2 * w3;
    const int s1 = (int)g.stride[1], s2 = (int)g.stride[2], s3 = (int)g.stride[3];
    const long long* p = tab + (valid ? c + base : 0);
    long long m[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) m[k] = kKeyMin;
    int jp = 0, j1 = 0, j2 = 0, j3 = 0;
    for (int e = 0; e < total; e += 8) {
        int off[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            off[k] = (w0 < 3 ? 0 : min(3 * jp, w0 - 3)) + j1 * s1 + j2 * s2 + j3 * s3;
            if (++jp == np) {
                jp = 0;
                if (++j1 == w1) {
                    j1 = 0;
                    if (++j2 == w2) { j2 = 0; ++j3; }
                }
            }
        }
        if (valid) {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (e + k < total) m[k] = max(m[k], __ldg(p + off[k]));
        }
    }
    return max(max(max(m[0], m[1]), max(m[2], m[3])), max(max(m[4], m[5]), max(m[6], m[7])));
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
// relax
// ---------------------------------------------------------------------------

// Per-lane view of the pair (x, u): validity, shape signature, offset of the
// lower corner from the cell, widths, and the absolute box when needed.
template <int D>
struct PairShape {
    bool valid;               // the lane holds a cell and the pair is not blocked
    bool odd;                 // box wraps or is too wide: gather cell by cell
    bool have_box;            // b holds the absolute box
    unsigned long long sig;   // equal signatures + equal base <=> same relative box
    int base;
    int w[4];
    Box<D> b;
};

template <int D, int FMT>
__device__ __forceinline__ void pair_shape(const InstView& v, long long c, int u, bool act, PairShape<D>& s) {
    const GridDesc& g = v.g;
    s.valid = false;
    s.odd = false;
    s.have_box = false;
    s.sig = 0;
    s.base = 0;
#pragma unroll
    for (int d = 0; d < 4; ++d) s.w[d] = 1;
    if (!act) return;
    if constexpr (FMT == kBoxCompact) {
        const unsigned long long r =
            (unsigned long long)__ldcs(reinterpret_cast<const compact_t<D>*>(v.boxes) + (long long)u * g.C + c);
        const int f0 = rec_byte(r, 1);
        if ((f0 & 0x7F) == 0) return;                 // blocked
        s.valid = true;
        s.sig = r;
        s.odd = (f0 & 0x80) != 0;
        int base = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            s.w[d] = rec_byte(r, 2 * d + 1) & 0x7F;
            base += rec_sbyte(r, 2 * d) * (int)g.stride[d];
        }
        s.base = base;
    } else {
        Box<D> b;
        if constexpr (FMT == kBoxRecompute) b = make_box<D>(v.dd, g, v.inputs, c, u);
        else b = load_box<D>(v.boxes, (long long)u * g.C + c);
        if (b.lo[0] == kBlocked) return;
        s.valid = true;
        s.have_box = true;
        s.b = b;
        long long lin = 0;
        unsigned long long wp = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int w = b.hi[d] - b.lo[d] + 1;
            s.w[d] = w;
            lin += (long long)b.lo[d] * g.stride[d];
            wp |= (unsigned long long)(w & 0xFFFF) << (16 * d);
            s.odd |= w > 0xFFFF;
            s.odd |= g.periodic[d] && (b.lo[d] + w > g.n[d]);
        }
        s.base = (int)(lin - c);
        s.sig = wp;
    }
}

// Relax cells[first + lane] for lane < count (count <= 32).  Returns the
// number of cells relaxed; in counting mode adds the cells of the exact F1
// (some box holds a cell changed in the previous pass) to *exact.
template <int D, int FMT, bool COUNT>
__device__ __forceinline__ int relax_chunk(const InstView& v, int first, int count, long long round, int* exact) {
    const int lane = threadIdx.x & 31;
    const GridDesc& g = v.g;
    const bool act = lane < count;
    const long long c = act ? v.cells[first + lane] : 0;
    long long best = 0;
    int bu = -1;
    bool in_exact = false;
    if (act) best = v.Vkey[c];
    // the next input's record and cost are loaded while this one is gathered
    PairShape<D> nx;
    pair_shape<D, FMT>(v, c, 0, act, nx);
    double ngv = nx.valid ? __ldcs(v.Gint + c) : 0.0;
    for (int u = 0; u < g.U; ++u) {
        PairShape<D> s = nx;
        const double gv = ngv;
        if (u + 1 < g.U) {
            pair_shape<D, FMT>(v, c, u + 1, act, nx);
            ngv = nx.valid ? __ldcs(v.Gint + (long long)(u + 1) * g.C + c) : 0.0;
        }
        const unsigned vmask = __ballot_sync(0xFFFFFFFFu, s.valid);
        if (!vmask) continue;
        const int leader = __ffs(vmask) - 1;
        const unsigned long long lsig = shfl_u64(s.sig, leader);
        const int lbase = __shfl_sync(0xFFFFFFFFu, s.base, leader);
        const bool same = !s.valid || (!s.odd && s.sig == lsig && s.base == lbase);
        long long m;
        if (__all_sync(0xFFFFFFFFu, same)) {
            int lw[4];
#pragma unroll
            for (int d = 0; d < 4; ++d) lw[d] = __shfl_sync(0xFFFFFFFFu, s.w[d], leader);
            m = box_max_rows<D>(v, c, s.valid, lbase, lw[0], lw[1], lw[2], lw[3]);
        } else {
            if (s.valid && !s.have_box) {
                s.b = decode_compact<D>(s.sig, g, c);
                s.have_box = true;
            }
            m = s.valid ? box_max<D>(v.Vkey, g, s.b) : kKeyInf;
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
        if (!s.valid || m == kKeyInf) continue;          // +inf + G = +inf
        const long long dk = key_of(gv + val_of(m));     // the one FP64 add
        if (dk < best) { best = dk; bu = u; }
    }
    const bool changed = bu >= 0;
    if (changed) {
        v.Vnew[c] = best;
        v.mu[c] = (unsigned char)bu;
    }
    const int slot = warp_append(changed, &v.ctr->nchg);
    if (changed) v.chg[slot] = (int)c;
    if constexpr (COUNT) *exact += __popc(__ballot_sync(0xFFFFFFFFu, in_exact));
    return count < 32 ? count : 32;
}

// ---------------------------------------------------------------------------
// propagate
// ---------------------------------------------------------------------------

// Set the bits `mask` of word wd of the upcoming frontier; the word is read
// first and updated with atomicOr only when some of its bits are still clear
// (the predecessor boxes of neighbouring changed cells overlap, so most marks
// end at the read).  Bits only go from 0 to 1 during propagate, so a stale
// read can only cost a redundant atomic.
__device__ __forceinline__ void mark_word(unsigned* fbits, int wd, unsigned mask) {
    if ((fbits[wd] & mask) != mask) atomicOr(&fbits[wd], mask);
}

__device__ __forceinline__ unsigned bit_range(int s, int e) {
    return (e == 31 ? 0xFFFFFFFFu : ((1u << (e + 1)) - 1u)) & ~((1u << s) - 1u);
}

// Commit one changed cell y and set the bits of its predecessor box (a whole
// warp; lanes take the box's rows, i.e. its dim-0 runs).
template <int D>
__device__ __forceinline__ void propagate_cell(const InstView& v, int y, bool commit) {
    const int lane = threadIdx.x & 31;
    const GridDesc& g = v.g;
    if (commit && lane == 0) {
        v.Vkey[y] = v.Vnew[y];
        if (v.stamp) v.stamp[y] = (int)v.ctr->round;
    }
    const short* q = v.pred + (long long)y * (2 * D);
    if (q[0] > q[D]) return;                      // y has no predecessor (warp-uniform)
    int ky[4];
    cell_coords(g, y, ky);
    int lo[D], len[D];
    int rows = 1;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const int n = g.n[d];
        int len_d = q[D + d] - q[d] + 1;
        if (g.periodic[d]) {
            if (len_d >= n) { lo[d] = 0; len_d = n; }
            else { int s = (ky[d] + q[d]) % n; if (s < 0) s += n; lo[d] = s; }
        } else {
            lo[d] = ky[d] + q[d];
        }
        len[d] = len_d;
        if (d > 0) rows *= len_d;
    }
    const int n0 = g.n[0];
    const int a0 = lo[0], e0 = lo[0] + len[0] - 1;
    const int e1 = min(e0, n0 - 1);
    const bool wrap = e0 >= n0;                   // periodic dim 0: the part past n0 - 1 wraps
    for (int r = lane; r < rows; r += 32) {
        int t = r;
        long long rowbase = 0;
#pragma unroll
        for (int d = 1; d < D; ++d) {
            const int j = t % len[d];
            t /= len[d];
            int xd = lo[d] + j;
            if (g.periodic[d] && xd >= g.n[d]) xd -= g.n[d];
            rowbase += (long long)xd * g.stride[d];
        }
        for (int part = 0; part < (wrap ? 2 : 1); ++part) {
            const long long a = rowbase + (part ? 0 : a0);
            const long long b = rowbase + (part ? e0 - n0 : e1);
            for (long long wd = a >> 5; wd <= (b >> 5); ++wd) {
                const long long lo_b = max(a, wd << 5), hi_b = min(b, (wd << 5) + 31);
                mark_word(v.fbits, (int)wd, bit_range((int)(lo_b & 31), (int)(hi_b & 31)));
            }
        }
    }
}

// ---------------------------------------------------------------------------
// window tables
// ---------------------------------------------------------------------------

// Recompute M2 and M3 at cell e from V (entries past a non-periodic row end
// take the max over the part inside the row; boxes never read them).
__device__ __forceinline__ void table_entry(const InstView& v, long long e) {
    const GridDesc& g = v.g;
    const int n0 = g.n[0];
    const long long row = e - (e % n0);
    const int x = (int)(e - row);
    const long long m = v.Vkey[e];
    long long m2 = m, m3 = m;
    for (int j = 1; j < 3; ++j) {
        int xj = x + j;
        if (xj >= n0) {
            if (!g.periodic[0]) break;
            xj -= n0;
        }
        const long long val = v.Vkey[row + xj];
        if (j == 1) m2 = max(m2, val);
        m3 = max(m3, val);
    }
    v.M2[e] = m2;
    v.M3[e] = m3;
}

// Refresh the entries whose window holds the changed cell y (e = y-2 .. y,
// inside its row or wrapping on a periodic dim 0).
__device__ __forceinline__ void refresh_tables(const InstView& v, long long y) {
    const GridDesc& g = v.g;
    const int n0 = g.n[0];
    const long long row = y - (y % n0);
    const int x = (int)(y - row);
    for (int j = 0; j < 3 && j < n0; ++j) {
        int xe = x - j;
        if (xe < 0) {
            if (!g.periodic[0]) break;
            xe += n0;
        }
        table_entry(v, row + xe);
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
        bits = v.fbits[wd];
        if (bits) v.fbits[wd] = 0u;
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
    k->total_changed += k->nchg;
    k->relaxed = 0;
    k->exact = 0;
    k->nchg = 0;
    k->round = r + 1;
    const int next = k->nnext;
    k->ncur = next;
    k->nnext = 0;
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
