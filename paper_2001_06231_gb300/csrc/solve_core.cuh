// solve_core.cuh -- per-warp device routines of Algorithm 1 (Sec. IV-A),
// shared by the single-instance solver (solve.cu) and the batched engine
// (batch.cu).
//
// Frontiers.  The upcoming frontier F2 is a bitmap with one bit per cell; a
// 32-bit word covers one segment of 32 consecutive cells.  A word that turns
// non-zero during a pass is appended (once) to the segment list of the next
// pass, so F1 of the next pass is the list of non-zero words.
//
// One pass of the while-loop is two kernels:
//   relax      warp per active segment, lanes = its 32 cells; for every cell
//              whose bit is set and u = 0..U-1:
//              d = G(x,u) + max_{y in F(x,u)} V(y) (one FP64 add, max on keys),
//              keep the lowest u with the smallest d; if d < V(x) write
//              Vnew(x), mu(x) and append x to the changed list (ballot + one
//              atomicAdd per warp).  V is read-only in this kernel, which
//              makes the pass synchronous (Jacobi).
//   propagate  warp per changed cell y: commit V(y) = Vnew(y) and set the
//              bits of y's predecessor box (F2 = union of pred of the changed
//              cells); lanes take the box's dim-0 runs, one word read per run
//              and an atomicOr only where bits are still clear.  The last block to finish swaps the
//              frontiers, counts the pass and evaluates the loop condition
//              F1 != empty and i < cap.
#pragma once
#include "bf_internal.cuh"
#include "dynamics.cuh"

namespace bfk {

struct Counters {
    int nseg[2];              // active segments per frontier (ping-pong by pass parity)
    int nchg;                 // cells changed in the current pass
    int err;                  // nonzero: invalid input seen during set-up
    long long round;          // passes completed (i of Algorithm 1)
    long long cap;            // |X| or the caller's smaller cap
    long long relaxed;        // cells relaxed in the current pass
    long long total_relaxed;  // summed over passes
    long long exact;          // cells of the exact F1 in the current pass (counting mode)
    long long total_exact;
    long long total_changed;
    unsigned blocks_done;     // blocks of the running propagate launch that finished
    int done;                 // loop condition became false
    int status;               // BF_CONVERGED / BF_NEG_CYCLE / BF_ITER_CAP
    int pad;
};

struct InstView {
    GridDesc g;
    DynDesc dd;
    const void* boxes;          // [U][C] records, or NULL in recompute mode
    const double* inputs;       // [U][udim] (recompute mode)
    const short* pred;          // [C][2D] predecessor offsets
    const double* Gint;         // [U][C] running cost, +inf on avoid cells
    long long* Vkey;            // [C] current values (keys)
    long long* Vnew;            // [C] values decided in the current pass
    unsigned char* mu;          // [C]
    unsigned* fbits;            // [S] upcoming-frontier bitmap (bit = cell)
    int* seglist0;              // [S] active segments, even passes
    int* seglist1;              // [S] odd passes
    int* chg;                   // [C] changed cells of the current pass
    Counters* ctr;
    long long* trace;           // [trace_cap][4] or NULL
    long long trace_cap;
    int* stamp;                 // [C] pass that last changed the cell (counting mode) or NULL
};

__device__ __forceinline__ int* seglist_of(const InstView& v, int par) {
    return par ? v.seglist1 : v.seglist0;
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

// max over the box of V for a whole warp whose valid lanes hold boxes of the
// same shape relative to their cells (same offset `base` of the lower corner
// from the cell, same widths `wpack`, no periodic wrap): element e of lane l
// sits at V[c_l + base + off(e)] with off(e) the same for every lane.  Lane e
// computes off(e) once; the gather loop broadcasts it with a shuffle, so
// every element is one coalesced warp load, with four loads in flight.
template <int D>
__device__ __forceinline__ long long box_max_uniform(const long long* __restrict__ V, const GridDesc& g,
                                                     long long c, bool valid, int base, unsigned wpack) {
    const int lane = threadIdx.x & 31;
    const int w0 = wpack & 0xFF;
    const int w1 = D > 1 ? (wpack >> 8) & 0xFF : 1;
    const int w2 = D > 2 ? (wpack >> 16) & 0xFF : 1;
    const int w3 = D > 3 ? (wpack >> 24) & 0xFF : 1;
    const int vol = w0 * w1 * w2 * w3;
    const long long* p = V + (valid ? c + base : 0);
    long long m0 = kKeyMin, m1 = kKeyMin;
    for (int e0 = 0; e0 < vol; e0 += 32) {
        const int e = e0 + lane;
        int off = 0;
        if (e < vol) {
            int t = e;
            off = t % w0;
            t /= w0;
            if (D > 1) { off += (int)((t % w1) * g.stride[1]); t /= w1; }
            if (D > 2) { off += (int)((t % w2) * g.stride[2]); t /= w2; }
            if (D > 3) { off += (int)(t * g.stride[3]); }
        }
        const int n = min(32, vol - e0);
        int k = 0;
        for (; k + 4 <= n; k += 4) {
            const int o0 = __shfl_sync(0xFFFFFFFFu, off, k);
            const int o1 = __shfl_sync(0xFFFFFFFFu, off, k + 1);
            const int o2 = __shfl_sync(0xFFFFFFFFu, off, k + 2);
            const int o3 = __shfl_sync(0xFFFFFFFFu, off, k + 3);
            if (valid) {
                const long long a0 = __ldg(p + o0), a1 = __ldg(p + o1);
                const long long a2 = __ldg(p + o2), a3 = __ldg(p + o3);
                m0 = max(m0, max(a0, a2));
                m1 = max(m1, max(a1, a3));
            }
        }
        for (; k < n; ++k) {
            const int o = __shfl_sync(0xFFFFFFFFu, off, k);
            if (valid) m0 = max(m0, __ldg(p + o));
        }
    }
    return max(m0, m1);
}

template <int D, bool RECOMP>
__device__ __forceinline__ Box<D> fetch_box(const InstView& v, long long c, int u, bool act) {
    Box<D> b;
    if (act) {
        if constexpr (RECOMP) b = make_box<D>(v.dd, v.g, v.inputs, c, u);
        else b = load_box<D>(v.boxes, (long long)u * v.g.C + c);
    } else {
        b.lo[0] = kBlocked;
#pragma unroll
        for (int d = 1; d < D; ++d) b.lo[d] = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) b.hi[d] = 0;
    }
    return b;
}

// Relax one segment (lanes = 32 consecutive cells).  Returns the number of
// cells relaxed; in counting mode also adds the cells of the exact F1 (some
// box holds a cell changed in the previous pass) to *exact.
//
// Per input the warp first checks whether every valid lane's box has the same
// shape relative to its cell (same linear offset of the lower corner, same
// widths, no periodic wrap inside the box).  That holds for dynamics that are
// translation invariant along the grid (the built-in systems away from
// boundaries); the warp then gathers with box_max_uniform.  Otherwise every
// lane walks its own box.  The next input's box and this input's cost are
// loaded ahead of the gather.
template <int D, bool RECOMP, bool COUNT>
__device__ __forceinline__ int relax_segment(const InstView& v, int seg, long long round, int* exact) {
    const int lane = threadIdx.x & 31;
    const GridDesc& g = v.g;
    const long long c = (long long)seg * 32 + lane;
    const unsigned word = v.fbits[seg];
    const bool act = (word >> lane) & 1u;            // bits are set only for cells < C
    if (lane == 0) v.fbits[seg] = 0u;
    long long best = 0;
    int bu = -1;
    bool in_exact = false;
    if (act) best = v.Vkey[c];
    Box<D> nb = fetch_box<D, RECOMP>(v, c, 0, act);
    for (int u = 0; u < g.U; ++u) {
        const Box<D> b = nb;
        if (u + 1 < g.U) nb = fetch_box<D, RECOMP>(v, c, u + 1, act);
        const bool valid = b.lo[0] != kBlocked;     // blocked: overflow set, d = +inf
        double gv = 0.0;
        if (valid) gv = __ldcs(v.Gint + (long long)u * g.C + c);
        // shape signature relative to the cell
        int base = 0;
        unsigned wpack = 0;
        bool odd = false;
        if (valid) {
            long long lin = 0;
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const int w = b.hi[d] - b.lo[d] + 1;
                lin += (long long)b.lo[d] * g.stride[d];
                wpack |= (unsigned)(w & 0xFF) << (8 * d);
                odd |= w > 255;
                odd |= g.periodic[d] && (b.lo[d] + w > g.n[d]);
            }
            base = (int)(lin - c);
        }
        const unsigned vmask = __ballot_sync(0xFFFFFFFFu, valid);
        if (!vmask) continue;
        const int leader = __ffs(vmask) - 1;
        const int lbase = __shfl_sync(0xFFFFFFFFu, base, leader);
        const unsigned lw = __shfl_sync(0xFFFFFFFFu, wpack, leader);
        const bool same = !valid || (!odd && base == lbase && wpack == lw);
        long long m;
        if (__all_sync(0xFFFFFFFFu, same)) {
            m = box_max_uniform<D>(v.Vkey, g, c, valid, lbase, lw);
        } else {
            m = valid ? box_max<D>(v.Vkey, g, b) : kKeyInf;
        }
        if constexpr (COUNT) {
            if (valid && !in_exact) in_exact = box_has_stamp<D>(v.stamp, g, b, (int)round - 1);
        }
        if (!valid || m == kKeyInf) continue;          // +inf + G = +inf
        const long long dk = key_of(gv + val_of(m));   // the one FP64 add
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
    return __popc(word);
}

// Set the bits `mask` of word wd of the upcoming frontier.  The word is
// read first and updated with atomicOr only when some of its bits are still
// clear: the predecessor boxes of neighbouring changed cells overlap, so most
// marks end at the read.  Bits only go from 0 to 1 within a propagate launch,
// so a stale (L1) read can only cost a redundant atomic, never skip a needed
// one.  Returns true when this lane turned the word from 0 to non-zero.
__device__ __forceinline__ bool mark_word(unsigned* fbits, int wd, unsigned mask) {
    if ((fbits[wd] & mask) == mask) return false;
    return atomicOr(&fbits[wd], mask) == 0u;
}

// Commit one changed cell y and set the bits of its predecessor box (a whole
// warp; lanes take the rows of the box, i.e. its dim-0 runs).  `par` is the
// parity of the segment list being filled.
template <int D>
__device__ __forceinline__ void propagate_cell(const InstView& v, int y, int par, bool commit) {
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
    int* list = seglist_of(v, par);
    int* cnt = &v.ctr->nseg[par];
    const int n0 = g.n[0];
    // dim-0 run [a0, e0] (same for every row); on a periodic dim 0 the part
    // past n0 - 1 wraps to the start of the row
    const int a0 = lo[0], e0 = lo[0] + len[0] - 1;
    const int e1 = min(e0, n0 - 1);
    const bool wrap = e0 >= n0;
    for (int r0 = 0; r0 < rows; r0 += 32) {
        const int r = r0 + lane;
        long long rowbase = 0;
        const bool on = r < rows;
        if (on) {
            int t = r;
#pragma unroll
            for (int d = 1; d < D; ++d) {
                const int j = t % len[d];
                t /= len[d];
                int xd = lo[d] + j;
                if (g.periodic[d] && xd >= g.n[d]) xd -= g.n[d];
                rowbase += (long long)xd * g.stride[d];
            }
        }
        // words of the run(s): [rowbase + a0, rowbase + e1] and, if wrapping,
        // [rowbase, rowbase + e0 - n0]
        for (int part = 0; part < (wrap ? 2 : 1); ++part) {
            const long long a = rowbase + (part ? 0 : a0);
            const long long b = rowbase + (part ? e0 - n0 : e1);
            const int wa = (int)(a >> 5);
            const int nw = on ? (int)(b >> 5) - wa + 1 : 0;
            const int nmax = (int)__reduce_max_sync(0xFFFFFFFFu, (unsigned)nw);
            for (int k = 0; k < nmax; ++k) {
                const int wd = wa + k;
                bool fresh = false;
                if (k < nw) {
                    const long long lo_b = max(a, (long long)wd << 5);
                    const long long hi_b = min(b, ((long long)wd << 5) + 31);
                    const int s = (int)(lo_b & 31), e = (int)(hi_b & 31);
                    const unsigned mask = (e == 31 ? 0xFFFFFFFFu : ((1u << (e + 1)) - 1u)) & ~((1u << s) - 1u);
                    fresh = mark_word(v.fbits, wd, mask);
                }
                const int slot = warp_append(fresh, cnt);
                if (fresh) list[slot] = wd;
            }
        }
    }
}

// End of a pass (one thread): trace, frontier swap, loop condition.
__device__ __forceinline__ int finish_pass(const InstView& v) {
    Counters* k = v.ctr;
    const long long r = k->round;
    const int par = (int)(r & 1);
    if (v.trace && r < v.trace_cap) {
        long long* t = v.trace + r * 4;
        t[0] = k->relaxed;
        t[1] = k->nchg;
        t[2] = k->nseg[par];
        t[3] = v.stamp ? k->exact : -1;
    }
    k->total_relaxed += k->relaxed;
    k->total_exact += k->exact;
    k->total_changed += k->nchg;
    k->relaxed = 0;
    k->exact = 0;
    k->nseg[par] = 0;
    k->nchg = 0;
    k->round = r + 1;
    const int next = k->nseg[par ^ 1];
    const int cont = (next > 0 && r + 1 < k->cap) ? 1 : 0;
    if (!cont) {
        k->done = 1;
        k->status = next == 0 ? BF_CONVERGED : (r + 1 >= v.g.C ? BF_NEG_CYCLE : BF_ITER_CAP);
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
