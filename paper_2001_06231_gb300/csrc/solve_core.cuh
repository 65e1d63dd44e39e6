// solve_core.cuh -- per-warp device routines of Algorithm 1 (Sec. IV-A),
// shared by the single-instance solver (solve.cu) and the batched engine
// (batch.cu).
//
// One pass of the while-loop is two kernels:
//   relax      for every active segment (32 consecutive cells, lanes = cells)
//              and every flagged cell x in it: for u = 0..U-1,
//              d = G(x,u) + max_{y in F(x,u)} V(y) (one FP64 add; max on keys),
//              keep the lowest u with the smallest d; if d < V(x) write
//              Vnew(x), mu(x) and append x to the changed list (ballot +
//              one atomicAdd per warp).  V is read-only in this kernel, which
//              makes the pass synchronous (Jacobi).
//   propagate  for every changed y: commit V(y) = Vnew(y) and flag every cell
//              of y's predecessor box for the next pass (F2 = union of pred of
//              changed cells); a segment whose flag goes 0 -> 1 is appended to
//              the next segment list.
// A third one-thread step swaps the frontiers, counts the pass and evaluates
// the loop condition F1 != empty and i < cap.
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
    long long relaxed;        // flagged cells relaxed in the current pass
    long long total_relaxed;  // summed over passes
    int done;                 // loop condition became false
    int status;               // BF_CONVERGED / BF_NEG_CYCLE / BF_ITER_CAP
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
    unsigned char* flag;        // [C] cell is in the next frontier
    unsigned* segflag;          // [nseg_total] segment is in the next list
    int* seglist0;              // [nseg_total]
    int* seglist1;
    int* chg;                   // [C] changed cells of the current pass
    Counters* ctr;
    long long* trace;           // [trace_cap][4] or NULL
    long long trace_cap;
};

__device__ __forceinline__ int* seglist_of(const InstView& v, int par) {
    return par ? v.seglist1 : v.seglist0;
}

// Relax one segment; returns the number of cells relaxed (warp-uniform).
template <int D, bool RECOMP>
__device__ __forceinline__ int relax_segment(const InstView& v, int seg) {
    const int lane = threadIdx.x & 31;
    const GridDesc& g = v.g;
    const long long c = (long long)seg * 32 + lane;
    bool act = false;
    if (c < g.C) act = v.flag[c] != 0;
    if (act) v.flag[c] = 0;
    if (lane == 0) v.segflag[seg] = 0u;
    long long best = 0;
    int bu = -1;
    if (act) {
        best = v.Vkey[c];
        for (int u = 0; u < g.U; ++u) {
            const long long p = (long long)u * g.C + c;
            Box<D> b;
            if constexpr (RECOMP) b = make_box<D>(v.dd, g, v.inputs, c, u);
            else b = load_box<D>(v.boxes, p);
            if (b.lo[0] == kBlocked) continue;            // overflow set: d = +inf
            const long long m = box_max<D>(v.Vkey, g, b);
            if (m == kKeyInf) continue;                    // +inf + G = +inf
            const double gv = __ldcs(v.Gint + p);
            const long long dk = key_of(gv + val_of(m));   // the one FP64 add
            if (dk < best) { best = dk; bu = u; }
        }
    }
    const bool changed = bu >= 0;
    if (changed) {
        v.Vnew[c] = best;
        v.mu[c] = (unsigned char)bu;
    }
    const int slot = warp_append(changed, &v.ctr->nchg);
    if (changed) v.chg[slot] = (int)c;
    return __popc(__ballot_sync(0xFFFFFFFFu, act));
}

// Commit one changed cell y and flag its predecessor box.  `par` is the
// parity of the segment list being filled.  Called by a whole warp.
template <int D>
__device__ __forceinline__ void propagate_cell(const InstView& v, int y, int par, bool commit) {
    const int lane = threadIdx.x & 31;
    const GridDesc& g = v.g;
    if (commit && lane == 0) v.Vkey[y] = v.Vnew[y];
    const short* q = v.pred + (long long)y * (2 * D);
    int lo[D], len[D];
    int total = 1;
    if (q[0] > q[D]) return;                      // y has no predecessor
    int ky[4];
    cell_coords(g, y, ky);
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const int n = g.n[d];
        int l = q[d], h = q[D + d];
        int len_d = h - l + 1;
        if (g.periodic[d]) {
            if (len_d >= n) { lo[d] = 0; len_d = n; }
            else { int s = ky[d] + l; s %= n; if (s < 0) s += n; lo[d] = s; }
        } else {
            lo[d] = ky[d] + l;
        }
        len[d] = len_d;
        total *= len_d;
    }
    int* list = seglist_of(v, par);
    int* cnt = &v.ctr->nseg[par];
    for (int base = 0; base < total; base += 32) {
        const int t = base + lane;
        bool mark = false;
        int seg = 0;
        if (t < total) {
            int r = t;
            long long x = 0;
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const int j = r % len[d];
                r /= len[d];
                int xd = lo[d] + j;
                if (g.periodic[d] && xd >= g.n[d]) xd -= g.n[d];
                x += (long long)xd * g.stride[d];
            }
            if (v.flag[x] == 0) v.flag[x] = 1;
            seg = (int)(x >> 5);
            if (v.segflag[seg] == 0u) mark = atomicExch(&v.segflag[seg], 1u) == 0u;
        }
        const int slot = warp_append(mark, cnt);
        if (mark) list[slot] = seg;
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
        t[3] = k->relaxed * v.g.U;
    }
    k->total_relaxed += k->relaxed;
    k->relaxed = 0;
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

}  // namespace bfk
