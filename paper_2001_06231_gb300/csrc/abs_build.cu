// abs_build.cu -- discrete abstraction on the device (Sec. V-B, Def.
// abstraction) and the predecessor index of Eq. (pred), plus the abstraction
// handle API of bfgpu.h.
//
// K1 build:    one thread per (cell, input), consecutive threads take
//              consecutive cells of one input, so the [U][C] box records are
//              written coalesced.  FP64 throughout (RK4 + growth bound).
// K2 pred:     one thread per (cell x, input u) walks the cells y of its box
//              and widens y's predecessor bounding box (offsets x - y per
//              dim) with read-check-then-atomicMin/Max; the plain read skips
//              the atomic whenever the bound already covers x (bounds only
//              widen, so a stale read never wrongly skips).  The result is
//              the bounding box of pred(y) = {x : exists u, y in F(x,u)}:
//              a superset of Eq. (pred), which the algorithm tolerates (the
//              paper notes pred may be replaced by a superset, Sec. V-B).
// K12 check:   validation of caller-supplied boxes; counts malformed records.
#include <cstdarg>
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>
#include <string>
#include <vector>

#include "bf_internal.cuh"
#include "dynamics.cuh"
#include "solve_core.cuh"

using namespace bfk;

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
namespace bfh {
static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

int cuda_fail(cudaError_t e, const char* what) {
    set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
    return e == cudaErrorMemoryAllocation ? BF_ERR_OOM : BF_ERR_CUDA;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
}  // namespace bfh

extern "C" const char* bf_last_error(void) { return bfh::g_err.c_str(); }

static int grid_blocks(long long work, int threads) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long need = (work + threads - 1) / threads;
    long long cap = (long long)sms * 16;
    if (need < 1) need = 1;
    return (int)(need < cap ? need : cap);
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
template <int D>
__global__ void k_build_boxes(DynDesc dd, GridDesc g, const double* __restrict__ inputs, void* boxes) {
    const long long total = g.C * g.U;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const int u = (int)(p / g.C);
        const long long c = p - (long long)u * g.C;
        Box<D> b = make_box<D>(dd, g, inputs, c, u);
        store_box<D>(boxes, p, b);
    }
}

// Shared RK4 parts of every (coordinates on dims >= 2, input) pair for the
// recompute mode (rk4_shared_part; key = k2 + n2 k3).
template <int D>
__global__ void k_rk_table(DynDesc dd, GridDesc g, const double* __restrict__ inputs, long long nkeys,
                           double* table) {
    const long long total = nkeys * g.U;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const long long key = p / g.U;
        const int u = (int)(p - key * g.U);
        const int k2 = (int)(key % g.n[2]);
        const int k3 = (int)(key / g.n[2]);
        double ckey[2];
        ckey[0] = dd.glo[2] + ((double)k2 + 0.5) * dd.eta[2];
        ckey[1] = D >= 4 ? dd.glo[3] + ((double)k3 + 0.5) * dd.eta[3] : 0.0;
        double* e = table + p * kRkEntry;
        rk4_shared_part<D>(dd, inputs + (long long)u * dd.udim, ckey, reinterpret_cast<double (*)[2]>(e),
                           e + 2 * kRkMaxSub, e + 2 * kRkMaxSub + 2);
    }
}

// external [C][U][2][D] -> internal [U][C] records, with validation
template <int D>
__global__ void k_import_boxes(GridDesc g, const short* __restrict__ ext, void* boxes,
                               unsigned long long* nbad) {
    const long long total = g.C * g.U;
    unsigned long long bad = 0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const int u = (int)(p / g.C);
        const long long c = p - (long long)u * g.C;
        const short* e = ext + (c * g.U + u) * (2 * D);
        Box<D> b;
#pragma unroll
        for (int d = 0; d < D; ++d) { b.lo[d] = e[d]; b.hi[d] = e[D + d]; }
        if (b.lo[0] == kBlocked) {
#pragma unroll
            for (int d = 1; d < D; ++d) b.lo[d] = 0;
#pragma unroll
            for (int d = 0; d < D; ++d) b.hi[d] = 0;
        } else {
            bool ok = true;
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const int n = g.n[d];
                if (b.lo[d] < 0 || b.lo[d] >= n || b.hi[d] < b.lo[d]) ok = false;
                if (g.periodic[d]) { if (b.hi[d] - b.lo[d] + 1 > n) ok = false; }
                else if (b.hi[d] >= n) ok = false;
            }
            if (!ok) {
                ++bad;
                b.lo[0] = kBlocked;
            }
        }
        store_box<D>(boxes, p, b);
    }
    if (bad) atomicAdd(nbad, bad);
}

template <int D>
__global__ void k_export_boxes(GridDesc g, DynDesc dd, const double* __restrict__ inputs,
                               const void* __restrict__ boxes, int fmt, int nstored, short* ext) {
    const long long total = g.C * g.U;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const int u = (int)(p / g.C);
        const long long c = p - (long long)u * g.C;
        Box<D> b;
        if (fmt == kBoxWide) {
            b = load_box<D>(boxes, p);
        } else if (fmt == kBoxRecompute || (fmt == kBoxHybrid && u >= nstored)) {
            b = make_box<D>(dd, g, inputs, c, u);
        } else {
            const unsigned long long r = D <= 2 ? reinterpret_cast<const unsigned*>(boxes)[p]
                                                : reinterpret_cast<const unsigned long long*>(boxes)[p];
            if (((r >> 8) & 0x7F) == 0) {
                b.lo[0] = kBlocked;
#pragma unroll
                for (int d = 1; d < D; ++d) b.lo[d] = 0;
#pragma unroll
                for (int d = 0; d < D; ++d) b.hi[d] = 0;
            } else {
                int k[4];
                cell_coords(g, c, k);
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    const int w = (int)((r >> (16 * d + 8)) & 0x7F);
                    int lo = k[d] + (int)(signed char)((r >> (16 * d)) & 0xFF);
                    if (g.periodic[d]) {
                        if (lo < 0) lo += g.n[d];
                        else if (lo >= g.n[d]) lo -= g.n[d];
                    }
                    b.lo[d] = lo;
                    b.hi[d] = lo + w - 1;
                }
            }
        }
        short* e = ext + (c * g.U + u) * (2 * D);
#pragma unroll
        for (int d = 0; d < D; ++d) { e[d] = (short)b.lo[d]; e[D + d] = (short)b.hi[d]; }
    }
}

// Wide absolute records -> compact relative records (see solve_core.cuh):
// per dim the lower corner relative to the cell (int8, periodic dims reduced
// to [-n/2, n/2)) and the width (1..127); width 0 on dim 0 = blocked; bit 7
// of dim 0's width byte = the box wraps around a periodic dim for this cell.
// Sets *fail when some box does not fit the format.
template <int D>
__device__ __forceinline__ unsigned long long encode_compact(const GridDesc& g, long long c, const Box<D>& b,
                                                             bool& bad) {
    unsigned long long rec = 0;
    if (b.lo[0] == kBlocked) return 0;
    int k[4];
    cell_coords(g, c, k);
    bool wrap = false;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const int n = g.n[d];
        const int w = b.hi[d] - b.lo[d] + 1;
        int rel = b.lo[d] - k[d];
        if (g.periodic[d]) {
            rel %= n;
            if (rel < 0) rel += n;
            if (rel >= n - n / 2) rel -= n;
            wrap |= (k[d] + rel < 0) || (k[d] + rel + w > n);
        }
        bad |= w > 127 || rel < -128 || rel > 127;
        rec |= (unsigned long long)(unsigned char)(signed char)rel << (16 * d);
        rec |= (unsigned long long)(w & 0x7F) << (16 * d + 8);
    }
    if (wrap) rec |= 0x80ull << 8;
    return rec;
}

template <int D>
__device__ __forceinline__ void store_compact(void* compact, long long p, unsigned long long rec) {
    if (D <= 2) reinterpret_cast<unsigned*>(compact)[p] = (unsigned)rec;
    else reinterpret_cast<unsigned long long*>(compact)[p] = rec;
}

template <int D>
__global__ void k_to_compact(GridDesc g, const void* __restrict__ wide, void* compact, int* fail) {
    const long long total = g.C * g.U;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const int u = (int)(p / g.C);
        const long long c = p - (long long)u * g.C;
        bool bad = false;
        const unsigned long long rec = encode_compact<D>(g, c, load_box<D>(wide, p), bad);
        if (bad) atomicExch(fail, 1);
        store_compact<D>(compact, p, rec);
    }
}

// Boxes of the first g.U inputs built straight into compact records (the
// hybrid mode's stored part); sets *fail when some box does not fit.
template <int D>
__global__ void k_build_compact(DynDesc dd, GridDesc g, const double* __restrict__ inputs, void* compact,
                                int* fail) {
    const long long total = g.C * g.U;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const int u = (int)(p / g.C);
        const long long c = p - (long long)u * g.C;
        bool bad = false;
        const unsigned long long rec = encode_compact<D>(g, c, make_box<D>(dd, g, inputs, c, u), bad);
        if (bad) atomicExch(fail, 1);
        store_compact<D>(compact, p, rec);
    }
}

// Plane shape table.  A plane is the set of cells with equal coordinates on
// dims >= 2 (the whole grid for D = 2); p = x / stride[2].  For dynamics
// invariant under translation along dims 0 and 1 (the built-in unicycle and
// fire models, whose right-hand sides do not depend on x and y) every
// non-blocked pair (x, u) of a plane has the same relative record.  The entry
// of (plane, input) is picked in up to three rounds, each taking the record of
// the lowest cell not excluded: the first non-blocked record; where that one
// is shared by less than half of the pairs, the lowest record that differs
// from it; where neither is, the lowest that differs from both.  The pick
// more pairs share stays (the earlier one on a tie), so the table does not
// depend on the order threads run in.  Records that differ from the entry are
// counted.
__device__ __forceinline__ long long plane_of(const GridDesc& g, long long x) {
    if (g.D <= 2) return 0;
    return (long long)grid_div(g, 1, grid_div(g, 0, (unsigned)x));
}

template <int D>
__device__ __forceinline__ unsigned long long compact_at(const void* compact, long long p) {
    return D <= 2 ? (unsigned long long)reinterpret_cast<const unsigned*>(compact)[p]
                  : reinterpret_cast<const unsigned long long*>(compact)[p];
}

// Per entry the lowest cell whose pair is non-blocked and whose record is
// neither ex1's nor ex2's entry (NULL: none), skipping the entries flagged in
// skip (or NULL); idx starts at all ones.
template <int D>
__global__ void k_shape_first(GridDesc g, const void* __restrict__ compact, unsigned* idx,
                              const unsigned long long* __restrict__ ex1, const unsigned long long* __restrict__ ex2,
                              const unsigned char* __restrict__ skip) {
    const long long total = g.C * g.U;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const int u = (int)(p / g.C);
        const long long x = p - (long long)u * g.C;
        const unsigned long long rec = compact_at<D>(compact, p);
        if (((rec >> 8) & 0x7F) == 0) continue;                // blocked
        const long long e = plane_of(g, x) * g.U + u;
        if (skip && skip[e]) continue;
        if ((ex1 && rec == ex1[e]) || (ex2 && rec == ex2[e])) continue;
        if ((unsigned)x < idx[e]) atomicMin(idx + e, (unsigned)x);
    }
}

// The records at the picked cells (0 where none was picked).
template <int D>
__global__ void k_shape_take(GridDesc g, const void* __restrict__ compact, const unsigned* __restrict__ idx,
                             long long n, unsigned long long* out) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        out[e] = idx[e] == 0xFFFFFFFFu ? 0ull : compact_at<D>(compact, (e % g.U) * g.C + idx[e]);
}

// Per entry the non-blocked pairs (nb, unless NULL) and those whose record is
// the entry's (hit); one atomic per group of lanes with the same entry.
template <int D>
__global__ void k_shape_count(GridDesc g, const void* __restrict__ compact, const unsigned long long* __restrict__ shape,
                              unsigned* hit, unsigned* nb) {
    const long long total = g.C * g.U;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long rounds = (total + stride - 1) / stride;
    const int lane = threadIdx.x & 31;
    for (long long it = 0; it < rounds; ++it) {
        const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x + it * stride;
        long long e = -1;
        bool h = false;
        if (p < total) {
            const int u = (int)(p / g.C);
            const long long x = p - (long long)u * g.C;
            const unsigned long long rec = compact_at<D>(compact, p);
            if (((rec >> 8) & 0x7F) != 0) {
                e = plane_of(g, x) * g.U + u;
                h = rec == shape[e];
            }
        }
        const unsigned grp = __match_any_sync(0xFFFFFFFFu, e);
        const unsigned hm = __ballot_sync(0xFFFFFFFFu, h) & grp;
        if (e >= 0 && lane == __ffs(grp) - 1) {
            if (nb) atomicAdd(nb + e, (unsigned)__popc(grp));
            if (hm) atomicAdd(hit + e, (unsigned)__popc(hm));
        }
    }
}

// Keep the later pick where more pairs share it (its hits into best).
__global__ void k_shape_choose(long long n, unsigned long long* shape, const unsigned long long* __restrict__ later,
                               unsigned* best, const unsigned* __restrict__ hit) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        if (later[e] != 0ull && hit[e] > best[e]) {
            shape[e] = later[e];
            best[e] = hit[e];
        }
}

__global__ void k_shape_retry(long long n, const unsigned* __restrict__ hit, const unsigned* __restrict__ nb,
                              unsigned char* skip) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        skip[e] = (2ull * hit[e] >= nb[e]) ? 1 : 0;
}

// Lookup lists of every (plane, input) of the shape table (thread per entry).
template <int D>
__global__ void k_plane_lists(GridDesc g, const unsigned long long* __restrict__ shape, long long P, int m33,
                              int pz, int* out) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < P * g.U;
         e += (long long)gridDim.x * blockDim.x)
        plane_offsets<D>(g, shape[e], (int)(e / g.U), m33 != 0, pz, out + e * kPlaneEnt);
}

// Cell masks (thread per cell, U <= 32): bit u when the pair (c, u) has a box
// whose record is its plane's entry, bit 32 + u when it has another record.
template <int D>
__global__ void k_cell_masks(GridDesc g, const void* __restrict__ compact, const unsigned long long* __restrict__ shape,
                             unsigned long long* out) {
    const compact_t<D>* rec = reinterpret_cast<const compact_t<D>*>(compact);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.C;
         c += (long long)gridDim.x * blockDim.x) {
        const long long p = plane_of_cell<D>(g, c);
        unsigned long long m = 0;
        for (int u = 0; u < g.U; ++u) {
            const unsigned long long r = (unsigned long long)rec[(long long)u * g.C + c];
            if ((rec_byte(r, 1) & 0x7F) == 0) continue;          // no box
            m |= (r == shape[p * g.U + u]) ? (1ull << u) : (1ull << (32 + u));
        }
        out[c] = m;
    }
}

template <int D>
__global__ void k_shape_check(GridDesc g, const void* __restrict__ compact, const unsigned long long* shape,
                              unsigned long long* mismatch) {
    const long long total = g.C * g.U;
    unsigned long long bad = 0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const int u = (int)(p / g.C);
        const long long x = p - (long long)u * g.C;
        const unsigned long long rec = compact_at<D>(compact, p);
        if (((rec >> 8) & 0x7F) == 0) continue;
        if (rec != shape[plane_of(g, x) * g.U + u]) ++bad;
    }
    if (bad) atomicAdd(mismatch, bad);
}

__global__ void k_fill_i32(int* a, long long n, int v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        a[i] = v;
}

template <int D>
__global__ void k_pred_scatter(GridDesc g, DynDesc dd, const double* __restrict__ inputs,
                               const void* __restrict__ boxes, int* plo, int* phi) {
    const long long total = g.C * g.U;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const int u = (int)(p / g.C);
        const long long x = p - (long long)u * g.C;
        Box<D> b = boxes ? load_box<D>(boxes, p) : make_box<D>(dd, g, inputs, x, u);
        if (b.lo[0] == kBlocked) continue;
        int kx[4];
        cell_coords(g, x, kx);
        int len[D], cnt = 1;
#pragma unroll
        for (int d = 0; d < D; ++d) { len[d] = b.hi[d] - b.lo[d] + 1; cnt *= len[d]; }
        for (int t = 0; t < cnt; ++t) {
            int r = t;
            long long y = 0;
            int off[D];
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const int j = r % len[d];
                r /= len[d];
                int yd = b.lo[d] + j;
                const int n = g.n[d];
                if (g.periodic[d] && yd >= n) yd -= n;
                y += (long long)yd * g.stride[d];
                int o = kx[d] - yd;
                if (g.periodic[d]) {
                    o %= n;
                    if (o < 0) o += n;
                    if (o >= n - n / 2) o -= n;   // o in [-(n/2), n - n/2 - 1]
                }
                off[d] = o;
            }
#pragma unroll
            for (int d = 0; d < D; ++d) {
                int* lo = plo + (long long)d * g.C + y;
                int* hi = phi + (long long)d * g.C + y;
                if (*((volatile int*)lo) > off[d]) atomicMin(lo, off[d]);
                if (*((volatile int*)hi) < off[d]) atomicMax(hi, off[d]);
            }
        }
    }
}

template <int D>
__global__ void k_pred_pack(GridDesc g, const int* __restrict__ plo, const int* __restrict__ phi,
                            short* pred) {
    for (long long y = blockIdx.x * (long long)blockDim.x + threadIdx.x; y < g.C;
         y += (long long)gridDim.x * blockDim.x) {
        short* q = pred + y * (2 * D);
        if (plo[y] > phi[y]) {          // no predecessor at all
#pragma unroll
            for (int d = 0; d < D; ++d) { q[d] = 32767; q[D + d] = -32768; }
            continue;
        }
#pragma unroll
        for (int d = 0; d < D; ++d) {
            q[d] = (short)plo[(long long)d * g.C + y];
            q[D + d] = (short)phi[(long long)d * g.C + y];
        }
    }
}

// Sum over cells of the dim-0 rows of the predecessor box, and the number of
// cells that have one: sums[0], sums[1].
template <int D>
__global__ void k_pred_rows(GridDesc g, const short* __restrict__ pred, unsigned long long* sums) {
    unsigned long long rows = 0, cells = 0;
    for (long long y = blockIdx.x * (long long)blockDim.x + threadIdx.x; y < g.C;
         y += (long long)gridDim.x * blockDim.x) {
        const short* q = pred + y * (2 * D);
        if (q[0] > q[D]) continue;
        unsigned long long r = 1;
#pragma unroll
        for (int d = 1; d < D; ++d) r *= (unsigned long long)(q[D + d] - q[d] + 1);
        rows += r;
        cells += 1;
    }
    for (int o = 16; o > 0; o >>= 1) {
        rows += __shfl_down_sync(0xFFFFFFFFu, rows, o);
        cells += __shfl_down_sync(0xFFFFFFFFu, cells, o);
    }
    if ((threadIdx.x & 31) == 0 && cells) {
        atomicAdd(sums, rows);
        atomicAdd(sums + 1, cells);
    }
}

// ---------------------------------------------------------------------------
// host API
// ---------------------------------------------------------------------------
void bf_solve_ws_free(bf_solve_ws* ws);   // solve.cu

static int check_grid(const bf_grid* grid, GridDesc& g) {
    if (!grid || grid->ndim < 1 || grid->ndim > 4) {
        bfh::set_error("grid: ndim must be 1..4");
        return BF_ERR_INVALID;
    }
    memset(&g, 0, sizeof g);
    g.D = grid->ndim;
    long long C = 1;
    for (int d = 0; d < g.D; ++d) {
        if (grid->n[d] < 1 || grid->n[d] > 16383) {
            bfh::set_error("grid: n[%d] = %d outside 1..16383", d, grid->n[d]);
            return BF_ERR_INVALID;
        }
        g.n[d] = grid->n[d];
        g.periodic[d] = grid->periodic[d] ? 1 : 0;
        g.stride[d] = C;
        C *= grid->n[d];
    }
    if (C > (1LL << 31) - 64) {
        bfh::set_error("grid: %lld cells exceed the 2^31 cell limit", C);
        return BF_ERR_INVALID;
    }
    for (int d = g.D; d < 4; ++d) { g.n[d] = 1; g.stride[d] = C; }
    g.C = C;
    grid_divisors(g);
    return BF_OK;
}

static DynDesc make_dyndesc(const bf_abstraction* a) {
    DynDesc dd;
    memset(&dd, 0, sizeof dd);
    dd.kind = a->dyn.kind;
    dd.substeps = a->dyn.rk4_substeps;
    dd.udim = a->udim;
    dd.tau = a->tau;
    for (int i = 0; i < 8; ++i) dd.p[i] = a->dyn.param[i];
    for (int d = 0; d < a->g.D; ++d) {
        dd.glo[d] = a->glo[d];
        dd.eta[d] = (a->ghi[d] - a->glo[d]) / (double)a->g.n[d];
    }
    return dd;
}

static size_t box_bytes(const GridDesc& g) { return (size_t)g.C * g.U * 4 * g.D; }

template <int D>
static int build_pred_t(bf_abstraction* a, cudaStream_t st) {
    const GridDesc& g = a->g;
    int *plo = nullptr, *phi = nullptr;
    BF_CUDA(cudaMallocAsync((void**)&plo, sizeof(int) * g.C * D, st));
    BF_CUDA(cudaMallocAsync((void**)&phi, sizeof(int) * g.C * D, st));
    k_fill_i32<<<grid_blocks(g.C * D, 256), 256, 0, st>>>(plo, g.C * D, 0x7FFFFFFF);
    k_fill_i32<<<grid_blocks(g.C * D, 256), 256, 0, st>>>(phi, g.C * D, (int)0x80000000);
    DynDesc dd = make_dyndesc(a);
    k_pred_scatter<D><<<grid_blocks(g.C * g.U, 256), 256, 0, st>>>(g, dd, a->d_inputs, a->d_boxes, plo, phi);
    k_pred_pack<D><<<grid_blocks(g.C, 256), 256, 0, st>>>(g, plo, phi, a->d_pred);
    BF_CUDA(cudaGetLastError());
    BF_CUDA(cudaFreeAsync(plo, st));
    BF_CUDA(cudaFreeAsync(phi, st));
    // mean predecessor-box rows: how much marking a changed cell costs
    unsigned long long* sums = nullptr;
    unsigned long long h[2] = {0, 0};
    BF_CUDA(cudaMallocAsync((void**)&sums, 2 * sizeof(unsigned long long), st));
    BF_CUDA(cudaMemsetAsync(sums, 0, 2 * sizeof(unsigned long long), st));
    k_pred_rows<D><<<grid_blocks(g.C, 256), 256, 0, st>>>(g, a->d_pred, sums);
    BF_CUDA(cudaGetLastError());
    BF_CUDA(cudaMemcpyAsync(h, sums, sizeof h, cudaMemcpyDeviceToHost, st));
    BF_CUDA(cudaFreeAsync(sums, st));
    BF_CUDA(cudaStreamSynchronize(st));
    a->pred_rows = h[1] ? (double)h[0] / (double)h[1] : 0.0;
    return BF_OK;
}

static int build_pred(bf_abstraction* a, cudaStream_t st) {
    switch (a->g.D) {
        case 1: return build_pred_t<1>(a, st);
        case 2: return build_pred_t<2>(a, st);
        case 3: return build_pred_t<3>(a, st);
        default: return build_pred_t<4>(a, st);
    }
}

// Replace the wide records by compact ones when every box fits the format.
template <int D>
static int to_compact_t(bf_abstraction* a, cudaStream_t st) {
    const size_t rec = D <= 2 ? 4 : 8;
    const size_t bytes = rec * (size_t)a->g.C * a->g.U;
    void* comp = nullptr;
    int* d_fail = nullptr;
    int h_fail = 0;
    BF_CUDA(cudaMalloc(&comp, bytes));
    cudaError_t e = cudaMalloc((void**)&d_fail, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(d_fail, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        k_to_compact<D><<<grid_blocks(a->g.C * a->g.U, 256), 256, 0, st>>>(a->g, a->d_boxes, comp, d_fail);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_fail, d_fail, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_fail);
    if (e != cudaSuccess) { cudaFree(comp); return bfh::cuda_fail(e, "compact box records"); }
    if (h_fail) {                          // keep the wide records
        cudaFree(comp);
        return BF_OK;
    }
    cudaFree(a->d_boxes);
    a->d_boxes = comp;
    a->box_fmt = kBoxCompact;
    a->bytes = a->bytes - box_bytes(a->g) + bytes;
    return BF_OK;
}

static int to_compact(bf_abstraction* a, cudaStream_t st) {
    switch (a->g.D) {
        case 1: return to_compact_t<1>(a, st);
        case 2: return to_compact_t<2>(a, st);
        case 3: return to_compact_t<3>(a, st);
        default: return to_compact_t<4>(a, st);
    }
}

// The plane shape table of a compact-record abstraction (grids of 2+ dims,
// dims 0 and 1 not periodic); left NULL otherwise.  Best effort: the solver
// works without it.
template <int D>
static int build_shapes_t(bf_abstraction* a, cudaStream_t st) {
    const GridDesc& g = a->g;
    const long long P = g.C / g.stride[2];
    unsigned long long* shape = nullptr;
    unsigned long long* d_bad = nullptr;
    unsigned long long h_bad = 0;
    const long long n = P * g.U;
    unsigned long long *first = nullptr, *second = nullptr, *third = nullptr;
    unsigned *hit1 = nullptr, *hit2 = nullptr, *nbk = nullptr, *idx = nullptr;
    unsigned char* skip = nullptr;
    BF_CUDA(cudaMalloc((void**)&shape, sizeof(unsigned long long) * n));
    cudaError_t e = cudaMalloc((void**)&d_bad, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void**)&first, sizeof(unsigned long long) * 3 * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&hit1, sizeof(unsigned) * 4 * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&skip, n);
    if (e == cudaSuccess) {
        second = first + n;
        third = first + 2 * n;
        hit2 = hit1 + n;
        nbk = hit1 + 2 * n;
        idx = hit1 + 3 * n;
        e = cudaMemsetAsync(hit1, 0, sizeof(unsigned) * 3 * n, st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
        const int nb = grid_blocks(g.C * g.U, 256);
        const int ne = grid_blocks(n, 256);
        auto pick = [&](unsigned long long* out, const unsigned long long* ex1, const unsigned long long* ex2,
                        const unsigned char* sk) {
            if (e == cudaSuccess) e = cudaMemsetAsync(idx, 0xFF, sizeof(unsigned) * n, st);
            k_shape_first<D><<<nb, 256, 0, st>>>(g, a->d_boxes, idx, ex1, ex2, sk);
            k_shape_take<D><<<ne, 256, 0, st>>>(g, a->d_boxes, idx, n, out);
        };
        pick(first, nullptr, nullptr, nullptr);
        k_shape_count<D><<<nb, 256, 0, st>>>(g, a->d_boxes, first, hit1, nbk);
        if (e == cudaSuccess) e = cudaMemcpyAsync(shape, first, sizeof(unsigned long long) * n, cudaMemcpyDeviceToDevice, st);
        // second round where the first pick is shared by less than half of the pairs
        k_shape_retry<<<ne, 256, 0, st>>>(n, hit1, nbk, skip);
        pick(second, first, nullptr, skip);
        k_shape_count<D><<<nb, 256, 0, st>>>(g, a->d_boxes, second, hit2, nullptr);
        k_shape_choose<<<ne, 256, 0, st>>>(n, shape, second, hit1, hit2);
        // third round where neither is
        if (e == cudaSuccess) e = cudaMemsetAsync(hit2, 0, sizeof(unsigned) * n, st);
        k_shape_retry<<<ne, 256, 0, st>>>(n, hit1, nbk, skip);
        pick(third, first, second, skip);
        k_shape_count<D><<<nb, 256, 0, st>>>(g, a->d_boxes, third, hit2, nullptr);
        k_shape_choose<<<ne, 256, 0, st>>>(n, shape, third, hit1, hit2);
        k_shape_check<D><<<nb, 256, 0, st>>>(g, a->d_boxes, shape, d_bad);
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, d_bad, sizeof h_bad, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_bad);
    cudaFree(first);
    cudaFree(hit1);
    cudaFree(skip);
    if (e != cudaSuccess) { cudaFree(shape); return bfh::cuda_fail(e, "plane shape table"); }
    a->d_shape = shape;
    a->nplanes = P;
    a->shape_mismatch = (long long)h_bad;
    a->bytes += sizeof(unsigned long long) * P * g.U;
    // the lookup lists of every entry, for gathers without and with the 3 x 3
    // windows, and with the plane-pair table along dims 2 and 3
    for (int k = 0; k < 4; ++k) {
        if (k >= 2 && k >= D) break;
        BF_CUDA(cudaMalloc((void**)&a->d_poffs[k], sizeof(int) * kPlaneEnt * n));
        k_plane_lists<D><<<grid_blocks(n, 128), 128, 0, st>>>(g, shape, P, k >= 1 ? 1 : 0, k >= 2 ? k : 0,
                                                              a->d_poffs[k]);
        BF_CUDA(cudaGetLastError());
        a->bytes += sizeof(int) * kPlaneEnt * n;
    }
    if (g.U <= 32) {
        BF_CUDA(cudaMalloc((void**)&a->d_fmask, sizeof(unsigned long long) * g.C));
        k_cell_masks<D><<<grid_blocks(g.C, 256), 256, 0, st>>>(g, a->d_boxes, shape, a->d_fmask);
        BF_CUDA(cudaGetLastError());
        a->bytes += sizeof(unsigned long long) * g.C;
    }
    return BF_OK;
}

// Predecessor templates from the shape table (host; planes x inputs entries).
// Every non-blocked pair (x, u) of source plane q has the box x + (rel, w) of
// the entry S[q][u] (no mismatch), so y in box(x, u) means, per dim d, x_d =
// y_d - rel_d - j_d with 0 <= j_d < w_d (dims >= 2 wrap on periodic dims):
// target plane p of y gets, for source plane q, the rows d1 = -(rel1 + j1)
// with dim-0 offsets -(rel0 + w0 - 1) .. -rel0.  Offsets of one (p, q, d1)
// from different inputs merge into their bounding range (a superset).  The
// result holds pred(y) of Eq. (pred) for every y of p; with the blocked pairs
// it may hold a few more cells, which the algorithm tolerates.  The per-input
// templates (U <= 32) keep each input's rows apart: the pairs (x, u) with y in
// box(x, u) exactly, for the per-input frontier.
static int build_templates(bf_abstraction* a, cudaStream_t st) {
    const GridDesc& g = a->g;
    const long long P = a->nplanes, U = g.U;
    std::vector<unsigned long long> S((size_t)(P * U));
    BF_CUDA(cudaMemcpyAsync(S.data(), a->d_shape, sizeof(unsigned long long) * P * U, cudaMemcpyDeviceToHost, st));
    BF_CUDA(cudaStreamSynchronize(st));
    const int n2 = g.D >= 3 ? g.n[2] : 1, n3 = g.D >= 4 ? g.n[3] : 1;
    // merged: (q, d1) -> dim-0 range; per input: (u, q, d1) -> dim-0 range
    std::vector<std::map<std::pair<int, int>, std::pair<int, int>>> tm((size_t)P);
    std::vector<std::map<std::tuple<int, int, int>, std::pair<int, int>>> tu((size_t)P);
    for (long long q = 0; q < P; ++q) {
        const int k2 = (int)(q % n2), k3 = (int)(q / n2);
        for (long long u = 0; u < U; ++u) {
            const unsigned long long r = S[(size_t)(q * U + u)];
            int w[4] = {1, 1, 1, 1}, rel[4] = {0, 0, 0, 0};
            for (int d = 0; d < g.D; ++d) {
                w[d] = (int)((r >> (16 * d + 8)) & 0x7F);
                rel[d] = (int)(signed char)((r >> (16 * d)) & 0xFF);
            }
            if (w[0] == 0) continue;                           // no pair of the plane
            for (int j3 = 0; j3 < w[3]; ++j3) {
                int t3 = k3 + rel[3] + j3;
                if (g.D >= 4 && g.periodic[3]) t3 = ((t3 % n3) + n3) % n3;
                if (t3 < 0 || t3 >= n3) continue;
                for (int j2 = 0; j2 < w[2]; ++j2) {
                    int t2 = k2 + rel[2] + j2;
                    if (g.D >= 3 && g.periodic[2]) t2 = ((t2 % n2) + n2) % n2;
                    if (t2 < 0 || t2 >= n2) continue;
                    const size_t tp = (size_t)(t2 + (long long)n2 * t3);
                    auto& m = tm[tp];
                    auto& mu_ = tu[tp];
                    for (int j1 = 0; j1 < w[1]; ++j1) {
                        const int d1 = -(rel[1] + j1), lo = -(rel[0] + w[0] - 1), hi = -rel[0];
                        auto it = m.find({(int)q, d1});
                        if (it == m.end()) m[{(int)q, d1}] = {lo, hi};
                        else it->second = {std::min(it->second.first, lo), std::max(it->second.second, hi)};
                        const auto key = std::make_tuple((int)u, (int)q, d1);
                        auto iu = mu_.find(key);
                        if (iu == mu_.end()) mu_[key] = {lo, hi};
                        else iu->second = {std::min(iu->second.first, lo), std::max(iu->second.second, hi)};
                    }
                }
            }
        }
    }
    // per plane: the entries without the flag, then those with it;
    // ptr[2p] = first, ptr[2p + 1] = first flagged, ptr[2p + 2] = end
    std::vector<int> ptr(2 * (size_t)P + 1, 0), uptr(2 * (size_t)P + 1, 0);
    std::vector<int4> ent, uent;
    std::vector<int4> flagged;
    for (long long p = 0; p < P; ++p) {
        const auto& m = tm[(size_t)p];
        flagged.clear();
        for (auto it = m.begin(); it != m.end(); ++it) {
            const int q = it->first.first, d1 = it->first.second;
            const int lo = it->second.first, hi = it->second.second;
            auto nx = m.find({q, d1 + 1});
            const int cov = (nx != m.end() && nx->second.first <= lo && nx->second.second >= hi) ? 1 : 0;
            (cov ? flagged : ent).push_back(make_int4(q, d1, (lo & 0xFFFF) | (hi << 16), cov));
        }
        ptr[2 * (size_t)p + 1] = (int)ent.size();
        ent.insert(ent.end(), flagged.begin(), flagged.end());
        ptr[2 * (size_t)p + 2] = (int)ent.size();
        const auto& mu_ = tu[(size_t)p];
        flagged.clear();
        for (auto it = mu_.begin(); it != mu_.end(); ++it) {
            const int u = std::get<0>(it->first), q = std::get<1>(it->first), d1 = std::get<2>(it->first);
            const int lo = it->second.first, hi = it->second.second;
            auto nx = mu_.find(std::make_tuple(u, q, d1 + 1));
            const int cov = (nx != mu_.end() && nx->second.first <= lo && nx->second.second >= hi) ? 1 : 0;
            (cov ? flagged : uent).push_back(make_int4(q, d1, (lo & 0xFFFF) | (hi << 16), cov | (u << 8)));
        }
        uptr[2 * (size_t)p + 1] = (int)uent.size();
        uent.insert(uent.end(), flagged.begin(), flagged.end());
        uptr[2 * (size_t)p + 2] = (int)uent.size();
    }
    int *dptr = nullptr, *duptr = nullptr;
    int4 *dent = nullptr, *duent = nullptr;
    cudaError_t e = cudaMalloc((void**)&dptr, sizeof(int) * ptr.size());
    if (e == cudaSuccess) e = cudaMalloc((void**)&dent, sizeof(int4) * std::max<size_t>(1, ent.size()));
    if (e == cudaSuccess) e = cudaMemcpyAsync(dptr, ptr.data(), sizeof(int) * ptr.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !ent.empty())
        e = cudaMemcpyAsync(dent, ent.data(), sizeof(int4) * ent.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && g.U <= 32) {
        e = cudaMalloc((void**)&duptr, sizeof(int) * uptr.size());
        if (e == cudaSuccess) e = cudaMalloc((void**)&duent, sizeof(int4) * std::max<size_t>(1, uent.size()));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(duptr, uptr.data(), sizeof(int) * uptr.size(), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && !uent.empty())
            e = cudaMemcpyAsync(duent, uent.data(), sizeof(int4) * uent.size(), cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(dptr); cudaFree(dent); cudaFree(duptr); cudaFree(duent);
        return bfh::cuda_fail(e, "predecessor templates");
    }
    a->d_tptr = dptr;
    a->d_tent = dent;
    a->tmpl_rows = P ? (double)ent.size() / (double)P : 0.0;
    a->bytes += sizeof(int) * ptr.size() + sizeof(int4) * ent.size();
    if (duptr) {
        a->d_uptr = duptr;
        a->d_uent = duent;
        a->utmpl_rows = P ? (double)uent.size() / (double)P : 0.0;
        a->bytes += sizeof(int) * uptr.size() + sizeof(int4) * uent.size();
    }
    return BF_OK;
}

static int build_shapes(bf_abstraction* a, cudaStream_t st) {
    if (a->box_fmt != kBoxCompact || a->g.D < 2 || a->g.periodic[0] || a->g.periodic[1]) return BF_OK;
    int rc;
    switch (a->g.D) {
        case 2: rc = build_shapes_t<2>(a, st); break;
        case 3: rc = build_shapes_t<3>(a, st); break;
        default: rc = build_shapes_t<4>(a, st); break;
    }
    if (rc == BF_OK && a->d_shape && a->shape_mismatch == 0) rc = build_templates(a, st);
    return rc;
}

static bf_abstraction* new_abs() {
    bf_abstraction* a = new bf_abstraction;
    memset(a, 0, sizeof *a);
    a->bsched = -1;
    cudaGetDevice(&a->device);
    return a;
}

extern "C" void abs_free(bf_abstraction* a) {
    if (!a) return;
    if (a->ws) bf_solve_ws_free(a->ws);
    cudaFree(a->d_boxes);
    cudaFree(a->d_pred);
    cudaFree(a->d_inputs);
    cudaFree(a->d_rk);
    cudaFree(a->d_shape);
    for (int k = 0; k < 4; ++k) cudaFree(a->d_poffs[k]);
    cudaFree(a->d_fmask);
    cudaFree(a->d_tptr);
    cudaFree(a->d_tent);
    cudaFree(a->d_uptr);
    cudaFree(a->d_uent);
    delete a;
}

extern "C" int abs_build(const bf_dynamics* dyn, const bf_grid* grid, const bf_inputs* inputs,
                         double tau, int32_t mode, void* stream, bf_abstraction** out) {
    if (!out) { bfh::set_error("abs_build: out is NULL"); return BF_ERR_INVALID; }
    *out = nullptr;
    GridDesc g;
    int rc = check_grid(grid, g);
    if (rc) return rc;
    if (!dyn || !inputs || !inputs->u || inputs->ninputs < 1 || inputs->ninputs > 254 || inputs->udim < 1) {
        bfh::set_error("abs_build: need dyn and 1..254 inputs with udim >= 1");
        return BF_ERR_INVALID;
    }
    const int need_d = dyn->kind == BF_DYN_LINEAR2D ? 2 : dyn->kind == BF_DYN_UNICYCLE3D ? 3
                     : dyn->kind == BF_DYN_FIRE4D ? 4 : -1;
    if (need_d < 0 || need_d != g.D) {
        bfh::set_error("abs_build: dynamics kind %d needs a %d-D grid", dyn->kind, need_d);
        return BF_ERR_INVALID;
    }
    if (dyn->kind != BF_DYN_LINEAR2D && (dyn->rk4_substeps < 1 || inputs->udim < 2)) {
        bfh::set_error("abs_build: need rk4_substeps >= 1 and 2 input components");
        return BF_ERR_INVALID;
    }
    if (!(tau > 0.0) || (mode != BF_MODE_STORED && mode != BF_MODE_RECOMPUTE)) {
        bfh::set_error("abs_build: need tau > 0 and a valid mode");
        return BF_ERR_INVALID;
    }
    for (int d = 0; d < g.D; ++d)
        if (!(grid->hi[d] > grid->lo[d])) {
            bfh::set_error("abs_build: grid extent of dim %d is empty", d);
            return BF_ERR_INVALID;
        }
    cudaStream_t st = (cudaStream_t)stream;
    bf_abstraction* a = new_abs();
    a->g = g;
    a->g.U = inputs->ninputs;
    for (int d = 0; d < g.D; ++d) { a->glo[d] = grid->lo[d]; a->ghi[d] = grid->hi[d]; }
    a->mode = mode;
    a->dyn = *dyn;
    a->tau = tau;
    a->udim = inputs->udim;
    size_t in_bytes = sizeof(double) * inputs->ninputs * inputs->udim;
    cudaError_t e = cudaMalloc(&a->d_inputs, in_bytes);
    if (e == cudaSuccess) e = cudaMemcpyAsync(a->d_inputs, inputs->u, in_bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMalloc((void**)&a->d_pred, sizeof(short) * 2 * g.D * g.C);
    if (e == cudaSuccess && mode == BF_MODE_STORED) e = cudaMalloc(&a->d_boxes, box_bytes(a->g));
    if (e != cudaSuccess) { abs_free(a); return bfh::cuda_fail(e, "abs_build allocation"); }
    a->bytes = in_bytes + sizeof(short) * 2 * g.D * g.C + (mode == BF_MODE_STORED ? box_bytes(a->g) : 0);
    DynDesc dd = make_dyndesc(a);
    if (mode == BF_MODE_STORED) {
        const int nb = grid_blocks(a->g.C * a->g.U, 128);
        switch (g.D) {
            case 2: k_build_boxes<2><<<nb, 128, 0, st>>>(dd, a->g, a->d_inputs, a->d_boxes); break;
            case 3: k_build_boxes<3><<<nb, 128, 0, st>>>(dd, a->g, a->d_inputs, a->d_boxes); break;
            default: k_build_boxes<4><<<nb, 128, 0, st>>>(dd, a->g, a->d_inputs, a->d_boxes); break;
        }
    }
    a->box_fmt = mode == BF_MODE_STORED ? kBoxWide : kBoxRecompute;
    a->nstored = mode == BF_MODE_STORED ? a->g.U : 0;
    rc = build_pred(a, st);
    if (rc == BF_OK) {
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = bfh::cuda_fail(e, "abs_build kernels");
    }
    if (rc == BF_OK && mode == BF_MODE_STORED) rc = to_compact(a, st);
    if (rc == BF_OK && mode == BF_MODE_STORED) rc = build_shapes(a, st);
    if (rc == BF_OK && mode == BF_MODE_RECOMPUTE && g.D >= 3 && dyn->rk4_substeps <= kRkMaxSub) {
        // the RK4 work shared by cells with equal coordinates on dims >= 2
        const long long nkeys = g.C / g.stride[2];
        const size_t bytes = sizeof(double) * kRkEntry * nkeys * a->g.U;
        e = cudaMalloc((void**)&a->d_rk, bytes);
        if (e == cudaSuccess) {
            const int nb = grid_blocks(nkeys * a->g.U, 64);
            if (g.D == 3) k_rk_table<3><<<nb, 64, 0, st>>>(dd, a->g, a->d_inputs, nkeys, a->d_rk);
            else k_rk_table<4><<<nb, 64, 0, st>>>(dd, a->g, a->d_inputs, nkeys, a->d_rk);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = bfh::cuda_fail(e, "recompute RK4 table");
        else a->bytes += bytes;
    }
    if (rc) { abs_free(a); return rc; }
    *out = a;
    return BF_OK;
}

// Memory-regulated build (Sec. IV-B): the recompute-mode abstraction plus the
// compact records of the first K inputs, K the most whose records fit in
// box_budget bytes.  K = U gives stored mode, K = 0 (or boxes that do not fit
// the compact records) recompute mode.
template <int D>
static int add_stored_inputs(bf_abstraction* a, int K, cudaStream_t st) {
    const size_t rec = D <= 2 ? 4 : 8;
    const size_t bytes = rec * (size_t)a->g.C * K;
    GridDesc gk = a->g;
    gk.U = K;
    void* comp = nullptr;
    int* d_fail = nullptr;
    int h_fail = 0;
    BF_CUDA(cudaMalloc(&comp, bytes));
    cudaError_t e = cudaMalloc((void**)&d_fail, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(d_fail, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        DynDesc dd = make_dyndesc(a);
        k_build_compact<D><<<grid_blocks(gk.C * K, 128), 128, 0, st>>>(dd, gk, a->d_inputs, comp, d_fail);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_fail, d_fail, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_fail);
    if (e != cudaSuccess) { cudaFree(comp); return bfh::cuda_fail(e, "hybrid box records"); }
    if (h_fail) { cudaFree(comp); return BF_OK; }      // stays in recompute mode
    a->d_boxes = comp;
    a->nstored = K;
    a->box_fmt = K == a->g.U ? kBoxCompact : kBoxHybrid;
    a->mode = K == a->g.U ? BF_MODE_STORED : BF_MODE_HYBRID;
    a->bytes += bytes;
    return BF_OK;
}

extern "C" int abs_build_hybrid(const bf_dynamics* dyn, const bf_grid* grid, const bf_inputs* inputs,
                                double tau, int64_t box_budget, void* stream, bf_abstraction** out) {
    if (box_budget < 0) { bfh::set_error("abs_build_hybrid: negative budget"); return BF_ERR_INVALID; }
    int rc = abs_build(dyn, grid, inputs, tau, BF_MODE_RECOMPUTE, stream, out);
    if (rc) return rc;
    bf_abstraction* a = *out;
    const long long rec = a->g.D <= 2 ? 4 : 8;
    const long long K = std::min<long long>(a->g.U, box_budget / (rec * a->g.C));
    if (K <= 0) return BF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    switch (a->g.D) {
        case 2: rc = add_stored_inputs<2>(a, (int)K, st); break;
        case 3: rc = add_stored_inputs<3>(a, (int)K, st); break;
        default: rc = add_stored_inputs<4>(a, (int)K, st); break;
    }
    if (rc) { abs_free(a); *out = nullptr; }
    return rc;
}

extern "C" int abs_stored_inputs(const bf_abstraction* a, int32_t* nstored) {
    if (!a || !nstored) { bfh::set_error("abs_stored_inputs: NULL argument"); return BF_ERR_INVALID; }
    *nstored = a->nstored;
    return BF_OK;
}

extern "C" int abs_from_boxes(const bf_grid* grid, int32_t ninputs, const int16_t* boxes,
                              void* stream, bf_abstraction** out) {
    if (!out || !boxes) { bfh::set_error("abs_from_boxes: NULL argument"); return BF_ERR_INVALID; }
    *out = nullptr;
    GridDesc g;
    int rc = check_grid(grid, g);
    if (rc) return rc;
    if (ninputs < 1 || ninputs > 254) { bfh::set_error("abs_from_boxes: ninputs must be 1..254"); return BF_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    bf_abstraction* a = new_abs();
    a->g = g;
    a->g.U = ninputs;
    for (int d = 0; d < g.D; ++d) { a->glo[d] = grid->lo[d]; a->ghi[d] = grid->hi[d]; }
    a->mode = BF_MODE_STORED;
    const size_t ext_bytes = box_bytes(a->g);
    const short* src = reinterpret_cast<const short*>(boxes);
    short* staged = nullptr;
    unsigned long long* d_bad = nullptr;
    unsigned long long h_bad = 0;
    cudaError_t e = cudaMalloc(&a->d_boxes, box_bytes(a->g));
    if (e == cudaSuccess) e = cudaMalloc((void**)&a->d_pred, sizeof(short) * 2 * g.D * g.C);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_bad, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess && !bfh::is_device_ptr(boxes)) {
        e = cudaMalloc((void**)&staged, ext_bytes);
        if (e == cudaSuccess) e = cudaMemcpyAsync(staged, boxes, ext_bytes, cudaMemcpyHostToDevice, st);
        src = staged;
    }
    if (e != cudaSuccess) {
        cudaFree(staged); cudaFree(d_bad); abs_free(a);
        return bfh::cuda_fail(e, "abs_from_boxes allocation");
    }
    a->bytes = box_bytes(a->g) + sizeof(short) * 2 * g.D * g.C;
    const int nb = grid_blocks(a->g.C * a->g.U, 256);
    switch (g.D) {
        case 1: k_import_boxes<1><<<nb, 256, 0, st>>>(a->g, src, a->d_boxes, d_bad); break;
        case 2: k_import_boxes<2><<<nb, 256, 0, st>>>(a->g, src, a->d_boxes, d_bad); break;
        case 3: k_import_boxes<3><<<nb, 256, 0, st>>>(a->g, src, a->d_boxes, d_bad); break;
        default: k_import_boxes<4><<<nb, 256, 0, st>>>(a->g, src, a->d_boxes, d_bad); break;
    }
    e = cudaMemcpyAsync(&h_bad, d_bad, sizeof h_bad, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(staged);
    cudaFree(d_bad);
    if (e != cudaSuccess) { abs_free(a); return bfh::cuda_fail(e, "abs_from_boxes import"); }
    if (h_bad) {
        abs_free(a);
        bfh::set_error("abs_from_boxes: %llu malformed boxes", h_bad);
        return BF_ERR_INVALID;
    }
    a->box_fmt = kBoxWide;
    a->nstored = a->g.U;
    rc = build_pred(a, st);
    if (rc == BF_OK) {
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = bfh::cuda_fail(e, "abs_from_boxes pred");
    }
    if (rc == BF_OK) rc = to_compact(a, st);
    if (rc == BF_OK) rc = build_shapes(a, st);
    if (rc) { abs_free(a); return rc; }
    *out = a;
    return BF_OK;
}

extern "C" int abs_export_boxes(const bf_abstraction* a, int16_t* out, void* stream) {
    if (!a || !out) { bfh::set_error("abs_export_boxes: NULL argument"); return BF_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = box_bytes(a->g);
    const bool dev = bfh::is_device_ptr(out);
    short* dst = reinterpret_cast<short*>(out);
    if (!dev) BF_CUDA(cudaMallocAsync((void**)&dst, bytes, st));
    DynDesc dd = make_dyndesc(a);
    const int nb = grid_blocks(a->g.C * a->g.U, 128);
    switch (a->g.D) {
        case 1: k_export_boxes<1><<<nb, 128, 0, st>>>(a->g, dd, a->d_inputs, a->d_boxes, a->box_fmt, a->nstored, dst); break;
        case 2: k_export_boxes<2><<<nb, 128, 0, st>>>(a->g, dd, a->d_inputs, a->d_boxes, a->box_fmt, a->nstored, dst); break;
        case 3: k_export_boxes<3><<<nb, 128, 0, st>>>(a->g, dd, a->d_inputs, a->d_boxes, a->box_fmt, a->nstored, dst); break;
        default: k_export_boxes<4><<<nb, 128, 0, st>>>(a->g, dd, a->d_inputs, a->d_boxes, a->box_fmt, a->nstored, dst); break;
    }
    BF_CUDA(cudaGetLastError());
    if (!dev) {
        BF_CUDA(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, st));
        BF_CUDA(cudaFreeAsync(dst, st));
    }
    BF_CUDA(cudaStreamSynchronize(st));
    return BF_OK;
}

extern "C" int abs_export_pred(const bf_abstraction* a, int16_t* out, void* stream) {
    if (!a || !out) { bfh::set_error("abs_export_pred: NULL argument"); return BF_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    BF_CUDA(cudaMemcpyAsync(out, a->d_pred, sizeof(short) * 2 * a->g.D * a->g.C, cudaMemcpyDefault, st));
    BF_CUDA(cudaStreamSynchronize(st));
    return BF_OK;
}

extern "C" int abs_shape_info(const bf_abstraction* a, int64_t* nplanes, int64_t* mismatch) {
    if (!a) { bfh::set_error("abs_shape_info: NULL abstraction"); return BF_ERR_INVALID; }
    if (nplanes) *nplanes = a->d_shape ? a->nplanes : 0;
    if (mismatch) *mismatch = a->d_shape ? a->shape_mismatch : 0;
    return BF_OK;
}

extern "C" int abs_info(const bf_abstraction* a, int64_t* ncells, int32_t* ninputs, int32_t* ndim,
                        int32_t* mode, int64_t* device_bytes, int32_t* box_record_bytes) {
    if (!a) { bfh::set_error("abs_info: NULL abstraction"); return BF_ERR_INVALID; }
    if (ncells) *ncells = a->g.C;
    if (ninputs) *ninputs = a->g.U;
    if (ndim) *ndim = a->g.D;
    if (mode) *mode = a->mode;
    if (device_bytes) *device_bytes = (int64_t)a->bytes;
    if (box_record_bytes)
        *box_record_bytes = (a->box_fmt == kBoxCompact || a->box_fmt == kBoxHybrid) ? (a->g.D <= 2 ? 4 : 8)
                          : a->box_fmt == kBoxWide ? 4 * a->g.D : 0;
    return BF_OK;
}
