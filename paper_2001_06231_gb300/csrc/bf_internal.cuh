// bf_internal.cuh -- device-side building blocks shared by the library's
// translation units (not part of the C ABI).
//
// Value keys.  The relaxation of Algorithm 1 needs max over a box, min over
// inputs and "d < W(x)" on FP64 values.  GB300 has little FP64 throughput, so
// V is kept in HBM as order-preserving int64 keys: for the IEEE-754 bit
// pattern b of a double, key = b ^ ((b >> 63) & 0x7fff...f).  Non-negative
// doubles keep their bits; negative ones get their magnitude bits flipped, so
// signed int64 order equals the order of the doubles (with -0 below +0; the
// library maps -0 inputs to +0, after which no -0 can arise, so key order and
// IEEE order agree on every value that occurs).  The map is its own inverse.
// One FP64 add per relaxation remains: d = G(x,u) + max V.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "bfgpu.h"

namespace bfk {

constexpr int16_t kBlocked = -32768;

// storage formats of an abstraction's boxes
constexpr int kBoxWide = 0;      // int16 absolute records [U][C] (4*D bytes)
constexpr int kBoxCompact = 1;   // int8 relative records [U][C] (4 bytes for D <= 2, else 8)
constexpr int kBoxRecompute = 2; // not stored: regenerated from the dynamics
constexpr int kBoxHybrid = 3;    // compact records for inputs u < nstored, recompute for the rest
constexpr long long kKeyInf = 0x7FF0000000000000LL;   // key(+inf) == bits(+inf)
constexpr long long kKeyMin = (long long)0x8000000000000000ULL;
constexpr unsigned char kHandover = 0xFF;

__host__ __device__ __forceinline__ long long key_from_bits(long long b) {
    return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}

__device__ __forceinline__ long long key_of(double v) {
    return key_from_bits(__double_as_longlong(v));
}

__device__ __forceinline__ double val_of(long long k) {
    return __longlong_as_double(key_from_bits(k));
}

// Grid geometry passed to kernels by value.
struct GridDesc {
    int D;
    int n[4];
    int periodic[4];
    long long stride[4];   // stride[d] = n[0]*...*n[d-1]
    long long C;
    int U;
    // x / n[d] for 0 <= x < 2^31 without a divide instruction (division by an
    // invariant integer, Granlund & Montgomery 1994): with l = ceil(log2 n),
    // m = floor(2^32 (2^l - n) / n) + 1, x / n = (umulhi(m, x) + x) >> l.
    unsigned dmul[4];
    int dshr[4];
};

// Host: the division constants of every dim (n[d] in 1..2^31-1).
inline void grid_divisors(GridDesc& g) {
    for (int d = 0; d < 4; ++d) {
        const unsigned long long n = (unsigned long long)(g.n[d] > 0 ? g.n[d] : 1);
        int l = 0;
        while ((1ull << l) < n) ++l;
        g.dmul[d] = (unsigned)(((1ull << 32) * ((1ull << l) - n)) / n + 1);
        g.dshr[d] = l;
    }
}

#ifdef __CUDACC__
__device__ __forceinline__ unsigned grid_div(const GridDesc& g, int d, unsigned x) {
    return (__umulhi(g.dmul[d], x) + x) >> g.dshr[d];
}

// Quotients t / d of box extents (1 <= d <= 255, 0 <= t < 2^23) by one
// multiply-high: with m = ceil(2^31 / d), m d = 2^31 + e and 0 <= e < d, so
// umulhi(2t, m) = floor(t m / 2^31) = floor(t / d + t e / (d 2^31)); writing
// t = q d + r (r <= d - 1), t e < 2^23 * 254 < 2^31 keeps r + t e / 2^31 below
// d and the floor at q.
struct RecipTable { unsigned m[256]; };
constexpr RecipTable make_recip_table() {
    RecipTable r{};
    for (unsigned d = 1; d < 256; ++d) r.m[d] = (unsigned)((0x80000000ull + d - 1) / d);
    return r;
}
static __constant__ RecipTable kRecip = make_recip_table();
constexpr unsigned kSmallDivMax = 1u << 23;
__device__ __forceinline__ unsigned small_div(unsigned t, unsigned m) { return __umulhi(t << 1, m); }
#endif

// Box of one (cell, input) pair in registers.
template <int D>
struct Box {
    int lo[D];
    int hi[D];
};

// Boxes live in HBM as [U][C] records of D int16 lo followed by D int16 hi
// (4*D bytes).  Lanes of a warp read consecutive cells of one input, so each
// warp load is one contiguous run of 32*4*D bytes; D = 4 is one 128-bit load
// per lane.  Boxes stream through once per pass: evict-first loads.
template <int D>
__device__ __forceinline__ Box<D> load_box(const void* __restrict__ boxes, long long idx) {
    Box<D> b;
    if constexpr (D == 4) {
        uint4 v = __ldcs(reinterpret_cast<const uint4*>(boxes) + idx);
        b.lo[0] = (short)(v.x & 0xFFFF); b.lo[1] = (short)(v.x >> 16);
        b.lo[2] = (short)(v.y & 0xFFFF); b.lo[3] = (short)(v.y >> 16);
        b.hi[0] = (short)(v.z & 0xFFFF); b.hi[1] = (short)(v.z >> 16);
        b.hi[2] = (short)(v.w & 0xFFFF); b.hi[3] = (short)(v.w >> 16);
    } else if constexpr (D == 3) {
        const unsigned* p = reinterpret_cast<const unsigned*>(boxes) + idx * 3;
        unsigned a = __ldcs(p), c = __ldcs(p + 1), e = __ldcs(p + 2);
        b.lo[0] = (short)(a & 0xFFFF); b.lo[1] = (short)(a >> 16);
        b.lo[2] = (short)(c & 0xFFFF); b.hi[0] = (short)(c >> 16);
        b.hi[1] = (short)(e & 0xFFFF); b.hi[2] = (short)(e >> 16);
    } else if constexpr (D == 2) {
        uint2 v = __ldcs(reinterpret_cast<const uint2*>(boxes) + idx);
        b.lo[0] = (short)(v.x & 0xFFFF); b.lo[1] = (short)(v.x >> 16);
        b.hi[0] = (short)(v.y & 0xFFFF); b.hi[1] = (short)(v.y >> 16);
    } else {
        unsigned v = __ldcs(reinterpret_cast<const unsigned*>(boxes) + idx);
        b.lo[0] = (short)(v & 0xFFFF);
        b.hi[0] = (short)(v >> 16);
    }
    return b;
}

template <int D>
__device__ __forceinline__ void store_box(void* boxes, long long idx, const Box<D>& b) {
    short* p = reinterpret_cast<short*>(boxes) + idx * (2 * D);
#pragma unroll
    for (int d = 0; d < D; ++d) { p[d] = (short)b.lo[d]; p[D + d] = (short)b.hi[d]; }
}

__device__ __forceinline__ int wrap_idx(int v, int n, int periodic) {
    return (periodic && v >= n) ? v - n : v;
}

// max over the box of V (as keys).  Rows along dim 0 are contiguous in
// memory; the other dims are walked with explicit loops.
template <int D>
__device__ __forceinline__ long long box_max(const long long* __restrict__ V, const GridDesc& g,
                                             const Box<D>& b) {
    long long m = kKeyMin;
    const int n0 = g.n[0], p0 = g.periodic[0];
    if constexpr (D == 1) {
        for (int i0 = b.lo[0]; i0 <= b.hi[0]; ++i0) m = max(m, __ldg(V + wrap_idx(i0, n0, p0)));
    } else if constexpr (D == 2) {
        for (int i1 = b.lo[1]; i1 <= b.hi[1]; ++i1) {
            const long long* row = V + (long long)wrap_idx(i1, g.n[1], g.periodic[1]) * g.stride[1];
            for (int i0 = b.lo[0]; i0 <= b.hi[0]; ++i0) m = max(m, __ldg(row + wrap_idx(i0, n0, p0)));
        }
    } else if constexpr (D == 3) {
        for (int i2 = b.lo[2]; i2 <= b.hi[2]; ++i2) {
            const long long* pl = V + (long long)wrap_idx(i2, g.n[2], g.periodic[2]) * g.stride[2];
            for (int i1 = b.lo[1]; i1 <= b.hi[1]; ++i1) {
                const long long* row = pl + (long long)wrap_idx(i1, g.n[1], g.periodic[1]) * g.stride[1];
                for (int i0 = b.lo[0]; i0 <= b.hi[0]; ++i0) m = max(m, __ldg(row + wrap_idx(i0, n0, p0)));
            }
        }
    } else {
        for (int i3 = b.lo[3]; i3 <= b.hi[3]; ++i3) {
            const long long* vol = V + (long long)wrap_idx(i3, g.n[3], g.periodic[3]) * g.stride[3];
            for (int i2 = b.lo[2]; i2 <= b.hi[2]; ++i2) {
                const long long* pl = vol + (long long)wrap_idx(i2, g.n[2], g.periodic[2]) * g.stride[2];
                for (int i1 = b.lo[1]; i1 <= b.hi[1]; ++i1) {
                    const long long* row = pl + (long long)wrap_idx(i1, g.n[1], g.periodic[1]) * g.stride[1];
                    for (int i0 = b.lo[0]; i0 <= b.hi[0]; ++i0) m = max(m, __ldg(row + wrap_idx(i0, n0, p0)));
                }
            }
        }
    }
    return m;
}

// Coordinates of cell c (grids hold fewer than 2^31 cells).
__device__ __forceinline__ void cell_coords(const GridDesc& g, long long c, int* k) {
    unsigned r = (unsigned)c;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        if (d < g.D) {
            const unsigned q = grid_div(g, d, r);
            k[d] = (int)(r - q * (unsigned)g.n[d]);
            r = q;
        }
    }
}

// Warp-aggregated append: every lane with `pred` set gets a distinct slot.
__device__ __forceinline__ int warp_append(unsigned pred, int* counter) {
    const unsigned lane = threadIdx.x & 31;
    unsigned mask = __ballot_sync(0xFFFFFFFFu, pred);
    int base = 0;
    if (mask) {
        const int leader = __ffs(mask) - 1;
        if ((int)lane == leader) base = atomicAdd(counter, __popc(mask));
        base = __shfl_sync(0xFFFFFFFFu, base, leader);
    }
    return base + __popc(mask & ((1u << lane) - 1u));
}

}  // namespace bfk

// ---------------------------------------------------------------------------
// host-side objects shared between translation units
// ---------------------------------------------------------------------------
struct bf_solve_ws;   // per-solve device workspace (solve.cu)

struct bf_abstraction {
    bfk::GridDesc g;
    double glo[4], ghi[4];
    int mode;
    int device;
    // dynamics (kept for RECOMPUTE mode and export)
    bf_dynamics dyn;
    double tau;
    int udim;
    double* d_inputs;         // [U][udim]
    double* d_rk;             // recompute / hybrid: shared RK4 parts [keys][U][entry] or NULL
    // stored mode: boxes [U][C], wide (4*D bytes) or compact records
    void* d_boxes;
    int box_fmt;              // bfk::kBoxWide / kBoxCompact / kBoxRecompute / kBoxHybrid
    int nstored;              // inputs with stored records (U, 0, or in between: hybrid)
    // plane shape table (compact records, grids of 2+ dims with dims 0 and 1
    // not periodic): per plane p (the cells with equal coordinates on dims
    // >= 2) and input u, the relative record shared by the plane's
    // non-blocked pairs (0: the plane has none) [nplanes][U], or NULL
    unsigned long long* d_shape;
    long long nplanes;
    long long shape_mismatch; // non-blocked records that differ from their plane's entry
    int* d_poffs[4];          // lookup lists of every (plane, input) [nplanes][U][kPlaneEnt]
                              // (solve_core.cuh), or NULL: [0] without the 3 x 3 window table,
                              // [1] with it, [2] / [3] with it and the plane-pair table along
                              // dim 2 / dim 3 (grids of 3+ / 4 dims)
    // per cell the inputs whose record is the plane's entry (bits 0..31) and
    // those with another record (bits 32..63); NULL where U > 32
    unsigned long long* d_fmask;   // [C]
    // predecessor templates (shape table with no mismatch): per target plane p
    // the rows (source plane q, dim-1 offset d1, dim-0 offsets lo..hi) whose
    // cells x = (y0 + lo .. y0 + hi, y1 + d1, q) hold pred(y) for every cell
    // y = (y0, y1, p); entries int4 {q, d1, lo & 0xFFFF | hi << 16, flags},
    // flags bit 0: row (q, d1 + 1) of the template spans lo..hi too
    int* d_tptr;              // [2 nplanes + 1]: plane p's entries at [d_tptr[2p], d_tptr[2p + 2]),
                              // those without the flag first, up to d_tptr[2p + 1]
    int4* d_tent;             // [d_tptr[2 nplanes]]
    double tmpl_rows;         // mean template entries per plane
    // per-input templates (U <= 32): the same rows kept apart by input, entries
    // int4 {q, d1, lo & 0xFFFF | hi << 16, flags | u << 8} (flags bit 0: row
    // (q, d1 + 1) of input u spans lo..hi too); NULL otherwise
    int* d_uptr;              // [2 nplanes + 1], as d_tptr
    int4* d_uent;             // [d_uptr[2 nplanes]]
    double utmpl_rows;        // mean per-input template entries per plane
    // predecessor index [C][2*D] int16 offsets (x = y + off), empty: lo0 > hi0
    short* d_pred;
    double pred_rows;         // mean dim-0 rows of a predecessor box (cells with one)
    size_t bytes;
    bf_solve_ws* ws;          // cached workspace of bf_solve
    int bsched;               // batched-engine schedule (kBs* bits; bf_tune_batch), -1: default
};

// batched-engine schedule bits (bf_abstraction::bsched)
constexpr int kBsWindow33 = 1;    // gathers read the 3 x 3 window table
constexpr int kBsPlane = 2;       // relax reads the plane lookup lists
constexpr int kBsTemplates = 4;   // marking reads the predecessor templates
constexpr int kBsPair = 8;        // plane relax takes two inputs per iteration
constexpr int kBsMark = 16;       // relax marks the next frontier (else a propagate launch)
constexpr int kBsMarkAuto = 32;   // ... when the group's predecessor boxes are small (kBsMark ignored)
constexpr int kBsQueue = 64;      // plane relax by cell masks, the pairs queued over the lanes
constexpr int kBsDefault = kBsWindow33 | kBsPlane | kBsTemplates | kBsPair | kBsMarkAuto;

namespace bfh {
// thread-local error message (bf_last_error)
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
bool is_device_ptr(const void* p);
}  // namespace bfh

#define BF_CUDA(call)                                              \
    do {                                                           \
        cudaError_t e__ = (call);                                  \
        if (e__ != cudaSuccess) return bfh::cuda_fail(e__, #call); \
    } while (0)

// parameters of the built-in dynamics (device code in dynamics.cuh)
namespace bfk {
struct DynDesc {
    int kind;
    int substeps;
    int udim;
    double tau;
    double p[8];
    double glo[4];
    double eta[4];
};
}  // namespace bfk
