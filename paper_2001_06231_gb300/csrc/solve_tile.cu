// solve_tile.cu -- the tile form of the relaxation (Alg. 1, relaxation and
// update lines) for passes whose frontier covers much of the grid.
//
// A block takes a tile: one plane q (the cells with equal coordinates on dims
// >= 2) and a band of kTileRows rows along dim 1, every column of dim 0.  For
// each input u the tile's boxes share the plane's relative record S[q][u]
// (plane shape table), so the window-table cells their gathers read form, per
// plane of the box on dims >= 2, one rectangle of the table: rows r0 + rel1
// .. r0 + kTileRows - 1 + rel1 + (rows of the box's lookups), columns x + rel0
// + (columns of the lookups).  Those rectangles ("slices") are copied into
// shared memory with TMA (cp.async.bulk.tensor.3d over the table viewed as a
// [planes][n1][n0] tensor of int64 keys, completion counted on an mbarrier),
// and every frontier cell of the tile takes its box maximum from shared
// memory.  A lane whose record is not the plane's entry (or an input whose
// slices do not fit the staging buffer) gathers from global memory instead.
// The cells not in F1 (read from the F1 bitmap that compaction keeps) are
// skipped; d, the strict-decrease test and the lowest-input rule are those of
// the list relax, so the results are the same bit for bit.
//
// Every wait on the mbarrier is bounded: after kTileSpin unsuccessful tries
// the block records a fault in the pass counters (the host reports it as an
// error), waits once more with the same bound for its copies in flight, and
// leaves.  Tensor maps cover only this device's own table arrays; no copy is
// multicast.
#include <cuda.h>
#include <cstring>

#include "solve_core.cuh"

using namespace bfk;

namespace {

constexpr int kTileRows = 8;          // rows of dim 1 per tile
constexpr int kTileSlices = 8;        // slices (box planes on dims >= 2) per input, at most
constexpr long long kTileSpin = 1 << 22;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// true once the phase of parity `ph` has completed; false after kTileSpin tries
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned ph) {
    for (long long i = 0; i < kTileSpin; ++i) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(ph)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int x, int y, int z,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(z),
          "r"(smem_u32(bar))
        : "memory");
}

}  // namespace

// Launch geometry of the tile relax (host-chosen per abstraction).
struct TileParams {
    int XT;          // threads across a row (multiple of 32, >= n0); kTileRows * XT / 256 rows per thread
    int BX;          // staged columns per slice row (even, <= 256)
    int RY;          // staged rows per slice
    int xbase;       // column of the first staged element (even; <= every input's dim-0 offset)
    int nbands;      // bands of kTileRows rows along dim 1
    int maxsl;       // slices the staging buffer holds (<= kTileSlices)
    long long ntiles;
};

// KR = rows per thread = kTileRows * XT / 256.
template <int D, bool MARK, int KR>
__global__ void __launch_bounds__(256) k_relax_tile(InstView v, TileParams tp, const __grid_constant__ CUtensorMap t0,
                                                    const __grid_constant__ CUtensorMap t1,
                                                    const __grid_constant__ CUtensorMap t2,
                                                    const __grid_constant__ CUtensorMap t3) {
    Counters* k = v.ctr;
    if (k->done || k->ncur < v.dense_min) return;
    // TMA writes shared memory at 128-byte aligned addresses: the buffer
    // starts at the first such address of the dynamic allocation (sized with
    // 128 bytes to spare) and every slice occupies a multiple of 16 keys
    extern __shared__ __align__(128) unsigned char tile_smem[];
    long long* buf = reinterpret_cast<long long*>(tile_smem + ((128u - (smem_u32(tile_smem) & 127u)) & 127u));
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int any;
    const GridDesc& g = v.g;
    const int n0 = g.n[0], n1 = g.n[1], U = g.U;
    const int tid = threadIdx.x;
    const int xt = tid % tp.XT, yt = tid / tp.XT;
    const int slots = 256 / tp.XT;                 // row slots; row kr of a thread = r0 + yt + kr * slots
    const int SL = ((tp.RY * tp.BX) + 15) & ~15;   // keys per slice (RY x BX staged, padded to 128 bytes)
    if (tid == 0) mbar_init(&bar, 1);
    __syncthreads();
    unsigned phase = 0;
    long long relaxed = 0;
    int dummy = 0;
    const long long rows_tot = (long long)n1;
    for (long long tile = blockIdx.x; tile < tp.ntiles; tile += gridDim.x) {
        const int q = (int)(tile / tp.nbands);
        const int r0 = (int)(tile - (long long)q * tp.nbands) * kTileRows;
        const int nrows = (int)min((long long)kTileRows, rows_tot - r0);
        const long long base = ((long long)q * n1 + r0) * n0;
        // any cell of F1 in the tile?
        if (tid == 0) any = 0;
        __syncthreads();
        {
            const long long w0 = base >> 5, w1 = (base + (long long)nrows * n0 - 1) >> 5;
            for (long long wd = w0 + tid; wd <= w1; wd += 256)
                if (v.f1bits[wd]) any = 1;
        }
        __syncthreads();
        if (!any) continue;
        // this thread's cells: column xt of rows r0 + yt + kr * slots
        long long c[KR];
        bool inF[KR];
        long long best[KR];
        int bu[KR];
#pragma unroll
        for (int kr = 0; kr < KR; ++kr) {
            const int y = yt + kr * slots;
            inF[kr] = false;
            c[kr] = base + (long long)y * n0 + xt;
            best[kr] = 0;
            bu[kr] = -1;
            if (xt < n0 && y < nrows) {
                inF[kr] = (v.f1bits[c[kr] >> 5] >> (c[kr] & 31)) & 1u;
                if (inF[kr]) {
                    best[kr] = v.Vkey[c[kr]];
                    ++relaxed;
                }
            }
        }
        int kq[4] = {0, 0, 0, 0};
        if (D >= 3) { kq[2] = q % g.n[2]; kq[3] = q / g.n[2]; }
        for (int u = 0; u < U; ++u) {
            const long long e = (long long)q * U + u;
            const unsigned long long S = __ldg(v.shape + e);
            if ((rec_byte(S, 1) & 0x7F) == 0) continue;      // every pair of the plane is blocked
            int w[4] = {1, 1, 1, 1}, rel[4] = {0, 0, 0, 0};
#pragma unroll
            for (int d = 0; d < D; ++d) {
                w[d] = rec_byte(S, 2 * d + 1) & 0x7F;
                rel[d] = rec_sbyte(S, 2 * d);
            }
            const bool use33 = v.M33 != nullptr && w[0] >= 3 && w[1] >= 3;
            const int tab = use33 ? 3 : (w[0] == 1 ? 0 : (w[0] == 2 ? 1 : 2));
            const int np = w[0] < 3 ? 1 : (w[0] + 2) / 3;
            const int nb = use33 ? (w[1] + 2) / 3 : w[1];
            const int rows_need = kTileRows + (use33 ? w[1] - 3 : w[1] - 1);
            const int amax = w[0] < 3 ? 0 : w[0] - 3;
            const int nsl = w[2] * w[3];
            const bool staged = nsl <= tp.maxsl && rows_need <= tp.RY && rel[0] >= tp.xbase &&
                                n0 - 1 + rel[0] + amax - tp.xbase < tp.BX;
            const long long* tabp = tab == 3 ? v.M33 : (tab == 2 ? v.M3 : (tab == 1 ? v.M2 : v.Vkey));
            if (staged) {
                if (tid == 0) {
                    const CUtensorMap* tm = tab == 3 ? &t3 : (tab == 2 ? &t2 : (tab == 1 ? &t1 : &t0));
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_expect(&bar, (unsigned)(nsl * tp.RY * tp.BX * 8));
                    int j = 0;
                    for (int j3 = 0; j3 < w[3]; ++j3)
                        for (int j2 = 0; j2 < w[2]; ++j2, ++j) {
                            int p2 = 0, p3 = 0;
                            if (D >= 3) {
                                p2 = kq[2] + rel[2] + j2;
                                if (g.periodic[2]) p2 = ((p2 % g.n[2]) + g.n[2]) % g.n[2];
                            }
                            if (D >= 4) {
                                p3 = kq[3] + rel[3] + j3;
                                if (g.periodic[3]) p3 = ((p3 % g.n[3]) + g.n[3]) % g.n[3];
                            }
                            const int pz = D >= 3 ? p2 + g.n[2] * p3 : 0;
                            tma_load_3d(buf + (long long)j * SL, tm, tp.xbase, r0 + rel[1], pz, &bar);
                        }
                }
                const bool ok = mbar_wait(&bar, phase);
                if (__syncthreads_or(!ok)) {                       // the whole block gives up together
                    if (tid == 0) atomicExch(&k->fault, 1);
                    (void)mbar_wait(&bar, phase);                  // the copies in flight, bounded
                    return;
                }
                phase ^= 1u;
            }
            const unsigned long long* rp = reinterpret_cast<const unsigned long long*>(v.boxes);
            const int* ent = v.poffs ? v.poffs + e * kPlaneEnt : nullptr;
#pragma unroll
            for (int kr = 0; kr < KR; ++kr) {
                if (!inF[kr]) continue;
                unsigned long long r;
                if constexpr (D <= 2) r = __ldcs(reinterpret_cast<const unsigned*>(v.boxes) + (long long)u * g.C + c[kr]);
                else r = __ldcs(rp + (long long)u * g.C + c[kr]);
                if ((rec_byte(r, 1) & 0x7F) == 0) continue;      // blocked
                long long m = kKeyMin;
                if (r == S && staged) {
                    const int y = yt + kr * slots;
                    const long long* s0 = buf + (long long)y * tp.BX + (xt + rel[0] - tp.xbase);
                    for (int j = 0; j < nsl; ++j)
                        for (int b = 0; b < nb; ++b) {
                            const long long* row = s0 + (long long)j * SL +
                                                   (long long)(use33 ? min(3 * b, w[1] - 3) : b) * tp.BX;
                            for (int a = 0; a < np; ++a) m = max(m, row[min(3 * a, amax)]);
                        }
                } else if (r == S && ent && (__ldg(ent) & 0xFF) != 0) {
                    const int L = __ldg(ent) & 0xFF;
                    for (int i = 0; i < L; ++i) m = max(m, __ldg(tabp + c[kr] + __ldg(ent + 4 + i)));
                } else {
                    m = box_max<D>(v.Vkey, g, decode_compact<D>(r, g, c[kr]));
                }
                if (m == kKeyInf) continue;                          // +inf + G = +inf
                const double gv = __ldcs(v.Gint + (long long)u * g.C + c[kr]);
                const long long dk = key_of(gv + val_of(m));         // the one FP64 add
                if (dk < best[kr]) { best[kr] = dk; bu[kr] = u; }
            }
            __syncthreads();                                         // the slices are free again
        }
#pragma unroll
        for (int kr = 0; kr < KR; ++kr)
            commit_cell<D, false, MARK>(v, inF[kr] ? c[kr] : 0, best[kr], inF[kr] ? bu[kr] : -1, false, &dummy);
    }
    if (relaxed) atomicAdd((unsigned long long*)&k->relaxed, (unsigned long long)relaxed);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

struct TileState {
    TileParams tp;
    CUtensorMap tm[4];        // Vkey, M2, M3, M33 as [planes][n1][n0] int64
    size_t smem;
    int blocks[2];            // grid of the kernel without / with marking (0: not set up yet)
};

// The tile geometry and tensor maps of an abstraction's tables, or an error
// when the abstraction does not fit the tile form (no shape table, dim 0
// wider than 256 cells or odd, staged rows too wide).  tables: Vkey, M2, M3,
// M33 (M33 may be NULL).
int tile_setup(const bf_abstraction* a, long long* const tables[4], TileState** out) {
    *out = nullptr;
    const GridDesc& g = a->g;
    if (!a->d_shape || a->g.D < 2 || g.n[0] > 256 || (g.n[0] & 1) || g.U > 254) return BF_ERR_UNSUPPORTED;
    const long long P = a->nplanes;
    // the dim-0 offsets of every plane entry
    const long long n = P * g.U;
    unsigned long long* S = new unsigned long long[(size_t)n];
    cudaError_t e = cudaMemcpy(S, a->d_shape, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { delete[] S; return bfh::cuda_fail(e, "tile setup"); }
    int lo = 0, hi = 0, maxsl = 1;
    bool any = false;
    for (long long i = 0; i < n; ++i) {
        const unsigned long long r = S[i];
        const int w0 = (int)((r >> 8) & 0x7F);
        if (w0 == 0) continue;
        const int rel0 = (int)(signed char)(r & 0xFF);
        const int amax = w0 < 3 ? 0 : w0 - 3;
        if (!any || rel0 < lo) lo = rel0;
        if (!any || rel0 + amax > hi) hi = rel0 + amax;
        int sl = 1;
        for (int d = 2; d < g.D; ++d) sl *= (int)((r >> (16 * d + 8)) & 0x7F);
        if (sl > maxsl) maxsl = sl;
        any = true;
    }
    delete[] S;
    if (!any) return BF_ERR_UNSUPPORTED;
    TileState* t = new TileState;
    memset(t, 0, sizeof *t);
    TileParams& tp = t->tp;
    tp.xbase = lo >= 0 ? (lo & ~1) : -(((-lo) + 1) & ~1);
    tp.BX = ((g.n[0] + hi - tp.xbase) + 1) & ~1;
    tp.RY = kTileRows + 3;
    tp.XT = g.n[0] <= 64 ? 64 : (g.n[0] <= 128 ? 128 : 256);
    tp.nbands = (g.n[1] + kTileRows - 1) / kTileRows;
    tp.ntiles = P * tp.nbands;
    tp.maxsl = maxsl < kTileSlices ? maxsl : kTileSlices;
    if (tp.BX > 256) { delete t; return BF_ERR_UNSUPPORTED; }
    t->smem = (size_t)tp.maxsl * (((size_t)tp.RY * tp.BX + 15) & ~(size_t)15) * 8 + 128;
    // cuTensorMapEncodeTiled through the runtime's driver entry point
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
        delete t;
        bfh::set_error("tile relax: cuTensorMapEncodeTiled is not available");
        return BF_ERR_UNSUPPORTED;
    }
    EncodeTiledFn encode = reinterpret_cast<EncodeTiledFn>(fn);
    const cuuint64_t dims[3] = {(cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)P};
    const cuuint64_t strides[2] = {(cuuint64_t)g.n[0] * 8, (cuuint64_t)g.n[0] * g.n[1] * 8};
    const cuuint32_t box[3] = {(cuuint32_t)tp.BX, (cuuint32_t)tp.RY, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    for (int i = 0; i < 4; ++i) {
        long long* ptr = tables[i] ? tables[i] : tables[0];
        const CUresult r = encode(&t->tm[i], CU_TENSOR_MAP_DATA_TYPE_INT64, 3, ptr, dims, strides, box, estr,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            delete t;
            bfh::set_error("tile relax: tensor map encoding failed (%d)", (int)r);
            return BF_ERR_UNSUPPORTED;
        }
    }
    *out = t;
    return BF_OK;
}

void tile_free(TileState* t) { delete t; }

template <int D, bool MARK, int KR>
static int launch_kr(const InstView& v, TileState* t, cudaStream_t st) {
    auto kern = k_relax_tile<D, MARK, KR>;
    int& blocks = t->blocks[MARK ? 1 : 0];
    if (!blocks) {
        BF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->smem));
        int per_sm = 1, dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, t->smem);
        long long b = (long long)(per_sm < 1 ? 1 : per_sm) * sms;
        if (b > t->tp.ntiles) b = t->tp.ntiles;
        blocks = (int)b;
    }
    kern<<<blocks, 256, t->smem, st>>>(v, t->tp, t->tm[0], t->tm[1], t->tm[2], t->tm[3]);
    return BF_OK;
}

template <int D, bool MARK>
static int launch_m(const InstView& v, TileState* t, cudaStream_t st) {
    switch (t->tp.XT) {
        case 64: return launch_kr<D, MARK, kTileRows * 64 / 256>(v, t, st);
        case 128: return launch_kr<D, MARK, kTileRows * 128 / 256>(v, t, st);
        default: return launch_kr<D, MARK, kTileRows * 256 / 256>(v, t, st);
    }
}

// One tile relax launch (the kernel returns at once unless the pass's F1
// holds at least v.dense_min cells).
int launch_relax_tile(const InstView& v, TileState* t, bool mark, cudaStream_t st) {
    switch (v.g.D) {
        case 2: return mark ? launch_m<2, true>(v, t, st) : launch_m<2, false>(v, t, st);
        case 3: return mark ? launch_m<3, true>(v, t, st) : launch_m<3, false>(v, t, st);
        default: return mark ? launch_m<4, true>(v, t, st) : launch_m<4, false>(v, t, st);
    }
}
