// noalloc.cu -- bf_solve_noalloc: the solve of bf_solve for callers that
// cannot let the library allocate device memory (see bfgpu.h).  The paper has
// no counterpart to this entry point.
//
// All working state lives in g_scratch, a file-scope device array of fixed
// size.  Host code must not use the name g_scratch as an address (on the host
// it only stands in for the symbol); the device address is looked up on each
// call with cudaGetSymbolAddress and passed to the kernels.  The passes
// are the same device routines as bf_solve (solve_core.cuh), launched from
// the host in groups of kPassesPerCheck, with one read of the counters per
// group; kernels launched after the loop condition turned false return at
// once.
#include <cstring>

#include "solve_core.cuh"

using namespace bfk;

namespace {

constexpr size_t kScratchBytes = BF_NOALLOC_SCRATCH_BYTES;
constexpr int kPassesPerCheck = 8;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch on the current device, looked up on every call
// (a cached address would go stale when the context is reset).
int scratch_base(void** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return bfh::cuda_fail(e, "cudaGetSymbolAddress(g_scratch)");
    *out = p;
    return BF_OK;
}

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

// Carve the scratch array; returns the bytes needed (may exceed the array).
struct Layout {
    size_t ctr, vkey, vnew, m2, m3, fbits, cells, chg, gint, total;
};

Layout plan(long long C, int U) {
    const long long S = (C + 31) / 32;
    Layout L;
    size_t o = 0;
    L.ctr = o;   o += round256(sizeof(Counters));
    L.vkey = o;  o += round256(8 * (size_t)C);
    L.vnew = o;  o += round256(8 * (size_t)C);
    L.m2 = o;    o += round256(8 * (size_t)C);
    L.m3 = o;    o += round256(8 * (size_t)C);
    L.fbits = o; o += round256(4 * (size_t)S);
    L.cells = o; o += round256(4 * (size_t)C);
    L.chg = o;   o += round256(4 * (size_t)C);
    L.gint = o;  o += round256(8 * (size_t)C * U);
    L.total = o;
    return L;
}

__global__ void k_na_counters(Counters* ctr, long long cap) {
    memset(ctr, 0, sizeof(Counters));
    ctr->cap = cap;
}

__global__ void k_na_costs(long long C, int U, const double* __restrict__ G,
                           const unsigned char* __restrict__ avoid, double* Gint, Counters* ctr) {
    init_costs_body(C, U, G, avoid, Gint, ctr);
}

__global__ void k_na_values(long long C, const double* __restrict__ terminal,
                            const unsigned char* __restrict__ target, const unsigned char* __restrict__ avoid,
                            long long* Vkey, long long* Vnew, unsigned char* mu, int* chg, Counters* ctr) {
    init_values_body(C, terminal, target, avoid, Vkey, Vnew, mu, chg, nullptr, ctr);
}

__global__ void k_na_tables(InstView v) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < v.g.C;
         c += (long long)gridDim.x * blockDim.x)
        table_entry(v, c);
}

template <int D, int FMT>
__global__ void __launch_bounds__(256, (FMT == kBoxRecompute || FMT == kBoxHybrid) ? 2 : 4) k_na_relax(InstView v) {
    Counters* k = v.ctr;
    if (k->done) return;
    const long long round = k->round;
    const int ncur = k->ncur;
    const int nchunks = (ncur + 31) >> 5;
    const int wpb = blockDim.x >> 5;
    const int nwarps = gridDim.x * wpb;
    long long relaxed = 0;
    int exact = 0;
    for (int ch = blockIdx.x * wpb + (threadIdx.x >> 5); ch < nchunks; ch += nwarps)
        relaxed += relax_chunk<D, FMT, false>(v, ch << 5, ncur - (ch << 5), round, &exact);
    if ((threadIdx.x & 31) == 0 && relaxed)
        atomicAdd((unsigned long long*)&k->relaxed, (unsigned long long)relaxed);
}

template <int D>
__global__ void __launch_bounds__(256, 4) k_na_propagate(InstView v, int commit) {
    Counters* k = v.ctr;
    if (k->done) return;
    const int nchg = k->nchg;
    const int wpb = blockDim.x >> 5;
    const int nwarps = gridDim.x * wpb;
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < nchg; i += nwarps)
        propagate_entry<D>(v, i, nchg, commit != 0);
}

__global__ void __launch_bounds__(256) k_na_compact(InstView v, long long nwords, int init) {
    Counters* k = v.ctr;
    if (k->done) return;
    for (long long wb = (long long)blockIdx.x * blockDim.x; wb < nwords; wb += (long long)gridDim.x * blockDim.x)
        compact_words(v, (int)wb, (int)nwords);
    if (!init) {
        const int nchg = k->nchg;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nchg; i += gridDim.x * blockDim.x)
            refresh_tables(v, v.chg[i]);
    }
    if (last_block_done(&k->blocks_done)) {
        if (init) start_loop(v);
        else finish_pass(v);
    }
}

__global__ void k_na_output(long long C, const long long* __restrict__ Vkey, double* V) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < C;
         c += (long long)gridDim.x * blockDim.x)
        V[c] = val_of(Vkey[c]);
}

int sms() {
    int dev = 0, n = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

template <typename K>
int wave(K kernel) {
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0);
    return (per_sm < 1 ? 1 : per_sm) * sms();
}

template <int D, int FMT>
void launch_relax(const InstView& v, int blocks, cudaStream_t st) {
    k_na_relax<D, FMT><<<blocks, 256, 0, st>>>(v);
}

template <int D>
int run(const bf_abstraction* a, const InstView& v, const double* G, const unsigned char* target,
        const unsigned char* avoid, const double* terminal, double* V, cudaStream_t st,
        Counters* hc_out) {
    const long long C = a->g.C;
    const int U = a->g.U;
    const long long S = (C + 31) / 32;
    const int fmt = a->box_fmt;
    const int nb = (int)(((C + 255) / 256) < (long long)sms() * 8 ? (C + 255) / 256 : (long long)sms() * 8);
    const int cb = (int)(((S + 255) / 256) < (long long)sms() * 8 ? (S + 255) / 256 : (long long)sms() * 8);
    const int rb = fmt == kBoxRecompute ? wave(k_na_relax<D, kBoxRecompute>)
                 : fmt == kBoxHybrid ? wave(k_na_relax<D, kBoxHybrid>)
                 : fmt == kBoxCompact ? wave(k_na_relax<D, kBoxCompact>) : wave(k_na_relax<D, kBoxWide>);
    const int pb = wave(k_na_propagate<D>);
    k_na_costs<<<nb, 256, 0, st>>>(C, U, G, avoid, const_cast<double*>(v.Gint), v.ctr);
    k_na_values<<<nb, 256, 0, st>>>(C, terminal, terminal ? nullptr : target, avoid, v.Vkey, v.Vnew, v.mu,
                                    v.chg, v.ctr);
    k_na_tables<<<nb, 256, 0, st>>>(v);
    k_na_propagate<D><<<pb, 256, 0, st>>>(v, 0);
    k_na_compact<<<cb, 256, 0, st>>>(v, S, 1);
    BF_CUDA(cudaGetLastError());
    Counters hc;
    for (;;) {
        BF_CUDA(cudaMemcpyAsync(&hc, v.ctr, sizeof hc, cudaMemcpyDeviceToHost, st));
        BF_CUDA(cudaStreamSynchronize(st));
        if (hc.done) break;
        for (int i = 0; i < kPassesPerCheck; ++i) {
            switch (fmt) {
                case kBoxCompact: launch_relax<D, kBoxCompact>(v, rb, st); break;
                case kBoxRecompute: launch_relax<D, kBoxRecompute>(v, rb, st); break;
                case kBoxHybrid: launch_relax<D, kBoxHybrid>(v, rb, st); break;
                default: launch_relax<D, kBoxWide>(v, rb, st); break;
            }
            k_na_propagate<D><<<pb, 256, 0, st>>>(v, 1);
            k_na_compact<<<cb, 256, 0, st>>>(v, S, 0);
        }
        BF_CUDA(cudaGetLastError());
    }
    k_na_output<<<nb, 256, 0, st>>>(C, v.Vkey, V);
    BF_CUDA(cudaGetLastError());
    BF_CUDA(cudaStreamSynchronize(st));
    *hc_out = hc;
    return BF_OK;
}

// Device (or managed) memory of device dev, or NULL.
bool on_device(const void* p, int dev) {
    if (!p) return true;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" int bf_solve_noalloc(const bf_abstraction* a, const double* G, const uint8_t* target,
                                const uint8_t* avoid, const double* terminal, int64_t max_iters,
                                double* V, uint8_t* mu, int64_t* iters, int32_t* status, void* stream) {
    if (!a || !G || !V || !mu || !iters || !status || (!target && !terminal)) {
        bfh::set_error("bf_solve_noalloc: NULL argument (need G, V, mu, iters, status and target or terminal)");
        return BF_ERR_INVALID;
    }
    int dev = 0;
    BF_CUDA(cudaGetDevice(&dev));
    if (!on_device(G, dev) || !on_device(target, dev) || !on_device(avoid, dev) || !on_device(terminal, dev) ||
        !on_device(V, dev) || !on_device(mu, dev)) {
        bfh::set_error("bf_solve_noalloc: every array must be device memory of the current device "
                       "(it does not stage host arrays)");
        return BF_ERR_INVALID;
    }
    const long long C = a->g.C;
    const int U = a->g.U;
    const Layout L = plan(C, U);
    if (L.total > kScratchBytes) {
        bfh::set_error("bf_solve_noalloc: %lld cells x %d inputs need %zu bytes of scratch, more than the "
                       "%zu bytes this entry point holds; use bf_solve", C, U, L.total, kScratchBytes);
        return BF_ERR_INVALID;
    }
    void* base = nullptr;
    int rc = scratch_base(&base);
    if (rc) return rc;
    unsigned char* s = static_cast<unsigned char*>(base);
    cudaStream_t st = (cudaStream_t)stream;
    InstView v;
    memset(&v, 0, sizeof v);
    view_from_abs(v, a);
    v.Gint = reinterpret_cast<const double*>(s + L.gint);
    v.Vkey = reinterpret_cast<long long*>(s + L.vkey);
    v.Vnew = reinterpret_cast<long long*>(s + L.vnew);
    v.M2 = reinterpret_cast<long long*>(s + L.m2);
    v.M3 = reinterpret_cast<long long*>(s + L.m3);
    v.mu = mu;
    v.fbits = reinterpret_cast<unsigned*>(s + L.fbits);
    v.cells = reinterpret_cast<int*>(s + L.cells);
    v.chg = reinterpret_cast<int*>(s + L.chg);
    v.ctr = reinterpret_cast<Counters*>(s + L.ctr);
    long long cap = C;
    if (max_iters > 0 && max_iters < cap) cap = max_iters;
    // what must start at zero: the counters (including the last-block counter
    // of the compaction) and the frontier bitmap
    k_na_counters<<<1, 1, 0, st>>>(v.ctr, cap);
    BF_CUDA(cudaMemsetAsync(v.fbits, 0, 4 * (size_t)((C + 31) / 32), st));
    Counters hc;
    switch (a->g.D) {
        case 1: rc = run<1>(a, v, G, target, avoid, terminal, V, st, &hc); break;
        case 2: rc = run<2>(a, v, G, target, avoid, terminal, V, st, &hc); break;
        case 3: rc = run<3>(a, v, G, target, avoid, terminal, V, st, &hc); break;
        default: rc = run<4>(a, v, G, target, avoid, terminal, V, st, &hc); break;
    }
    if (rc) return rc;
    if (hc.err) {
        bfh::set_error("bf_solve_noalloc: NaN, -inf or |value| > 2^64 in G or the terminal cost");
        return BF_ERR_INVALID;
    }
    *iters = hc.round;
    *status = hc.status;
    return BF_OK;
}
