// solve.cu -- bf_solve: Algorithm 1 (generalized Bellman-Ford-Yen, Sec. IV-A)
// on one abstraction, on one GPU.
//
// Device state per solve (workspace, cached in the abstraction handle): the
// InstView arrays of solve_core.cuh (values as int64 keys, window-max tables,
// frontier bitmap and compacted frontier list, changed list) plus
//   Gint   f64 [U][C]  running cost, input-major (coalesced per input),
//                      +inf on avoid cells; -0 read as +0.
//
// Round driver: the passes run inside one CUDA graph whose body (relax ->
// propagate -> compact) sits in a conditional WHILE node; the last block of
// compact evaluates "F1 != empty and i < cap" on the device and sets the
// condition, so a whole solve is one graph launch with no host round trip per
// pass.  The set-up (lines 1-10 of Algorithm 1) and the output conversion are
// ordinary launches on the caller's stream.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include <math_constants.h>

#include "solve_core.cuh"

using namespace bfk;

// Tile relax for dense passes (solve_tile.cu).
struct TileState;
int tile_setup(const bf_abstraction* a, long long* const tables[4], TileState** out);
void tile_free(TileState* t);
int launch_relax_tile(const InstView& v, TileState* t, bool mark, cudaStream_t st);

// Mean predecessor-box rows up to which relax marks the next frontier itself.
constexpr double kFuseMarkRows = 64.0;

struct bf_solve_ws {
    long long C = 0;
    int U = 0, D = 0;
    int device = 0;
    long long nwords = 0;
    long long* Vkey = nullptr;
    long long* Vnew = nullptr;
    long long* M2 = nullptr;
    long long* M3 = nullptr;
    long long* M33 = nullptr;       // D >= 2: 3 x 3 windows on dims 0-1 (not with a successor class)
    long long* M33P = nullptr;      // plane-pair table (allocated when a schedule first asks for it)
    int pz = 0;                     // its dim (2 .. D - 1), 0: the gathers do not read it
    int masked = 0;                 // the plane relax reads the cell masks: 1 = inputs in turn (two
                                    // or four per iteration by `pair`), 2 = the pairs queued over the
                                    // lanes (one or two per lane and round by `pair`)
    int pm_blocks_full[2] = {0, 0}; // one full wave of the masked plane relax kernel, by `pair`
    int pq_blocks_full[2] = {0, 0}; // the same for the pair-queue kernel
    bool pfront = false;            // per-input frontier (with the per-input templates)
    unsigned* ubits = nullptr;      // [2][U][S] (allocated when a schedule first asks for it)
    bool use33 = false;             // gathers read M33 (bf_tune may switch it on)
    bool use_plane = true;          // relax reads the plane lookup lists (when the abstraction has them)
    bool use_tmpl = true;           // marking reads the predecessor templates (when the abstraction has them)
    unsigned char* mu = nullptr;
    unsigned* fbits = nullptr;
    int* cells = nullptr;
    int* chg = nullptr;
    double* Gint = nullptr;
    Counters* ctr = nullptr;
    int* stamp = nullptr;           // counting mode only
    long long* cand_key = nullptr;  // input slices of small frontiers
    int* cand_u = nullptr;
    int* slice_cnt = nullptr;
    long long slice_cap = 0;
    // staging for host inputs / outputs
    double* stage_G = nullptr;      // [C][U]
    double* stage_T = nullptr;      // [C]
    unsigned char* stage_tgt = nullptr;
    unsigned char* stage_avoid = nullptr;
    double* stage_V = nullptr;
    long long* trace = nullptr;
    long long trace_cap = 0;
    // graph of the pass loop
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    int relax_blocks = 0, prop_blocks = 0, compact_blocks = 0;
    int relax_blocks_full = 0;      // one full wave of the relax kernel
    int pl_blocks_full[4] = {0, 0, 0, 0};   // one full wave of the plane relax kernel, by form
                                            // (pair + 2 occ)
    bool pair = false;              // the plane relax kernel takes two inputs per iteration
    bool occ = false;               // ... with one block per SM more
    int dense_pct = 0;              // passes whose F1 holds at least this share (percent) of the
                                    // cells take the tile relax; 0: never
    TileState* tile = nullptr;      // tile geometry and tensor maps (set up on first use)
    bool tile_failed = false;       // the abstraction does not fit the tile form
    unsigned* f1bits = nullptr;     // [S] F1 as a bitmap (tile relax)
    unsigned long long* fc[2] = {nullptr, nullptr};   // frontier cache buffers [U - K][fc_alloc]
    long long* fc_tag = nullptr;                      // [C]
    long long fc_alloc = 0;         // cells the buffers hold
    long long fc_cap = 0;           // cells the current solve caches (0: none)
    int slice_target = kSliceTarget;
    bool tuned = false;             // bf_tune chose the schedule below
    bool fuse_mark = true;          // relax marks F2 (no propagate launch per pass)
    int inplace = 0;                // schedule the views (and the graph) were made for
    // successor class (allocated on first use)
    int cls = 0;                    // class in use for the views (and the graph)
    unsigned char* rmask = nullptr; // [C] device copy of the class mask
    double* GRint = nullptr;        // [U][C]
    long long* VN = nullptr;
    long long* VR = nullptr;
    long long* M2R = nullptr;
    long long* M3R = nullptr;
    double* stage_GR = nullptr;
    std::mutex mtx;
};

void bf_solve_ws_free(bf_solve_ws* w) {
    if (!w) return;
    if (w->exec) cudaGraphExecDestroy(w->exec);
    if (w->graph) cudaGraphDestroy(w->graph);
    cudaFree(w->Vkey); cudaFree(w->Vnew); cudaFree(w->M2); cudaFree(w->M3); cudaFree(w->M33); cudaFree(w->M33P); cudaFree(w->mu);
    cudaFree(w->fbits); cudaFree(w->cells); cudaFree(w->chg); cudaFree(w->Gint); cudaFree(w->ctr);
    cudaFree(w->stage_G); cudaFree(w->stage_T); cudaFree(w->stage_tgt); cudaFree(w->stage_avoid);
    cudaFree(w->stage_V); cudaFree(w->trace); cudaFree(w->stamp);
    cudaFree(w->cand_key); cudaFree(w->cand_u); cudaFree(w->slice_cnt);
    cudaFree(w->rmask); cudaFree(w->GRint); cudaFree(w->VN); cudaFree(w->VR); cudaFree(w->M2R);
    cudaFree(w->M3R); cudaFree(w->stage_GR);
    cudaFree(w->f1bits);
    cudaFree(w->ubits);
    cudaFree(w->fc[0]); cudaFree(w->fc[1]); cudaFree(w->fc_tag);
    if (w->tile) tile_free(w->tile);
    delete w;
}

// ---------------------------------------------------------------------------
// set-up kernels
// ---------------------------------------------------------------------------

// Set-up kernels (bodies in solve_core.cuh, shared with bf_solve_noalloc).
__global__ void k_init_costs(long long C, int U, const double* __restrict__ G,
                             const unsigned char* __restrict__ avoid, double* Gint, Counters* ctr) {
    init_costs_body(C, U, G, avoid, Gint, ctr);
}

__global__ void k_init_values(long long C, const double* __restrict__ terminal,
                              const unsigned char* __restrict__ target,
                              const unsigned char* __restrict__ avoid, long long* Vkey,
                              long long* Vnew, unsigned char* mu, int* chg, int* stamp,
                              Counters* ctr) {
    init_values_body(C, terminal, target, avoid, Vkey, Vnew, mu, chg, stamp, ctr);
}

__global__ void k_init_tables(InstView v) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < v.g.C;
         c += (long long)gridDim.x * blockDim.x) {
        table_entry(v, c);
        if (v.M33) table33_entry(v, c);
    }
}

__global__ void k_init_table_pair(InstView v) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < v.g.C;
         c += (long long)gridDim.x * blockDim.x)
        table33p_entry(v, c);
}

__global__ void k_init_counters(Counters* ctr, long long cap) {
    memset(ctr, 0, sizeof(Counters));
    ctr->cap = cap;
}

// ---------------------------------------------------------------------------
// pass kernels
// ---------------------------------------------------------------------------
// Generic relax (solve_stored.cu: wide and compact records;
// solve_recompute.cu, solve_hybrid.cu: the modes that regenerate boxes).
void launch_relax_stored(const InstView& v, int fmt, bool count, bool mark, int blocks, cudaStream_t st);
int relax_wave_stored(int D, int fmt);
void launch_relax_recompute(const InstView& v, bool count, bool mark, int blocks, cudaStream_t st);
int relax_wave_recompute(int D);
void launch_relax_hybrid(const InstView& v, bool count, bool mark, int blocks, cudaStream_t st);
int relax_wave_hybrid(int D);

// Relax on abstractions with plane lookup lists (solve_plane.cu).
int plane_relax_wave(int D, bool pair, bool occ);
void launch_relax_plane(const InstView& v, bool count, bool mark, bool pair, bool occ, int blocks, cudaStream_t st);
int masked_relax_wave(int D, bool quad);
void launch_relax_masked(const InstView& v, bool mark, bool quad, int blocks, cudaStream_t st);
int queue_relax_wave(int D, int U, bool two);
void launch_relax_queue(const InstView& v, bool mark, bool two, int blocks, cudaStream_t st);

// Propagate (warp per changed cell): set F2's bits from the changed list
// (set-up: the finite cells; the passes mark F2 inside relax).
template <int D>
__global__ void __launch_bounds__(256, 4) k_propagate(InstView v, int commit) {
    Counters* k = v.ctr;
    if (k->done) return;
    const int nchg = k->nchg;
    const int wpb = blockDim.x >> 5;
    const int nwarps = gridDim.x * wpb;
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < nchg; i += nwarps)
        propagate_entry<D>(v, i, nchg, commit != 0);
}

// Compact F2 into the next frontier list, refresh the window tables around
// the changed cells, and (last block) close the pass or, after the set-up,
// decide whether to loop.  With a graph the last block sets the WHILE
// condition.
__global__ void __launch_bounds__(256) k_compact(InstView v, long long nwords, int init,
                                                 cudaGraphConditionalHandle h, int use_graph) {
    Counters* k = v.ctr;
    if (k->done) {
        if (use_graph && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0);
        return;
    }
    for (long long wb = (long long)blockIdx.x * blockDim.x; wb < nwords; wb += (long long)gridDim.x * blockDim.x)
        compact_words(v, (int)wb, (int)nwords);
    if (!init) {
        // commit W of the changed cells and refresh the window tables around them
        const int nchg = k->nchg;
        const int round = (int)k->round;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nchg; i += gridDim.x * blockDim.x) {
            const int y = v.chg[i];
            v.Vkey[y] = v.Vnew[y];
            if (v.stamp) v.stamp[y] = round;
            refresh_tables(v, y);
        }
    }
    if (last_block_done(&k->blocks_done)) {
        const int cont = init ? start_loop(v) : finish_pass(v);
        if (use_graph) cudaGraphSetConditional(h, cont);
    }
}

// First node of the graph: copy "not done" into the WHILE condition.
__global__ void k_loop_cond(Counters* k, cudaGraphConditionalHandle h) {
    cudaGraphSetConditional(h, k->done ? 0 : 1);
}

__global__ void k_output(long long C, const long long* __restrict__ Vkey, double* V) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < C;
         c += (long long)gridDim.x * blockDim.x)
        V[c] = val_of(Vkey[c]);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int sm_count() {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

static int blocks_for(long long work, int threads) {
    long long need = (work + threads - 1) / threads;
    long long cap = (long long)sm_count() * 8;
    if (need < 1) need = 1;
    return (int)(need < cap ? need : cap);
}

template <typename K>
static int full_wave(K kernel, int threads) {
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    if (per_sm < 1) per_sm = 1;
    return per_sm * sm_count();
}

// Device bytes a bf_solve workspace of this abstraction holds at most: state,
// window tables, costs, staging of host inputs and outputs, slice buffers
// (one wave of 8 warps per block on every SM, at most 8 blocks per SM) and
// the F1 bitmap of the tile relax.
size_t solve_ws_bytes(const bf_abstraction* a) {
    const size_t C = (size_t)a->g.C, U = (size_t)a->g.U, S = (C + 31) / 32;
    const size_t slice = 2ull * kSliceTargetMax * (size_t)sm_count() * 8 * 8 * 32;
    return C * (6 * 8 + 1 + 4 + 4) + 4 * S * (2 * U + 1) + 2 * 8 * C * U + 8 * C + 8 * C + 2 * C + slice * 12 + slice / 8 + 4 * S +
           sizeof(Counters);
}

static int ws_get(const bf_abstraction* a, bf_solve_ws** out) {
    bf_abstraction* am = const_cast<bf_abstraction*>(a);
    if (am->ws) { *out = am->ws; return BF_OK; }
    bf_solve_ws* w = new bf_solve_ws;
    w->C = a->g.C;
    w->U = a->g.U;
    w->D = a->g.D;
    cudaGetDevice(&w->device);
    w->nwords = (a->g.C + 31) / 32;
    const long long C = w->C, S = w->nwords;
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
    A((void**)&w->Vkey, 8 * C);
    A((void**)&w->Vnew, 8 * C);
    A((void**)&w->M2, 8 * C);
    A((void**)&w->M3, 8 * C);
    if (w->D >= 2) A((void**)&w->M33, 8 * C);
    A((void**)&w->mu, C);
    A((void**)&w->fbits, 4 * S);
    A((void**)&w->cells, 4 * C);
    A((void**)&w->chg, 4 * C);
    A((void**)&w->Gint, 8 * C * w->U);
    A((void**)&w->ctr, sizeof(Counters));
    if (e != cudaSuccess) { bf_solve_ws_free(w); return bfh::cuda_fail(e, "bf_solve workspace"); }
    am->ws = w;
    *out = w;
    return BF_OK;
}

static InstView make_view(const bf_abstraction* a, bf_solve_ws* w) {
    InstView v;
    memset(&v, 0, sizeof v);
    view_from_abs(v, a);
    v.Gint = w->Gint;
    v.Vkey = w->Vkey;
    v.Vnew = w->Vnew;
    v.M2 = w->M2;
    v.M3 = w->M3;
    v.M33 = (w->cls || !w->use33) ? nullptr : w->M33;   // the class tables have no 3 x 3 windows
    if (v.M33 && w->pz >= 2 && w->M33P && a->d_poffs[w->pz]) {
        v.M33P = w->M33P;
        v.pz = w->pz;
    }
    if (!w->cls && w->use_plane) {
        v.poffs = a->d_poffs[v.M33P ? v.pz : (v.M33 ? 1 : 0)];
        if (w->masked) v.fmask = a->d_fmask;
    }
    if (w->use_tmpl && a->d_tent) {
        v.tptr = a->d_tptr;
        v.tent = a->d_tent;
        if (w->pfront && a->d_uent && w->ubits && !w->cls) {
            v.uptr = a->d_uptr;
            v.uent = a->d_uent;
            v.ubits = w->ubits;
        }
    }
    v.nwords = w->nwords;
    if (w->fc_cap > 0) {
        v.fc[0] = w->fc[0];
        v.fc[1] = w->fc[1];
        v.fc_tag = w->fc_tag;
        v.fc_cap = w->fc_cap;
    }
    if (w->dense_pct > 0 && w->tile && !w->cls) {
        v.f1bits = w->f1bits;
        v.dense_min = (a->g.C * w->dense_pct + 99) / 100;
        if (v.dense_min < 1) v.dense_min = 1;
    }
    v.mu = w->mu;
    v.fbits = w->fbits;
    v.cells = w->cells;
    v.chg = w->chg;
    v.ctr = w->ctr;
    v.trace = w->trace;
    v.trace_cap = w->trace_cap;
    v.cand_key = w->cand_key;
    v.cand_u = w->cand_u;
    v.slice_cnt = w->slice_cnt;
    v.slice_cap = w->slice_cap;
    v.slice_target = w->slice_target;
    v.inplace = w->inplace;
    if (w->cls) {
        v.rmask = w->rmask;
        v.GRint = w->GRint;
        v.VN = w->VN;
        v.VR = w->VR;
        v.M2R = w->M2R;
        v.M3R = w->M3R;
    }
    return v;
}

void launch_relax_cls(const InstView& v, bool mark, int blocks, cudaStream_t st);         // solve_cls.cu
void launch_relax_cls_count(const InstView& v, bool mark, int blocks, cudaStream_t st);   // solve_cls_count.cu

// Launch one pass: relax, then (unless relax marks the next frontier itself)
// propagate, then compact (which commits W and closes the pass).  With timing
// events, relax and the rest of the pass are bracketed.
struct PassTimers {
    cudaEvent_t e[4];
};

template <int D, int FMT>
static void launch_relax(bf_solve_ws* w, const InstView& v, cudaStream_t st, bool count) {
    if constexpr (FMT == kBoxCompact && D >= 2) {
        if (v.fmask && !count && v.poffs && v.g.U <= kPlaneUMax) {
            const int full = (w->masked == 2 ? w->pq_blocks_full : w->pm_blocks_full)[w->pair ? 1 : 0];
            if (full > 0) {
                int b = (int)(((long long)w->relax_blocks * full + w->relax_blocks_full - 1) / w->relax_blocks_full);
                if (b < 1) b = 1;
                if (w->masked == 2) launch_relax_queue(v, w->fuse_mark, w->pair, b, st);
                else launch_relax_masked(v, w->fuse_mark, w->pair, b, st);
                return;
            }
        }
        const int form = count ? 0 : (w->pair ? 1 : 0) + (w->occ ? 2 : 0);
        const int full = w->pl_blocks_full[form];
        if (v.poffs && v.g.U <= kPlaneUMax && full > 0) {
            // the same share of its own wave as the generic kernel's grid
            int b = (int)(((long long)w->relax_blocks * full + w->relax_blocks_full - 1) / w->relax_blocks_full);
            if (b < 1) b = 1;
            launch_relax_plane(v, count, w->fuse_mark, w->pair, w->occ && !count, b, st);
            return;
        }
    }
    if (FMT == kBoxRecompute) launch_relax_recompute(v, count, w->fuse_mark, w->relax_blocks, st);
    else if (FMT == kBoxHybrid) launch_relax_hybrid(v, count, w->fuse_mark, w->relax_blocks, st);
    else launch_relax_stored(v, FMT, count, w->fuse_mark, w->relax_blocks, st);
}

template <int D>
static void launch_pass(const bf_abstraction* a, bf_solve_ws* w, const InstView& v, cudaStream_t st,
                        cudaGraphConditionalHandle h, int use_graph, bool count, PassTimers* tm) {
    if (tm) cudaEventRecord(tm->e[0], st);
    // dense passes: the tile relax (the list relax below then returns at once)
    if (v.f1bits && !count) launch_relax_tile(v, w->tile, w->fuse_mark, st);
    if (v.rmask) {
        if (count) launch_relax_cls_count(v, w->fuse_mark, w->relax_blocks, st);
        else launch_relax_cls(v, w->fuse_mark, w->relax_blocks, st);
    }
    else switch (a->box_fmt) {
        case kBoxCompact: launch_relax<D, kBoxCompact>(w, v, st, count); break;
        case kBoxRecompute: launch_relax<D, kBoxRecompute>(w, v, st, count); break;
        case kBoxHybrid: launch_relax<D, kBoxHybrid>(w, v, st, count); break;
        default: launch_relax<D, kBoxWide>(w, v, st, count); break;
    }
    if (tm) { cudaEventRecord(tm->e[1], st); cudaEventRecord(tm->e[2], st); }
    if (!w->fuse_mark) k_propagate<D><<<w->prop_blocks, 256, 0, st>>>(v, 0);
    k_compact<<<w->compact_blocks, 256, 0, st>>>(v, w->nwords, 0, h, use_graph);
    if (tm) cudaEventRecord(tm->e[3], st);
}

static void launch_pass_any(const bf_abstraction* a, bf_solve_ws* w, const InstView& v, cudaStream_t st,
                            cudaGraphConditionalHandle h, int use_graph, bool count = false,
                            PassTimers* tm = nullptr) {
    switch (a->g.D) {
        case 1: launch_pass<1>(a, w, v, st, h, use_graph, count, tm); break;
        case 2: launch_pass<2>(a, w, v, st, h, use_graph, count, tm); break;
        case 3: launch_pass<3>(a, w, v, st, h, use_graph, count, tm); break;
        default: launch_pass<4>(a, w, v, st, h, use_graph, count, tm); break;
    }
}

// Set-up tail: the first propagate (pred of the finite cells) and compaction.
static void launch_setup_frontier(const bf_abstraction* a, bf_solve_ws* w, const InstView& v, cudaStream_t st) {
    switch (a->g.D) {
        case 1: k_propagate<1><<<w->prop_blocks, 256, 0, st>>>(v, 0); break;
        case 2: k_propagate<2><<<w->prop_blocks, 256, 0, st>>>(v, 0); break;
        case 3: k_propagate<3><<<w->prop_blocks, 256, 0, st>>>(v, 0); break;
        default: k_propagate<4><<<w->prop_blocks, 256, 0, st>>>(v, 0); break;
    }
    k_compact<<<w->compact_blocks, 256, 0, st>>>(v, w->nwords, 1, 0, 0);
}

template <int D>
static void set_blocks(const bf_abstraction* a, bf_solve_ws* w) {
    if (D >= 2 && a->box_fmt == kBoxCompact && a->d_shape && a->g.U <= kPlaneUMax) {
        for (int f = 0; f < 4; ++f) w->pl_blocks_full[f] = plane_relax_wave(D, f & 1, f >> 1);
        if (a->d_fmask)
            for (int f = 0; f < 2; ++f) {
                w->pm_blocks_full[f] = masked_relax_wave(D, f != 0);
                w->pq_blocks_full[f] = queue_relax_wave(D, a->g.U, f != 0);
            }
    }
    w->relax_blocks = a->box_fmt == kBoxRecompute ? relax_wave_recompute(D)
                      : a->box_fmt == kBoxHybrid ? relax_wave_hybrid(D) : relax_wave_stored(D, a->box_fmt);
    w->prop_blocks = full_wave(k_propagate<D>, 256);
    // marking inside relax pays when predecessor boxes are small: the marks
    // then cost less than a separate launch per pass (bf_tune may override)
    if (!w->tuned) w->fuse_mark = (a->d_tent ? a->tmpl_rows : a->pred_rows) <= kFuseMarkRows;
    w->compact_blocks = blocks_for(w->nwords, 256);
}

// Launch shapes and slice buffers (once per workspace; caller holds w->mtx).
static int ws_blocks(const bf_abstraction* a, bf_solve_ws* w, cudaStream_t st) {
    if (w->relax_blocks) return BF_OK;
    switch (a->g.D) {
        case 1: set_blocks<1>(a, w); break;
        case 2: set_blocks<2>(a, w); break;
        case 3: set_blocks<3>(a, w); break;
        default: set_blocks<4>(a, w); break;
    }
    // slice buffers: a sliced pass has nchunks < slice_target x warps and
    // fewer than 2 x slice_target x warps (chunk, slice) items
    w->relax_blocks_full = w->relax_blocks;
    long long warps = w->relax_blocks;
    for (int i = 0; i < 4; ++i)
        if (w->pl_blocks_full[i] > warps) warps = w->pl_blocks_full[i];
    for (int i = 0; i < 2; ++i) {
        if (w->pm_blocks_full[i] > warps) warps = w->pm_blocks_full[i];
        if (w->pq_blocks_full[i] > warps) warps = w->pq_blocks_full[i];
    }
    warps *= 8;
    const long long cap = 2LL * kSliceTargetMax * warps * 32;
    cudaError_t e = cudaMalloc((void**)&w->cand_key, sizeof(long long) * cap);
    if (e == cudaSuccess) e = cudaMalloc((void**)&w->cand_u, sizeof(int) * cap);
    if (e == cudaSuccess) e = cudaMalloc((void**)&w->slice_cnt, sizeof(int) * (cap / 32));
    if (e == cudaSuccess) e = cudaMemsetAsync(w->slice_cnt, 0, sizeof(int) * (cap / 32), st);
    if (e != cudaSuccess) {
        cudaFree(w->cand_key); cudaFree(w->cand_u); cudaFree(w->slice_cnt);
        w->cand_key = nullptr; w->cand_u = nullptr; w->slice_cnt = nullptr;
        w->relax_blocks = 0;
        return bfh::cuda_fail(e, "slice buffers");
    }
    w->slice_cap = cap;
    return BF_OK;
}

// Build (once per workspace) the graph: [loop condition] -> WHILE { pass }.
static int ws_graph(const bf_abstraction* a, bf_solve_ws* w) {
    if (w->exec) return BF_OK;
    cudaGraph_t graph;
    BF_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle h;
    BF_CUDA(cudaGraphConditionalHandleCreate(&h, graph, 0, cudaGraphCondAssignDefault));
    // condition node: loop while the set-up did not already finish the solve
    cudaGraphNode_t n0;
    {
        void* args[] = {(void*)&w->ctr, (void*)&h};
        cudaKernelNodeParams kp;
        memset(&kp, 0, sizeof kp);
        kp.func = (void*)k_loop_cond;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(1);
        kp.kernelParams = args;
        BF_CUDA(cudaGraphAddKernelNode(&n0, graph, nullptr, 0, &kp));
    }
    // cudaGraphNodeParams has no usable default constructor: zero raw storage
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    memset(cp_raw, 0, sizeof cp_raw);
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t nc;
    BF_CUDA(cudaGraphAddNode(&nc, graph, &n0, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    // capture one pass into the body
    cudaStream_t cs;
    BF_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    BF_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    InstView v = make_view(a, w);
    launch_pass_any(a, w, v, cs, h, 1);
    cudaGraph_t captured;
    cudaError_t e = cudaStreamEndCapture(cs, &captured);
    cudaStreamDestroy(cs);
    BF_CUDA(e);
    BF_CUDA(cudaGraphInstantiate(&w->exec, graph, 0));
    w->graph = graph;
    return BF_OK;
}

static int stage_in(const void* src, size_t bytes, void** stage, cudaStream_t st, const void** dev) {
    if (!src) { *dev = nullptr; return BF_OK; }
    if (bfh::is_device_ptr(src)) { *dev = src; return BF_OK; }
    if (!*stage) BF_CUDA(cudaMalloc(stage, bytes));
    BF_CUDA(cudaMemcpyAsync(*stage, src, bytes, cudaMemcpyHostToDevice, st));
    *dev = *stage;
    return BF_OK;
}

extern "C" int bf_solve(const bf_abstraction* a, const double* G, const uint8_t* target,
                        const uint8_t* avoid, const bf_solve_opts* opts, double* V, uint8_t* mu,
                        int64_t* iters, int32_t* status, void* stream) {
    if (!a || !G || !V || !mu || !iters || !status) {
        bfh::set_error("bf_solve: NULL argument");
        return BF_ERR_INVALID;
    }
    const double* terminal = opts ? opts->terminal : nullptr;
    if (!terminal && !target) {
        bfh::set_error("bf_solve: need a target mask or a terminal cost");
        return BF_ERR_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    bf_solve_ws* w = nullptr;
    int rc = ws_get(a, &w);
    if (rc) return rc;
    std::lock_guard<std::mutex> lock(w->mtx);
    const long long C = w->C;
    const int U = w->U;
    if ((rc = ws_blocks(a, w, st))) return rc;
    // schedule (the graph holds the view by value: rebuild it on a change)
    const int sched = opts ? opts->schedule : BF_SCHED_JACOBI;
    if (sched != BF_SCHED_JACOBI && sched != BF_SCHED_INPLACE) {
        bfh::set_error("bf_solve: unknown schedule %d", sched);
        return BF_ERR_INVALID;
    }
    const uint8_t* cls_mask = opts ? opts->succ_class : nullptr;
    const double* cls_cost = opts ? opts->G_class : nullptr;
    if (cls_mask && !cls_cost) {
        bfh::set_error("bf_solve: succ_class needs G_class");
        return BF_ERR_INVALID;
    }
    const int cls = cls_mask ? 1 : 0;
    if (sched != w->inplace || cls != w->cls) {
        if (w->exec) { cudaGraphExecDestroy(w->exec); w->exec = nullptr; }
        if (w->graph) { cudaGraphDestroy(w->graph); w->graph = nullptr; }
        w->inplace = sched;
        w->cls = cls;
    }
    if (cls && !w->VN) {
        BF_CUDA(cudaMalloc((void**)&w->rmask, C));
        BF_CUDA(cudaMalloc((void**)&w->GRint, sizeof(double) * C * U));
        BF_CUDA(cudaMalloc((void**)&w->VN, 8 * C));
        BF_CUDA(cudaMalloc((void**)&w->VR, 8 * C));
        BF_CUDA(cudaMalloc((void**)&w->M2R, 8 * C));
        BF_CUDA(cudaMalloc((void**)&w->M3R, 8 * C));
    }
    // frontier cache of the regenerated records (recompute / hybrid modes);
    // the graph holds the view by value: rebuild it when the size changes
    {
        long long want = (opts && opts->frontier_cache > 0 && a->nstored < U &&
                          (a->box_fmt == kBoxRecompute || a->box_fmt == kBoxHybrid))
                             ? (opts->frontier_cache < C ? opts->frontier_cache : C) : 0;
        if (want < 0) want = 0;
        if (want > w->fc_alloc) {
            cudaFree(w->fc[0]); cudaFree(w->fc[1]);
            w->fc[0] = w->fc[1] = nullptr;
            w->fc_alloc = 0;
            const size_t n = (size_t)want * (size_t)(U - a->nstored);
            BF_CUDA(cudaMalloc((void**)&w->fc[0], 8 * n));
            BF_CUDA(cudaMalloc((void**)&w->fc[1], 8 * n));
            if (!w->fc_tag) BF_CUDA(cudaMalloc((void**)&w->fc_tag, 8 * C));
            w->fc_alloc = want;
        }
        if (want != w->fc_cap) {
            w->fc_cap = want;
            if (w->exec) { cudaGraphExecDestroy(w->exec); w->exec = nullptr; }
            if (w->graph) { cudaGraphDestroy(w->graph); w->graph = nullptr; }
        }
    }
    // trace buffer (device side), sized to the request
    const long long tcap = (opts && opts->trace) ? opts->trace_cap : 0;
    if (tcap > w->trace_cap) {
        cudaFree(w->trace);
        w->trace = nullptr;
        w->trace_cap = 0;
        BF_CUDA(cudaMalloc((void**)&w->trace, sizeof(long long) * 4 * tcap));
        w->trace_cap = tcap;
        if (w->exec) { cudaGraphExecDestroy(w->exec); w->exec = nullptr; }
        if (w->graph) { cudaGraphDestroy(w->graph); w->graph = nullptr; }
    }
    if (tcap > 0) BF_CUDA(cudaMemsetAsync(w->trace, 0xFF, sizeof(long long) * 4 * w->trace_cap, st));
    // inputs
    const void *dG, *dT, *dTgt, *dAv;
    if ((rc = stage_in(G, sizeof(double) * C * U, (void**)&w->stage_G, st, &dG))) return rc;
    if ((rc = stage_in(terminal, sizeof(double) * C, (void**)&w->stage_T, st, &dT))) return rc;
    if ((rc = stage_in(terminal ? nullptr : target, C, (void**)&w->stage_tgt, st, &dTgt))) return rc;
    if ((rc = stage_in(avoid, C, (void**)&w->stage_avoid, st, &dAv))) return rc;
    long long cap = C;
    if (opts && opts->max_iters > 0 && opts->max_iters < cap) cap = opts->max_iters;
    const int flags = opts ? opts->flags : 0;
    const bool count = (flags & BF_FLAG_COUNT_EXACT) != 0;
    const bool timed = (flags & BF_FLAG_TIME_KERNELS) != 0;
    const bool host_loop = (flags & BF_FLAG_HOST_LOOP) || count || timed;
    if (count && !w->stamp) BF_CUDA(cudaMalloc((void**)&w->stamp, sizeof(int) * C));
    // set-up: lines 1-10 of Algorithm 1
    k_init_counters<<<1, 1, 0, st>>>(w->ctr, cap);
    BF_CUDA(cudaMemsetAsync(w->fbits, 0, 4 * w->nwords, st));
    InstView v = make_view(a, w);
    if (v.ubits) BF_CUDA(cudaMemsetAsync(w->ubits, 0, 8 * w->nwords * U, st));
    if (w->fc_cap > 0) BF_CUDA(cudaMemsetAsync(w->fc_tag, 0, 8 * C, st));    // no cell cached before pass 0
    k_init_costs<<<blocks_for(C, 256), 256, 0, st>>>(C, U, (const double*)dG, (const unsigned char*)dAv,
                                                     w->Gint, w->ctr);
    if (cls) {
        const void* dGR;
        if ((rc = stage_in(cls_cost, sizeof(double) * C * U, (void**)&w->stage_GR, st, &dGR))) return rc;
        BF_CUDA(cudaMemcpyAsync(w->rmask, cls_mask, C, cudaMemcpyDefault, st));
        k_init_costs<<<blocks_for(C, 256), 256, 0, st>>>(C, U, (const double*)dGR, (const unsigned char*)dAv,
                                                         w->GRint, w->ctr);
    }
    k_init_values<<<blocks_for(C, 256), 256, 0, st>>>(C, (const double*)dT, (const unsigned char*)dTgt,
                                                      (const unsigned char*)dAv, w->Vkey, w->Vnew, w->mu,
                                                      w->chg, count ? w->stamp : nullptr, w->ctr);
    if (count) v.stamp = w->stamp;
    k_init_tables<<<blocks_for(C, 256), 256, 0, st>>>(v);
    if (v.M33P) k_init_table_pair<<<blocks_for(C, 256), 256, 0, st>>>(v);
    launch_setup_frontier(a, w, v, st);
    BF_CUDA(cudaGetLastError());
    double relax_ms = 0.0, prop_ms = 0.0;
    if (host_loop) {
        PassTimers tm{};
        if (timed)
            for (int i = 0; i < 4; ++i) BF_CUDA(cudaEventCreate(&tm.e[i]));
        Counters hc;
        long long launched = 0;
        for (;;) {
            BF_CUDA(cudaMemcpyAsync(&hc, w->ctr, sizeof hc, cudaMemcpyDeviceToHost, st));
            BF_CUDA(cudaStreamSynchronize(st));
            if (timed && launched > 0) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, tm.e[0], tm.e[1]);
                relax_ms += ms;
                cudaEventElapsedTime(&ms, tm.e[2], tm.e[3]);
                prop_ms += ms;
            }
            if (hc.done) break;
            launch_pass_any(a, w, v, st, 0, 0, count, timed ? &tm : nullptr);
            ++launched;
            BF_CUDA(cudaGetLastError());
        }
        if (timed)
            for (int i = 0; i < 4; ++i) cudaEventDestroy(tm.e[i]);
    } else {
        if ((rc = ws_graph(a, w))) return rc;
        BF_CUDA(cudaGraphLaunch(w->exec, st));
    }
    // outputs
    const bool vdev = bfh::is_device_ptr(V);
    double* dV = V;
    if (!vdev) {
        if (!w->stage_V) BF_CUDA(cudaMalloc((void**)&w->stage_V, 8 * C));
        dV = w->stage_V;
    }
    k_output<<<blocks_for(C, 256), 256, 0, st>>>(C, w->Vkey, dV);
    BF_CUDA(cudaGetLastError());
    if (!vdev) BF_CUDA(cudaMemcpyAsync(V, dV, 8 * C, cudaMemcpyDeviceToHost, st));
    BF_CUDA(cudaMemcpyAsync(mu, w->mu, C, cudaMemcpyDefault, st));
    Counters hc;
    BF_CUDA(cudaMemcpyAsync(&hc, w->ctr, sizeof hc, cudaMemcpyDeviceToHost, st));
    if (tcap > 0)
        BF_CUDA(cudaMemcpyAsync(opts->trace, w->trace, sizeof(long long) * 4 * tcap, cudaMemcpyDeviceToHost, st));
    BF_CUDA(cudaStreamSynchronize(st));
    if (hc.err) {
        bfh::set_error("bf_solve: NaN, -inf or |value| > 2^64 in G or the terminal cost");
        return BF_ERR_INVALID;
    }
    if (hc.fault) {
        bfh::set_error("bf_solve: the tile relax gave up waiting for its shared-memory copies");
        return BF_ERR_TIMEOUT;
    }
    *iters = hc.round;
    *status = hc.status;
    if (opts && opts->stats) {
        bf_solve_stats* o = opts->stats;
        // set-up: counters, costs, values, tables, first propagate, first
        // compaction, loop condition (graph); two or three kernels per pass;
        // output
        o->kernel_launches = (host_loop ? 7 : 8) + (v.M33P ? 1 : 0) +
                             ((w->fuse_mark ? 2 : 3) + (v.f1bits && !count ? 1 : 0)) * hc.round;
        o->relaxed_cells = hc.total_relaxed;
        // pairs taken up: counted by the masked relax, else every input of a relaxed cell
        o->executed_pairs = (v.fmask && !count) ? hc.total_pairs : hc.total_relaxed * U;
        o->exact_f1_cells = count ? hc.total_exact : -1;
        o->changed_cells = hc.total_changed;
        o->relax_launches = hc.round;
        o->relax_ms = timed ? relax_ms : 0.0;
        o->propagate_ms = timed ? prop_ms : 0.0;
    }
    return BF_OK;
}

// ---------------------------------------------------------------------------
// schedule tuning
// ---------------------------------------------------------------------------

// Time one configuration: one warm solve, then the mean of four.
static int tune_time(const bf_abstraction* a, const double* G, const uint8_t* target, const uint8_t* avoid,
                     const bf_solve_opts* o, double* V, uint8_t* mu, cudaStream_t st, double* ms) {
    int64_t iters;
    int32_t status;
    int rc = bf_solve(a, G, target, avoid, o, V, mu, &iters, &status, st);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    BF_CUDA(cudaEventCreate(&e0));
    BF_CUDA(cudaEventCreate(&e1));
    cudaEventRecord(e0, st);
    for (int r = 0; r < 4 && rc == BF_OK; ++r) rc = bf_solve(a, G, target, avoid, o, V, mu, &iters, &status, st);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = t / 4.0;
    return rc;
}

// The tile relax's geometry, tensor maps and F1 bitmap (once per workspace);
// BF_ERR_UNSUPPORTED when the abstraction does not fit the tile form.
static int ws_tile(const bf_abstraction* a, bf_solve_ws* w, cudaStream_t st) {
    if (w->tile) return BF_OK;
    if (w->tile_failed) return BF_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(w->mtx);
    int rc = ws_blocks(a, w, st);
    if (rc) return rc;
    long long* tables[4] = {w->Vkey, w->M2, w->M3, w->M33};
    if (!w->f1bits) {
        cudaError_t e = cudaMalloc((void**)&w->f1bits, 4 * w->nwords);
        if (e != cudaSuccess) return bfh::cuda_fail(e, "F1 bitmap");
    }
    rc = tile_setup(a, tables, &w->tile);
    if (rc) {
        w->tile_failed = true;
        w->tile = nullptr;
    }
    return rc;
}

struct Sched {
    int slice = kSliceTarget;
    bool fuse = true;
    int blocks = 0;
    bool use33 = false;
    bool plane = true;
    bool tmpl = true;
    bool pair = false;
    bool occ = false;
    int dense = 0;
    int masked = 0;
    int pz = 0;
    bool pfront = false;
};

static bool same_sched(const Sched& x, const Sched& y) {
    return x.slice == y.slice && x.fuse == y.fuse && x.blocks == y.blocks && x.use33 == y.use33 &&
           x.plane == y.plane && x.tmpl == y.tmpl && x.pair == y.pair && x.occ == y.occ && x.dense == y.dense &&
           x.masked == y.masked && x.pz == y.pz && x.pfront == y.pfront;
}

static bool base_plane_on(const Sched& s) { return s.plane; }

// Put schedule s in force; the plane-pair table is allocated on first use
// (without memory the schedule goes without it).
static void set_schedule(const bf_abstraction* a, bf_solve_ws* w, const Sched& s) {
    std::lock_guard<std::mutex> lock(w->mtx);
    int pz = (s.pz >= 2 && s.pz < w->D && s.pz < 4 && a->d_poffs[s.pz]) ? s.pz : 0;
    if (pz && !w->M33P && cudaMalloc((void**)&w->M33P, 8 * w->C) != cudaSuccess) {
        cudaGetLastError();
        w->M33P = nullptr;
        pz = 0;
    }
    w->pz = pz;
    w->masked = a->d_fmask != nullptr ? s.masked : 0;
    bool pf = s.pfront && a->d_uent != nullptr;
    if (pf && !w->ubits) {
        if (cudaMalloc((void**)&w->ubits, 8 * w->nwords * w->U) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(w->ubits);
            w->ubits = nullptr;
            pf = false;
        }
    }
    w->pfront = pf;
    w->slice_target = s.slice;
    w->fuse_mark = s.fuse;
    w->relax_blocks = s.blocks;
    w->use33 = s.use33 && w->M33 != nullptr;
    w->use_plane = s.plane;
    w->use_tmpl = s.tmpl;
    w->pair = s.pair;
    w->occ = s.occ;
    w->dense_pct = s.dense;
    w->tuned = true;
    if (w->exec) { cudaGraphExecDestroy(w->exec); w->exec = nullptr; }
    if (w->graph) { cudaGraphDestroy(w->graph); w->graph = nullptr; }
}

extern "C" int bf_tune(const bf_abstraction* a, const double* G, const uint8_t* target, const uint8_t* avoid,
                       const bf_solve_opts* opts, bf_tune_result* out, void* stream) {
    if (!a || !G || !out) {
        bfh::set_error("bf_tune: NULL argument");
        return BF_ERR_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    bf_solve_opts o;
    memset(&o, 0, sizeof o);
    if (opts) o = *opts;
    o.flags = 0;                  // timed as the graph-launched solve
    o.trace = nullptr;
    o.trace_cap = 0;
    o.stats = nullptr;
    const long long C = a->g.C;
    double* V = nullptr;
    uint8_t* mu = nullptr;
    BF_CUDA(cudaMalloc((void**)&V, 8 * C));
    cudaError_t e = cudaMalloc((void**)&mu, C);
    if (e != cudaSuccess) { cudaFree(V); return bfh::cuda_fail(e, "bf_tune buffers"); }
    // default schedule first (sets up the workspace)
    double best = 0.0;
    int rc = tune_time(a, G, target, avoid, &o, V, mu, st, &best);
    bf_solve_ws* w = a->ws;
    if (rc == BF_OK && !w) rc = BF_ERR_CUDA;
    if (rc) { cudaFree(V); cudaFree(mu); return rc; }
    const int full = w->relax_blocks_full;
    Sched b;
    b.slice = w->slice_target;
    b.fuse = w->fuse_mark;
    b.blocks = w->relax_blocks;
    b.use33 = w->use33;
    b.plane = w->use_plane;
    b.tmpl = w->use_tmpl;
    b.pair = w->pair;
    b.occ = w->occ;
    b.dense = w->dense_pct;
    b.masked = w->masked;
    b.pz = w->pz;
    b.pfront = w->pfront;
    out->default_ms = best;
    int tried = 1;
    const bool cls = opts && opts->succ_class;
    const bool has33 = w->M33 && !cls, hasp = a->d_poffs[0] && !cls, hast = a->d_tent != nullptr;
    const bool hasd = !cls && ws_tile(a, w, st) == BF_OK;
    // two whole schedules first (the pair-queue relax, with the per-input
    // frontier and marking in its own launch, or without it and marking in
    // relax): their settings help each other, which one dimension at a time
    // would not find
    if (hasp && has33 && a->d_fmask) {
        for (int k = 0; k < 2 && rc == BF_OK; ++k) {
            Sched c = b;
            c.use33 = true;
            c.plane = true;
            c.tmpl = hast;
            c.masked = 2;
            c.pair = true;
            c.pfront = k == 0 && a->d_uent != nullptr;
            c.fuse = k != 0;
            if (same_sched(c, b)) continue;
            set_schedule(a, w, c);
            double ms = 0.0;
            rc = tune_time(a, G, target, avoid, &o, V, mu, st, &ms);
            ++tried;
            if (rc == BF_OK && ms < best) {
                best = ms;
                b = c;
            }
        }
    }
    // coordinate descent: each dimension's values with the others at the best
    // so far, two rounds
    for (int round = 0; round < 2 && rc == BF_OK; ++round) {
        for (int dim = 0; dim < 12 && rc == BF_OK; ++dim) {
            const int nval = (dim == 0 || dim == 9) ? 4 : (dim == 7 ? 3 : (dim == 10 ? a->g.D - 1 : 2));
            if (dim == 7 && !hasd) continue;
            if (dim == 9 && !(hasp && a->d_fmask && base_plane_on(b))) continue;
            if (dim == 10 && !(hasp && has33 && a->g.D >= 3 && base_plane_on(b) && b.use33)) continue;
            if (dim == 11 && !(a->d_uent && b.tmpl)) continue;
            if (dim == 8 && !(hasp && base_plane_on(b))) continue;
            if ((dim == 3 && !has33) || (dim == 4 && !hasp) || (dim == 5 && !hast)) continue;
            if (dim == 6 && !(hasp && base_plane_on(b))) continue;
            const Sched base = b;                              // timed already
            for (int k = 0; k < nval && rc == BF_OK; ++k) {
                Sched c = base;
                const int slices[4] = {0, 1, 2, kSliceTargetMax};
                switch (dim) {
                    case 0: c.slice = slices[k]; break;
                    case 1: c.fuse = k != 0; break;
                    case 2: c.blocks = k == 0 ? full : (full + 1) / 2; break;
                    case 3: c.use33 = k != 0; break;
                    case 4: c.plane = k != 0; break;
                    case 5: c.tmpl = k != 0; break;
                    case 6: c.pair = k != 0; break;
                    case 7: c.dense = k == 0 ? 0 : (k == 1 ? 15 : 35); break;
                    case 8: c.occ = k != 0; break;
                    case 9:      // cell masks, with the per-input frontier for the queue form
                        c.masked = k < 3 ? k : 2;
                        if (k == 3) c.pfront = a->d_uent != nullptr && b.tmpl;
                        break;
                    case 10: c.pz = k == 0 ? 0 : k + 1; break;
                    default: c.pfront = k != 0; break;
                }
                if (same_sched(c, base)) continue;
                set_schedule(a, w, c);
                double ms = 0.0;
                rc = tune_time(a, G, target, avoid, &o, V, mu, st, &ms);
                ++tried;
                if (rc == BF_OK && ms < best) {
                    best = ms;
                    b = c;
                }
            }
        }
    }
    set_schedule(a, w, b);
    cudaFree(V);
    cudaFree(mu);
    if (rc) return rc;
    out->slice_target = b.slice;
    out->fuse_mark = b.fuse ? 1 : 0;
    out->window33 = b.use33 && w->M33 ? 1 : 0;
    out->relax_blocks = b.blocks;
    out->plane_lists = (b.plane && hasp) ? 1 : 0;
    out->templates = (b.tmpl && hast) ? 1 : 0;
    out->pair_inputs = (b.pair && b.plane && hasp) ? 1 : 0;
    out->dense_pct = hasd ? b.dense : 0;
    out->occupancy = (b.occ && b.plane && hasp) ? 1 : 0;
    out->cell_masks = (b.plane && hasp) ? w->masked : 0;
    out->pair_dim = (w->pz && b.use33 && b.plane && hasp) ? w->pz : 0;
    out->input_frontier = (w->pfront && b.tmpl && hast) ? 1 : 0;
    out->candidates = tried;
    out->best_ms = best;
    return BF_OK;
}

extern "C" int bf_set_schedule(const bf_abstraction* a, const bf_tune_result* sched, void* stream) {
    if (!a || !sched) {
        bfh::set_error("bf_set_schedule: NULL argument");
        return BF_ERR_INVALID;
    }
    const int st_ = sched->slice_target;
    if (st_ < 0 || st_ > kSliceTargetMax) {
        bfh::set_error("bf_set_schedule: slice_target %d outside 0..%d", st_, kSliceTargetMax);
        return BF_ERR_INVALID;
    }
    bf_solve_ws* w = nullptr;
    int rc = ws_get(a, &w);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lock(w->mtx);
        if ((rc = ws_blocks(a, w, (cudaStream_t)stream))) return rc;
    }
    int blocks = sched->relax_blocks;
    if (blocks <= 0 || blocks > w->relax_blocks_full) blocks = w->relax_blocks_full;
    Sched c;
    c.slice = st_;
    c.fuse = sched->fuse_mark != 0;
    c.blocks = blocks;
    c.use33 = sched->window33 != 0;
    c.plane = sched->plane_lists != 0;
    c.tmpl = sched->templates != 0;
    c.pair = sched->pair_inputs != 0;
    c.dense = sched->dense_pct;
    c.occ = sched->occupancy != 0;
    c.masked = sched->cell_masks;
    if (c.masked < 0 || c.masked > 2) {
        bfh::set_error("bf_set_schedule: cell_masks %d outside 0..2", c.masked);
        return BF_ERR_INVALID;
    }
    c.pz = sched->pair_dim;
    c.pfront = sched->input_frontier != 0;
    if (c.pz != 0 && (c.pz < 2 || c.pz >= a->g.D)) {
        bfh::set_error("bf_set_schedule: pair_dim %d outside 0, 2 .. D - 1", c.pz);
        return BF_ERR_INVALID;
    }
    if (c.dense < 0 || c.dense > 100) {
        bfh::set_error("bf_set_schedule: dense_pct %d outside 0..100", c.dense);
        return BF_ERR_INVALID;
    }
    if (c.dense > 0 && ws_tile(a, w, (cudaStream_t)stream) != BF_OK) c.dense = 0;
    set_schedule(a, w, c);
    return BF_OK;
}
