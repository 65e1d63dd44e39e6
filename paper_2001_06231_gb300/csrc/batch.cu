// batch.cu -- bf_solve_batch and the batched pass engine (batch_engine.cuh).
//
// Work distribution: one-block planning kernels turn the per-instance work
// counts (32-cell chunks of the current frontier, changed cells, 256-word
// chunks of the frontier bitmap) into exclusive prefixes over the instance
// list, ordered by group.  A relax (or propagate) launch for group g then has
// scan[gend] - scan[gbeg] work items; warp w takes item k, finds its instance
// by binary search over the prefix and runs the same per-warp routine as the
// single solve.  The planning kernel after the compaction also closes the
// pass of every unfinished instance (finish_pass) and counts the instances
// still running.
#include <math_constants.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "batch_engine.cuh"

using namespace bfk;

namespace bfb {

// ---------------------------------------------------------------------------
// set-up kernels (one instance at a time)
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool b_clean(double v, double& out) {
    if (v != v) return false;
    if (v == -CUDART_INF) return false;
    if (v != CUDART_INF && fabs(v) > 18446744073709551616.0) return false;
    out = (v == 0.0) ? 0.0 : v;
    return true;
}

__global__ void k_b_counters(Counters* ctr, long long cap) {
    memset(ctr, 0, sizeof(Counters));
    ctr->cap = cap;
}

__global__ void k_b_costs(long long C, int U, const double* __restrict__ G,
                          const unsigned char* __restrict__ avoid, double* Gint, Counters* ctr) {
    bool bad = false;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < C;
         c += (long long)gridDim.x * blockDim.x) {
        const bool av = avoid && avoid[c];
        for (int u = 0; u < U; ++u) {
            double v;
            if (!b_clean(__ldg(G + c * U + u), v)) bad = true;
            Gint[(long long)u * C + c] = av ? CUDART_INF : v;
        }
    }
    if (bad) atomicOr(&ctr->err, 1);
}

__global__ void k_b_values(long long C, const double* __restrict__ terminal,
                           const unsigned char* __restrict__ target, const unsigned char* __restrict__ avoid,
                           long long* Vkey, long long* Vnew, unsigned char* mu, int* chg, Counters* ctr) {
    bool bad = false;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long start = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long rounds = (C + stride - 1) / stride;
    for (long long it = 0; it < rounds; ++it) {
        const long long c = start + it * stride;
        bool finite = false;
        if (c < C) {
            double t;
            if (terminal) {
                if (!b_clean(terminal[c], t)) { bad = true; t = CUDART_INF; }
            } else {
                t = (target && target[c]) ? 0.0 : CUDART_INF;
            }
            if (avoid && avoid[c]) t = CUDART_INF;
            const long long k = key_of(t);
            Vkey[c] = k;
            Vnew[c] = k;
            mu[c] = kHandover;
            finite = k != kKeyInf;
        }
        const int slot = warp_append(finite, &ctr->nchg);
        if (finite) chg[slot] = (int)c;
    }
    if (bad) atomicOr(&ctr->err, 1);
}

__global__ void k_b_tables(InstView v) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < v.g.C;
         c += (long long)gridDim.x * blockDim.x) {
        table_entry(v, c);
        if (v.M33) table33_entry(v, c);
    }
}

// Set-up tail of one instance: pred of the finite cells -> F2 bits.
template <int D>
__global__ void __launch_bounds__(256, 4) k_b_propagate_init(InstView v) {
    const int nchg = v.ctr->nchg;
    const int wpb = blockDim.x >> 5;
    const int nwarps = gridDim.x * wpb;
    for (int i = blockIdx.x * wpb + (threadIdx.x >> 5); i < nchg; i += nwarps)
        propagate_entry<D>(v, i, nchg, false);
}

// Set-up tail of one instance: compact F1 and decide whether it loops.  The
// instance then looks like one whose previous pass just closed, so it can
// join a running batch.
__global__ void __launch_bounds__(256) k_b_compact_init(InstView v, long long nwords) {
    for (long long wb = (long long)blockIdx.x * blockDim.x; wb < nwords; wb += (long long)gridDim.x * blockDim.x)
        compact_words(v, (int)wb, (int)nwords);
    if (last_block_done(&v.ctr->blocks_done)) start_loop(v);
}

__global__ void k_b_output(long long C, const long long* __restrict__ Vkey, double* V) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < C;
         c += (long long)gridDim.x * blockDim.x)
        V[c] = val_of(Vkey[c]);
}

// ---------------------------------------------------------------------------
// batched pass kernels
// ---------------------------------------------------------------------------

// Largest i in [beg, end) with scan[i] <= pos.
__device__ __forceinline__ int find_instance(const int* __restrict__ scan, int beg, int end, int pos) {
    int lo = beg, hi = end - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (scan[mid] <= pos) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Exclusive prefix over the n per-instance counts already stored in out[0..n)
// (one block; each thread owns a contiguous chunk).  out[n] = total.
__device__ void block_exclusive_scan(int* out, int n, int* sums) {
    const int t = threadIdx.x, bd = blockDim.x;
    const int chunk = (n + bd - 1) / bd;
    const int i0 = min(n, t * chunk), i1 = min(n, i0 + chunk);
    int local = 0;
    for (int i = i0; i < i1; ++i) local += out[i];
    sums[t] = local;
    __syncthreads();
    for (int off = 1; off < bd; off <<= 1) {
        const int x = t >= off ? sums[t - off] : 0;
        __syncthreads();
        sums[t] += x;
        __syncthreads();
    }
    int run = t > 0 ? sums[t - 1] : 0;
    for (int i = i0; i < i1; ++i) {
        const int c = out[i];
        out[i] = run;
        run += c;
    }
    __syncthreads();
    if (t == 0) out[n] = sums[bd - 1];
    __syncthreads();
}

// Planning (one block of 1024 threads).
//   mode 1 (after relax):      prefixes of the changed cells and of the
//                              compaction chunks of every unfinished instance.
//   mode 2 (after compaction): close the pass of every unfinished instance;
//                              prefix of the next pass's relax chunks.
//   mode 3 (instance set changed): prefix of the next pass's relax chunks.
// In modes 2 and 3 also counts the unfinished instances (and sets the WHILE
// condition of the graph).
__global__ void __launch_bounds__(1024) k_b_plan(BatchDev b, int mode, cudaGraphConditionalHandle h,
                                                 int use_graph) {
    __shared__ int sums[1024];
    __shared__ int active;
    const int t = threadIdx.x, bd = blockDim.x;
    if (t == 0) active = 0;
    __syncthreads();
    const int n = b.n;
    int alive = 0;
    for (int i = t; i < n; i += bd) {
        const InstView& v = b.views[i];
        Counters* k = v.ctr;
        if (mode == 1) {
            const bool run = !k->done;
            b.scan_chg[i] = run ? k->nchg : 0;
            b.scan_cmp[i] = run ? (int)((((v.g.C + 31) >> 5) + 255) >> 8) : 0;
        } else {
            int cnt = 0;
            if (!k->done) {
                if (mode == 2) finish_pass(v);
                if (!k->done) cnt = (k->ncur + 31) >> 5;
            }
            if (!k->done) ++alive;
            b.scan[i] = cnt;
        }
    }
    if (alive) atomicAdd(&active, alive);
    __syncthreads();
    if (mode == 1) {
        block_exclusive_scan(b.scan_chg, n, sums);
        block_exclusive_scan(b.scan_cmp, n, sums);
    } else {
        block_exclusive_scan(b.scan, n, sums);
        if (t == 0) {
            *b.active = active;
            if (use_graph) {
                int cont = active > 0 ? 1 : 0;
                if (use_graph == 2) cont = cont && (--*b.step_left > 0);   // bounded step
                cudaGraphSetConditional(h, cont);
            }
        }
    }
}

__global__ void k_b_cond(const int* active, cudaGraphConditionalHandle h) {
    cudaGraphSetConditional(h, *active > 0 ? 1 : 0);
}

// First node of a bounded step: `passes` passes at most, none when all are done.
__global__ void k_b_step_init(int* step_left, const int* active, int passes, cudaGraphConditionalHandle h) {
    *step_left = passes;
    cudaGraphSetConditional(h, (*active > 0 && passes > 0) ? 1 : 0);
}

template <int D, int FMT, bool MARK>
__global__ void __launch_bounds__(256, (FMT == kBoxRecompute || FMT == kBoxHybrid) ? 2 : 4) k_b_relax(BatchDev b, int g) {
    const int beg = b.gbeg[g], end = b.gbeg[g + 1];
    if (beg >= end) return;
    const int base = b.scan[beg], total = b.scan[end] - base;
    const int wpb = blockDim.x >> 5;
    const int nwarps = gridDim.x * wpb;
    for (int item = blockIdx.x * wpb + (threadIdx.x >> 5); item < total; item += nwarps) {
        const int pos = base + item;
        const int i = find_instance(b.scan, beg, end, pos);
        const InstView& v = b.views[i];
        const int ch = pos - b.scan[i];
        int exact = 0;
        const int r = relax_chunk<D, FMT, false, MARK>(v, ch << 5, v.ctr->ncur - (ch << 5), v.ctr->round, &exact);
        if ((threadIdx.x & 31) == 0 && r)
            atomicAdd((unsigned long long*)&v.ctr->relaxed, (unsigned long long)r);
    }
}

// The group's relax on plane lookup lists (every instance of the group has
// them): per-warp staging of the lists in dynamic shared memory.
template <int D, bool MARK, bool PAIR>
__global__ void __launch_bounds__(256, PAIR ? 3 : 4) k_b_relax_pl(BatchDev b, int g) {
    const int beg = b.gbeg[g], end = b.gbeg[g + 1];
    if (beg >= end) return;
    extern __shared__ __align__(16) unsigned char b_plane_smem[];
    PlaneStage* st = reinterpret_cast<PlaneStage*>(b_plane_smem) + (threadIdx.x >> 5);
    const int base = b.scan[beg], total = b.scan[end] - base;
    const int wpb = blockDim.x >> 5;
    const int nwarps = gridDim.x * wpb;
    for (int item = blockIdx.x * wpb + (threadIdx.x >> 5); item < total; item += nwarps) {
        const int pos = base + item;
        const int i = find_instance(b.scan, beg, end, pos);
        const InstView& v = b.views[i];
        const int ch = pos - b.scan[i];
        int exact = 0;
        const int r = relax_chunk<D, kBoxCompact, false, MARK, false, PAIR ? 2 : 1>(
            v, ch << 5, v.ctr->ncur - (ch << 5), v.ctr->round, &exact, st);
        if ((threadIdx.x & 31) == 0 && r)
            atomicAdd((unsigned long long*)&v.ctr->relaxed, (unsigned long long)r);
    }
}

// The group's relax by cell masks with the pairs queued over the lanes
// (relax_plane_q; every instance of the group has the masks and lists).  The
// stage is emptied before each chunk: consecutive chunks of a warp may belong
// to different instances.
template <int D, bool MARK, int UM, bool R2>
__global__ void __launch_bounds__(UM == 16 ? 256 : 128, 3) k_b_relax_pq(BatchDev b, int g) {
    const int beg = b.gbeg[g], end = b.gbeg[g + 1];
    if (beg >= end) return;
    extern __shared__ __align__(16) unsigned char b_pair_smem[];
    PairStage<UM>* st = reinterpret_cast<PairStage<UM>*>(b_pair_smem) + (threadIdx.x >> 5);
    const int base = b.scan[beg], total = b.scan[end] - base;
    const int wpb = blockDim.x >> 5;
    const int nwarps = gridDim.x * wpb;
    long long taken = 0;
    for (int item = blockIdx.x * wpb + (threadIdx.x >> 5); item < total; item += nwarps) {
        const int pos = base + item;
        const int i = find_instance(b.scan, beg, end, pos);
        const InstView& v = b.views[i];
        const int ch = pos - b.scan[i];
        int exact = 0;
        __syncwarp();
        if ((threadIdx.x & 31) == 0) st->plane = -1;
        __syncwarp();
        const int r = relax_chunk<D, kBoxCompact, false, MARK, false, R2 ? 6 : 5, UM>(
            v, ch << 5, v.ctr->ncur - (ch << 5), v.ctr->round, &exact, st, &taken);
        if ((threadIdx.x & 31) == 0 && r)
            atomicAdd((unsigned long long*)&v.ctr->relaxed, (unsigned long long)r);
    }
}

template <int D>
__global__ void __launch_bounds__(256, 4) k_b_propagate(BatchDev b, int g) {
    const int beg = b.gbeg[g], end = b.gbeg[g + 1];
    if (beg >= end) return;
    const int base = b.scan_chg[beg], total = b.scan_chg[end] - base;
    const int wpb = blockDim.x >> 5;
    const int nwarps = gridDim.x * wpb;
    for (int item = blockIdx.x * wpb + (threadIdx.x >> 5); item < total; item += nwarps) {
        const int pos = base + item;
        const int i = find_instance(b.scan_chg, beg, end, pos);
        const InstView& v = b.views[i];
        propagate_entry<D>(v, pos - b.scan_chg[i], v.ctr->nchg, false);      // compact commits
    }
}

// Compaction of every unfinished instance (block per 256-word chunk) and the
// refresh of the window tables around every changed cell.
__global__ void __launch_bounds__(256) k_b_compact(BatchDev b) {
    const int n = b.n;
    const int total = b.scan_cmp[n];
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int i = find_instance(b.scan_cmp, 0, n, item);
        const InstView& v = b.views[i];
        const int nwords = (int)((v.g.C + 31) >> 5);
        compact_words(v, (item - b.scan_cmp[i]) << 8, nwords);
    }
    const int tchg = b.scan_chg[n];
    for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < tchg; item += gridDim.x * blockDim.x) {
        const int i = find_instance(b.scan_chg, 0, n, item);
        const InstView& v = b.views[i];
        const int y = v.chg[item - b.scan_chg[i]];
        v.Vkey[y] = v.Vnew[y];                                  // commit W
        refresh_tables(v, y);
    }
}

// ---------------------------------------------------------------------------
// Engine
// ---------------------------------------------------------------------------
static int n_sms() {
    int dev = 0, n = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

static int blocks_for(long long work) {
    long long need = (work + 255) / 256;
    const long long cap = (long long)n_sms() * 8;
    return (int)std::max(1LL, std::min(need, cap));
}

static size_t r256(size_t b) { return (b + 255) & ~size_t(255); }

Engine::Engine(cudaStream_t st) : st_(st) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (cudaMemPoolCreate(&pool_, &props) == cudaSuccess) {
        unsigned long long keep = ~0ull;
        cudaMemPoolSetAttribute(pool_, cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
        pool_ = nullptr;                    // fall back to the device's default pool
        cudaGetLastError();
    }
}

int Engine::alloc(void** p, size_t bytes) {
    if (pool_) BF_CUDA(cudaMallocFromPoolAsync(p, bytes, pool_, st_));
    else BF_CUDA(cudaMallocAsync(p, bytes, st_));
    return BF_OK;
}

Engine::~Engine() {
    drop_step_graphs();
    for (InstState* s : insts_) {
        cudaFreeAsync(s->mem, st_);
        delete s;
    }
    insts_.clear();
    if (dev_mem_) cudaFreeAsync(dev_mem_, st_);
    cudaStreamSynchronize(st_);
    if (pool_) cudaMemPoolDestroy(pool_);
}

size_t Engine::state_bytes(const bf_abstraction* a, bool stage_G, bool stage_T, bool stage_V) const {
    return state_bytes_for(a->g.C, a->g.U, stage_G, stage_T, stage_V);
}

size_t Engine::state_bytes_for(long long Cc, int Uc, bool stage_G, bool stage_T, bool stage_V) {
    const size_t C = (size_t)Cc, U = (size_t)Uc, S = (C + 31) / 32;
    size_t o = r256(sizeof(Counters)) + 5 * r256(8 * C) + r256(C) + r256(4 * S) + 2 * r256(4 * C) +
               r256(8 * C * U);
    if (stage_G) o += r256(8 * C * U);
    if (stage_T) o += r256(8 * C) + r256(C) + r256(C);   // terminal or target, plus avoid
    if (stage_V) o += r256(8 * C);
    return o;
}

static int group_of(const bf_abstraction* a) {
    return (a->g.D - 1) * 4 + a->box_fmt;
}

int Engine::add(const bf_abstraction* a, const double* G, const unsigned char* target,
                const unsigned char* avoid, const double* terminal, long long max_iters, double* V,
                unsigned char* mu, InstState** out) {
    if (!a || !G || !V || !mu || (!target && !terminal)) {
        bfh::set_error("batch: instance needs an abstraction, G, V, mu and a target or terminal cost");
        return BF_ERR_INVALID;
    }
    const long long C = a->g.C;
    const int U = a->g.U;
    const long long S = (C + 31) / 32;
    const bool sG = !bfh::is_device_ptr(G);
    const bool sT = terminal && !bfh::is_device_ptr(terminal);
    const bool sTg = !terminal && target && !bfh::is_device_ptr(target);
    const bool sAv = avoid && !bfh::is_device_ptr(avoid);
    const bool vdev = bfh::is_device_ptr(V);
    const bool mdev = bfh::is_device_ptr(mu);
    size_t o = 0;
    const size_t o_ctr = o;  o += r256(sizeof(Counters));
    const size_t o_vk = o;   o += r256(8 * (size_t)C);
    const size_t o_vn = o;   o += r256(8 * (size_t)C);
    const size_t o_m2 = o;   o += r256(8 * (size_t)C);
    const size_t o_m3 = o;   o += r256(8 * (size_t)C);
    const size_t o_m33 = o;  o += r256(8 * (size_t)C);
    const size_t o_mu = o;   o += r256((size_t)C);
    const size_t o_fb = o;   o += r256(4 * (size_t)S);
    const size_t o_cl = o;   o += r256(4 * (size_t)C);
    const size_t o_chg = o;  o += r256(4 * (size_t)C);
    const size_t o_gi = o;   o += r256(8 * (size_t)C * U);
    const size_t o_sg = o;   o += sG ? r256(8 * (size_t)C * U) : 0;
    const size_t o_st = o;   o += sT ? r256(8 * (size_t)C) : 0;
    const size_t o_stg = o;  o += sTg ? r256((size_t)C) : 0;
    const size_t o_sav = o;  o += sAv ? r256((size_t)C) : 0;
    const size_t o_sv = o;   o += vdev ? 0 : r256(8 * (size_t)C);
    void* mem = nullptr;
    if (int rc = alloc(&mem, o)) return rc;
    unsigned char* m = static_cast<unsigned char*>(mem);
    InstState* s = new InstState;
    s->a = a;
    s->mem = mem;
    s->group = group_of(a);
    s->cap = (max_iters > 0 && max_iters < C) ? max_iters : C;
    InstView& v = s->view;
    memset(&v, 0, sizeof v);
    view_from_abs(v, a);
    v.ctr = reinterpret_cast<Counters*>(m + o_ctr);
    v.Vkey = reinterpret_cast<long long*>(m + o_vk);
    v.Vnew = reinterpret_cast<long long*>(m + o_vn);
    v.M2 = reinterpret_cast<long long*>(m + o_m2);
    v.M3 = reinterpret_cast<long long*>(m + o_m3);
    // the batched schedule of the abstraction (bf_tune_batch) or the default
    const int bs = a->bsched >= 0 ? a->bsched : kBsDefault;
    if ((bs & kBsWindow33) && a->g.D >= 2) v.M33 = reinterpret_cast<long long*>(m + o_m33);
    if ((bs & kBsPlane) && a->d_poffs[0]) v.poffs = a->d_poffs[v.M33 ? 1 : 0];
    if ((bs & kBsQueue) && a->d_fmask) v.fmask = a->d_fmask;
    if ((bs & kBsTemplates) && a->d_tent) {
        v.tptr = a->d_tptr;
        v.tent = a->d_tent;
    }
    v.mu = m + o_mu;
    v.fbits = reinterpret_cast<unsigned*>(m + o_fb);
    v.cells = reinterpret_cast<int*>(m + o_cl);
    v.chg = reinterpret_cast<int*>(m + o_chg);
    v.Gint = reinterpret_cast<const double*>(m + o_gi);
    // inputs
    const double* dG = G;
    if (sG) {
        BF_CUDA(cudaMemcpyAsync(m + o_sg, G, 8 * (size_t)C * U, cudaMemcpyHostToDevice, st_));
        dG = reinterpret_cast<const double*>(m + o_sg);
    }
    const double* dT = terminal;
    if (sT) {
        BF_CUDA(cudaMemcpyAsync(m + o_st, terminal, 8 * (size_t)C, cudaMemcpyHostToDevice, st_));
        dT = reinterpret_cast<const double*>(m + o_st);
    }
    const unsigned char* dTg = terminal ? nullptr : target;
    if (sTg) {
        BF_CUDA(cudaMemcpyAsync(m + o_stg, target, (size_t)C, cudaMemcpyHostToDevice, st_));
        dTg = m + o_stg;
    }
    const unsigned char* dAv = avoid;
    if (sAv) {
        BF_CUDA(cudaMemcpyAsync(m + o_sav, avoid, (size_t)C, cudaMemcpyHostToDevice, st_));
        dAv = m + o_sav;
    }
    s->Vdev = vdev ? V : reinterpret_cast<double*>(m + o_sv);
    s->V_host = vdev ? nullptr : V;
    s->mu_host = mdev ? nullptr : mu;
    s->mu_dev_out = mdev ? mu : nullptr;
    // lines 1-10 of Algorithm 1
    k_b_counters<<<1, 1, 0, st_>>>(v.ctr, s->cap);
    BF_CUDA(cudaMemsetAsync(v.fbits, 0, 4 * (size_t)S, st_));
    const int nb = blocks_for(C);
    k_b_costs<<<nb, 256, 0, st_>>>(C, U, dG, dAv, const_cast<double*>(v.Gint), v.ctr);
    k_b_values<<<nb, 256, 0, st_>>>(C, dT, dTg, dAv, v.Vkey, v.Vnew, v.mu, v.chg, v.ctr);
    k_b_tables<<<nb, 256, 0, st_>>>(v);
    const int pb = n_sms() * 4;
    switch (a->g.D) {
        case 1: k_b_propagate_init<1><<<pb, 256, 0, st_>>>(v); break;
        case 2: k_b_propagate_init<2><<<pb, 256, 0, st_>>>(v); break;
        case 3: k_b_propagate_init<3><<<pb, 256, 0, st_>>>(v); break;
        default: k_b_propagate_init<4><<<pb, 256, 0, st_>>>(v); break;
    }
    k_b_compact_init<<<blocks_for(S), 256, 0, st_>>>(v, S);
    BF_CUDA(cudaGetLastError());
    insts_.push_back(s);
    if (out) *out = s;
    return BF_OK;
}

void Engine::remove(InstState* s) {
    auto it = std::find(insts_.begin(), insts_.end(), s);
    if (it != insts_.end()) insts_.erase(it);
    cudaFreeAsync(s->mem, st_);
    delete s;
}

int Engine::rebuild() {
    std::stable_sort(insts_.begin(), insts_.end(),
                     [](const InstState* x, const InstState* y) { return x->group < y->group; });
    const int n = (int)insts_.size();
    memset(&dev_, 0, sizeof dev_);
    dev_.n = n;
    // groups (same dimension and box format)
    int ng = 0;
    for (int i = 0; i < n; ++i) {
        const int g = insts_[i]->group;
        const bf_abstraction* a = insts_[i]->a;
        const int bs = a->bsched >= 0 ? a->bsched : kBsDefault;
        if (ng == 0 || (group_D_[ng - 1] - 1) * 4 + group_fmt_[ng - 1] != g) {
            group_D_[ng] = g / 4 + 1;
            group_fmt_[ng] = g % 4;
            group_mark_[ng] = true;
            // the first instance's schedule decides the group's kernels
            group_fixed_mark_[ng] = !(bs & kBsMarkAuto);
            if (group_fixed_mark_[ng]) group_mark_[ng] = (bs & kBsMark) != 0;
            group_plane_[ng] = (bs & kBsPlane) != 0 && group_fmt_[ng] == kBoxCompact && group_D_[ng] >= 2;
            group_pair_[ng] = (bs & kBsPair) != 0;
            group_queue_[ng] = group_plane_[ng] && (bs & kBsQueue) != 0;
            group_wide_[ng] = false;
            dev_.gbeg[ng] = i;
            ++ng;
        }
        // relax marks the next frontier itself when every predecessor box (or
        // template) of the group is small (as in the single solve)
        const double rows = insts_[i]->view.tent ? a->tmpl_rows : a->pred_rows;
        if (!group_fixed_mark_[ng - 1] && rows > kFuseMarkRowsBatch) group_mark_[ng - 1] = false;
        if (!a->d_poffs[0] || a->g.U > kPlaneUMax) group_plane_[ng - 1] = false;
        if (!group_plane_[ng - 1] || !insts_[i]->view.fmask) group_queue_[ng - 1] = false;
        if (a->g.U > 16) group_wide_[ng - 1] = true;
    }
    dev_.ngroups = ng;
    dev_.gbeg[ng] = n;
    drop_step_graphs();
    const size_t need = r256(sizeof(InstView) * std::max(n, 1)) + 3 * r256(4 * (size_t)(n + 1)) + 2 * r256(4);
    if (need > dev_mem_bytes_) {
        if (dev_mem_) BF_CUDA(cudaFreeAsync(dev_mem_, st_));
        dev_mem_ = nullptr;
        if (int rc = alloc(&dev_mem_, need)) return rc;
        dev_mem_bytes_ = need;
    }
    unsigned char* m = static_cast<unsigned char*>(dev_mem_);
    dev_.views = reinterpret_cast<InstView*>(m);
    m += r256(sizeof(InstView) * std::max(n, 1));
    dev_.scan = reinterpret_cast<int*>(m);
    m += r256(4 * (size_t)(n + 1));
    dev_.scan_chg = reinterpret_cast<int*>(m);
    m += r256(4 * (size_t)(n + 1));
    dev_.scan_cmp = reinterpret_cast<int*>(m);
    m += r256(4 * (size_t)(n + 1));
    dev_.active = reinterpret_cast<int*>(m);
    m += r256(4);
    dev_.step_left = reinterpret_cast<int*>(m);
    host_views_.resize(n);
    for (int g = 0; g < ng; ++g)
        for (int i = dev_.gbeg[g]; i < dev_.gbeg[g + 1]; ++i) {
            host_views_[i] = insts_[i]->view;
            // the plane kernel reads every instance's lists; the other kernels none
            InstView& hv = host_views_[i];
            hv.poffs = group_plane_[g] ? insts_[i]->a->d_poffs[hv.M33 ? 1 : 0] : nullptr;
        }
    if (n)
        BF_CUDA(cudaMemcpyAsync(dev_.views, host_views_.data(), sizeof(InstView) * n, cudaMemcpyHostToDevice,
                                st_));
    // work offsets of the next pass for the new instance set
    if (n) k_b_plan<<<1, 1024, 0, st_>>>(dev_, 3, 0, 0);
    BF_CUDA(cudaGetLastError());
    if (!relax_blocks_) {
        relax_blocks_ = n_sms() * 4;
        prop_blocks_ = n_sms() * 4;
        compact_blocks_ = n_sms() * 8;
    }
    return BF_OK;
}

template <int D, bool MARK>
static void launch_relax_pl(const BatchDev& b, int g, bool pair, cudaStream_t st) {
    const size_t sm = 8 * sizeof(PlaneStage);
    const int blocks = n_sms() * (pair ? 3 : 4);
    if (pair) k_b_relax_pl<D, MARK, true><<<blocks, 256, sm, st>>>(b, g);
    else k_b_relax_pl<D, MARK, false><<<blocks, 256, sm, st>>>(b, g);
}

template <int D, bool MARK, int UM, bool R2>
static void launch_relax_pq_t(const BatchDev& b, int g, cudaStream_t st) {
    const size_t sm = (UM == 16 ? 8 : 4) * sizeof(PairStage<UM>);
    static bool once = false;
    if (!once) {
        cudaFuncSetAttribute((const void*)k_b_relax_pq<D, MARK, UM, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sm);
        once = true;
    }
    k_b_relax_pq<D, MARK, UM, R2><<<n_sms() * 3, UM == 16 ? 256 : 128, sm, st>>>(b, g);
}

template <int D, bool MARK>
static void launch_relax_pq(const BatchDev& b, int g, bool wide, bool pair, cudaStream_t st) {
    if (wide) {
        if (pair) launch_relax_pq_t<D, MARK, 32, true>(b, g, st);
        else launch_relax_pq_t<D, MARK, 32, false>(b, g, st);
    } else {
        if (pair) launch_relax_pq_t<D, MARK, 16, true>(b, g, st);
        else launch_relax_pq_t<D, MARK, 16, false>(b, g, st);
    }
}

template <int D, bool MARK>
static void launch_relax_m(const BatchDev& b, int g, int fmt, int blocks, cudaStream_t st) {
    switch (fmt) {
        case kBoxCompact: k_b_relax<D, kBoxCompact, MARK><<<blocks, 256, 0, st>>>(b, g); break;
        case kBoxRecompute: k_b_relax<D, kBoxRecompute, MARK><<<blocks / 2, 256, 0, st>>>(b, g); break;
        case kBoxHybrid: k_b_relax<D, kBoxHybrid, MARK><<<blocks / 2, 256, 0, st>>>(b, g); break;
        default: k_b_relax<D, kBoxWide, MARK><<<blocks, 256, 0, st>>>(b, g); break;
    }
}

template <int D>
static void launch_relax(const BatchDev& b, int g, int fmt, bool mark, bool plane, bool pair, bool queue, bool wide,
                         int blocks, cudaStream_t st) {
    if constexpr (D >= 2) {
        if (queue) {
            if (mark) launch_relax_pq<D, true>(b, g, wide, pair, st);
            else launch_relax_pq<D, false>(b, g, wide, pair, st);
            return;
        }
        if (plane) {
            if (mark) launch_relax_pl<D, true>(b, g, pair, st);
            else launch_relax_pl<D, false>(b, g, pair, st);
            return;
        }
    }
    if (mark) launch_relax_m<D, true>(b, g, fmt, blocks, st);
    else launch_relax_m<D, false>(b, g, fmt, blocks, st);
}

template <int D>
static void launch_prop(const BatchDev& b, int g, int blocks, cudaStream_t st) {
    k_b_propagate<D><<<blocks, 256, 0, st>>>(b, g);
}

void Engine::launch_pass(cudaGraphConditionalHandle h, int use_graph) {
    for (int g = 0; g < dev_.ngroups; ++g) {
        const bool mark = group_mark_[g], pl = group_plane_[g], pr = group_pair_[g];
        const bool q = group_queue_[g], wd = group_wide_[g];
        switch (group_D_[g]) {
            case 1: launch_relax<1>(dev_, g, group_fmt_[g], mark, false, false, false, false, relax_blocks_, st_); break;
            case 2: launch_relax<2>(dev_, g, group_fmt_[g], mark, pl, pr, q, wd, relax_blocks_, st_); break;
            case 3: launch_relax<3>(dev_, g, group_fmt_[g], mark, pl, pr, q, wd, relax_blocks_, st_); break;
            default: launch_relax<4>(dev_, g, group_fmt_[g], mark, pl, pr, q, wd, relax_blocks_, st_); break;
        }
    }
    k_b_plan<<<1, 1024, 0, st_>>>(dev_, 1, h, use_graph);
    for (int g = 0; g < dev_.ngroups; ++g) {
        if (group_mark_[g]) continue;                        // relax marked the next frontier
        switch (group_D_[g]) {
            case 1: launch_prop<1>(dev_, g, prop_blocks_, st_); break;
            case 2: launch_prop<2>(dev_, g, prop_blocks_, st_); break;
            case 3: launch_prop<3>(dev_, g, prop_blocks_, st_); break;
            default: launch_prop<4>(dev_, g, prop_blocks_, st_); break;
        }
    }
    k_b_compact<<<compact_blocks_, 256, 0, st_>>>(dev_);
    k_b_plan<<<1, 1024, 0, st_>>>(dev_, 2, h, use_graph);
}

int Engine::run_to_completion() {
    if (dev_.n == 0) return BF_OK;
    cudaGraph_t graph;
    BF_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle h;
    BF_CUDA(cudaGraphConditionalHandleCreate(&h, graph, 0, cudaGraphCondAssignDefault));
    cudaGraphNode_t n0;
    {
        void* args[] = {(void*)&dev_.active, (void*)&h};
        cudaKernelNodeParams kp;
        memset(&kp, 0, sizeof kp);
        kp.func = (void*)k_b_cond;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(1);
        kp.kernelParams = args;
        BF_CUDA(cudaGraphAddKernelNode(&n0, graph, nullptr, 0, &kp));
    }
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
    cudaStream_t cs;
    BF_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    BF_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    cudaStream_t keep = st_;
    st_ = cs;
    launch_pass(h, 1);
    st_ = keep;
    cudaGraph_t captured;
    cudaError_t e = cudaStreamEndCapture(cs, &captured);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return bfh::cuda_fail(e, "batch graph capture"); }
    cudaGraphExec_t exec;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return bfh::cuda_fail(e, "batch graph instantiate"); }
    e = cudaGraphLaunch(exec, st_);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bfh::cuda_fail(e, "batch graph launch");
    return BF_OK;
}

void Engine::drop_step_graphs() {
    for (int i = 0; i < 2; ++i) {
        if (step_exec_[i]) cudaGraphExecDestroy(step_exec_[i]);
        step_exec_[i] = nullptr;
        step_passes_[i] = 0;
    }
}

int Engine::build_step_graph(int passes, cudaGraphExec_t* out) {
    cudaGraph_t graph;
    BF_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return bfh::cuda_fail(e, "step graph handle"); }
    cudaGraphNode_t n0;
    {
        int* left = dev_.step_left;
        const int* act = dev_.active;
        void* args[] = {(void*)&left, (void*)&act, (void*)&passes, (void*)&h};
        cudaKernelNodeParams kp;
        memset(&kp, 0, sizeof kp);
        kp.func = (void*)k_b_step_init;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(1);
        kp.kernelParams = args;
        e = cudaGraphAddKernelNode(&n0, graph, nullptr, 0, &kp);
        if (e != cudaSuccess) { cudaGraphDestroy(graph); return bfh::cuda_fail(e, "step graph node"); }
    }
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    memset(cp_raw, 0, sizeof cp_raw);
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t nc;
    e = cudaGraphAddNode(&nc, graph, &n0, nullptr, 1, &cp);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return bfh::cuda_fail(e, "step graph loop"); }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return bfh::cuda_fail(e, "step graph stream"); }
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaStream_t keep = st_;
        st_ = cs;
        launch_pass(h, 2);
        st_ = keep;
        cudaGraph_t captured;
        e = cudaStreamEndCapture(cs, &captured);
    }
    cudaStreamDestroy(cs);
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bfh::cuda_fail(e, "step graph");
    return BF_OK;
}

int Engine::step(int passes, bool graph) {
    if (dev_.n == 0 || passes <= 0) return BF_OK;
    if (!graph) {
        for (int p = 0; p < passes; ++p) launch_pass(0, 0);
        BF_CUDA(cudaGetLastError());
        return BF_OK;
    }
    int slot = -1;
    for (int i = 0; i < 2; ++i)
        if (step_exec_[i] && step_passes_[i] == passes) slot = i;
    if (slot < 0) {
        slot = step_exec_[0] ? (step_exec_[1] ? 0 : 1) : 0;
        if (step_exec_[slot]) cudaGraphExecDestroy(step_exec_[slot]);
        step_exec_[slot] = nullptr;
        const int rc = build_step_graph(passes, &step_exec_[slot]);
        if (rc) return rc;
        step_passes_[slot] = passes;
    }
    BF_CUDA(cudaGraphLaunch(step_exec_[slot], st_));
    return BF_OK;
}

int Engine::read_counters(std::vector<Counters>& out) {
    out.resize(insts_.size());
    for (size_t i = 0; i < insts_.size(); ++i)
        BF_CUDA(cudaMemcpyAsync(&out[i], insts_[i]->view.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st_));
    BF_CUDA(cudaStreamSynchronize(st_));
    return BF_OK;
}

int Engine::finish_instance(InstState* s, int64_t* iters, int32_t* status, int* err) {
    const long long C = s->a->g.C;
    k_b_output<<<blocks_for(C), 256, 0, st_>>>(C, s->view.Vkey, s->Vdev);
    BF_CUDA(cudaGetLastError());
    if (s->V_host) BF_CUDA(cudaMemcpyAsync(s->V_host, s->Vdev, 8 * (size_t)C, cudaMemcpyDeviceToHost, st_));
    if (s->mu_host) BF_CUDA(cudaMemcpyAsync(s->mu_host, s->view.mu, (size_t)C, cudaMemcpyDeviceToHost, st_));
    else BF_CUDA(cudaMemcpyAsync(s->mu_dev_out, s->view.mu, (size_t)C, cudaMemcpyDeviceToDevice, st_));
    Counters hc;
    BF_CUDA(cudaMemcpyAsync(&hc, s->view.ctr, sizeof hc, cudaMemcpyDeviceToHost, st_));
    BF_CUDA(cudaStreamSynchronize(st_));
    *iters = hc.round;
    *status = hc.status;
    *err = hc.err;
    return BF_OK;
}

}  // namespace bfb

extern "C" int bf_solve_batch(int32_t n, const bf_abstraction* const* abs, const double* const* G,
                              const uint8_t* const* target, const uint8_t* const* avoid,
                              const double* const* terminal, int64_t max_iters, double* const* V,
                              uint8_t* const* mu, int64_t* iters, int32_t* status, void* stream) {
    if (n < 0 || (n > 0 && (!abs || !G || !V || !mu || !iters || !status))) {
        bfh::set_error("bf_solve_batch: NULL argument array");
        return BF_ERR_INVALID;
    }
    if (n == 0) return BF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    bfb::Engine eng(st);
    std::vector<bfb::InstState*> order(n);
    for (int i = 0; i < n; ++i) {
        int rc = eng.add(abs[i], G[i], target ? target[i] : nullptr, avoid ? avoid[i] : nullptr,
                         terminal ? terminal[i] : nullptr, max_iters, V[i], mu[i], &order[i]);
        if (rc) return rc;
    }
    int rc = eng.rebuild();
    if (rc) return rc;
    rc = eng.run_to_completion();
    if (rc) return rc;
    int first_err = -1;
    for (int i = 0; i < n; ++i) {
        int err = 0;
        rc = eng.finish_instance(order[i], &iters[i], &status[i], &err);
        if (rc) return rc;
        if (err && first_err < 0) first_err = i;
    }
    if (first_err >= 0) {
        bfh::set_error("bf_solve_batch: instance %d has NaN, -inf or |value| > 2^64 in G or the terminal cost",
                       first_err);
        return BF_ERR_INVALID;
    }
    return BF_OK;
}

// ---------------------------------------------------------------------------
// schedule tuning of the batched form
// ---------------------------------------------------------------------------
static int batch_time(int32_t n, const bf_abstraction* const* abs, const double* const* G,
                      const uint8_t* const* target, const uint8_t* const* avoid, const double* const* terminal,
                      int64_t max_iters, double* const* V, uint8_t* const* mu, int64_t* it, int32_t* stv,
                      cudaStream_t st, double* ms) {
    int rc = bf_solve_batch(n, abs, G, target, avoid, terminal, max_iters, V, mu, it, stv, st);
    if (rc) return rc;
    cudaEvent_t e0, e1;
    BF_CUDA(cudaEventCreate(&e0));
    BF_CUDA(cudaEventCreate(&e1));
    cudaEventRecord(e0, st);
    for (int r = 0; r < 2 && rc == BF_OK; ++r) rc = bf_solve_batch(n, abs, G, target, avoid, terminal, max_iters, V, mu, it, stv, st);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = t / 2.0;
    return rc;
}

extern "C" int bf_tune_batch(int32_t n, const bf_abstraction* const* abs, const double* const* G,
                             const uint8_t* const* target, const uint8_t* const* avoid,
                             const double* const* terminal, int64_t max_iters, bf_tune_result* out, void* stream) {
    if (n <= 0 || !abs || !G || !out) {
        bfh::set_error("bf_tune_batch: NULL argument or no instance");
        return BF_ERR_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<double*> V(n, nullptr);
    std::vector<uint8_t*> mu(n, nullptr);
    std::vector<int64_t> it(n);
    std::vector<int32_t> stv(n);
    int rc = BF_OK;
    for (int i = 0; i < n && rc == BF_OK; ++i) {
        cudaError_t e = cudaMalloc((void**)&V[i], 8 * (size_t)abs[i]->g.C);
        if (e == cudaSuccess) e = cudaMalloc((void**)&mu[i], (size_t)abs[i]->g.C);
        if (e != cudaSuccess) rc = bfh::cuda_fail(e, "bf_tune_batch buffers");
    }
    std::vector<int> keep(n);
    for (int i = 0; i < n; ++i) keep[i] = abs[i]->bsched;
    auto set_all = [&](int bs) {
        for (int i = 0; i < n; ++i) const_cast<bf_abstraction*>(abs[i])->bsched = bs;
    };
    double best = 0.0;
    int tried = 0;
    int b = kBsDefault;
    if (rc == BF_OK) {
        set_all(-1);
        rc = batch_time(n, abs, G, target, avoid, terminal, max_iters, V.data(), mu.data(), it.data(), stv.data(),
                        st, &best);
        ++tried;
    }
    const double default_ms = best;
    // coordinate descent over the schedule bits, two rounds; the marking
    // dimension times both fixed choices against marking by box size
    const int bits[6] = {kBsMark, kBsWindow33, kBsPlane, kBsTemplates, kBsPair, kBsQueue};
    for (int round = 0; round < 2 && rc == BF_OK; ++round)
        for (int k = 0; k < 6 && rc == BF_OK; ++k) {
            const int base = b;
            int cands[2];
            if (k == 0) {
                cands[0] = base & ~(kBsMark | kBsMarkAuto);
                cands[1] = (base & ~kBsMarkAuto) | kBsMark;
            } else {
                cands[0] = base & ~bits[k];
                cands[1] = base | bits[k];
            }
            for (int j = 0; j < 2 && rc == BF_OK; ++j) {
                const int c = cands[j];
                if (c == base) continue;
                set_all(c);
                double ms = 0.0;
                rc = batch_time(n, abs, G, target, avoid, terminal, max_iters, V.data(), mu.data(), it.data(),
                                stv.data(), st, &ms);
                ++tried;
                if (rc == BF_OK && ms < best) {
                    best = ms;
                    b = c;
                }
            }
        }
    for (int i = 0; i < n; ++i) {
        cudaFree(V[i]);
        cudaFree(mu[i]);
    }
    if (rc) {
        for (int i = 0; i < n; ++i) const_cast<bf_abstraction*>(abs[i])->bsched = keep[i];
        return rc;
    }
    set_all(b);
    const int bs = b;
    memset(out, 0, sizeof *out);
    out->fuse_mark = (bs & kBsMarkAuto) ? -1 : ((bs & kBsMark) ? 1 : 0);
    out->window33 = (bs & kBsWindow33) ? 1 : 0;
    out->plane_lists = (bs & kBsPlane) ? 1 : 0;
    out->templates = (bs & kBsTemplates) ? 1 : 0;
    out->pair_inputs = (bs & kBsPair) ? 1 : 0;
    out->cell_masks = (bs & kBsQueue) ? 2 : 0;
    out->candidates = tried;
    out->best_ms = best;
    out->default_ms = default_ms;
    return BF_OK;
}

extern "C" int bf_set_batch_schedule(bf_abstraction* a, const bf_tune_result* sched) {
    if (!a || !sched) {
        bfh::set_error("bf_set_batch_schedule: NULL argument");
        return BF_ERR_INVALID;
    }
    if (sched->fuse_mark < -1 || sched->fuse_mark > 1) {
        bfh::set_error("bf_set_batch_schedule: fuse_mark must be -1, 0 or 1");
        return BF_ERR_INVALID;
    }
    int bs = (sched->window33 ? kBsWindow33 : 0) | (sched->plane_lists ? kBsPlane : 0) |
             (sched->templates ? kBsTemplates : 0) | (sched->pair_inputs ? kBsPair : 0) |
             (sched->cell_masks ? kBsQueue : 0);
    if (sched->fuse_mark == 1) bs |= kBsMark;
    if (sched->fuse_mark == -1) bs |= kBsMarkAuto;
    a->bsched = bs;
    return BF_OK;
}
