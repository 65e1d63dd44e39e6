// serve.cu -- the served form: continuous batching of solve requests on one
// GPU (bf_serve_* in bfgpu.h).
//
// One engine thread owns a stream and a batched pass engine (batch_engine.cuh).
// Each loop iteration it
//   1. admits waiting requests in arrival order while the slot count and the
//      device-memory budget allow (resolving the request's system to a
//      resident abstraction, built in STORED mode when its boxes fit the
//      budget, else in HYBRID mode with the records of as many inputs as
//      fit, else in RECOMPUTE mode -- the memory regulation of Sec. IV-B),
//      copies their inputs to the device and runs their set-up;
//   2. runs a bounded number of passes over every admitted request;
//   3. reads the per-request counters, copies the results of finished
//      requests to their host buffers and frees their state.
// Requests that arrive while others are on the GPU thus join the next step.
// While the engine is idle and at most kDirectMax requests wait, the oldest
// runs at once as a plain bf_solve on the stream (one graph launch for all
// its passes, on the abstraction's cached workspace, whose bytes count against
// the budget from the first such request on); a longer queue goes to the
// engine together.
// The engine runs each request exactly as bf_solve would, so results do not
// depend on what else is in the mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "batch_engine.cuh"

size_t solve_ws_bytes(const bf_abstraction* a);   // solve.cu

namespace {

// An idle engine takes up to this many waiting requests one at a time as plain
// solves (one graph launch each); a longer queue goes to the batched engine.
constexpr int kDirectMax = 4;

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct SystemKey {
    bf_dynamics dyn;
    bf_grid grid;
    std::vector<double> inputs;
    int32_t ninputs = 0, udim = 0;
    double tau = 0.0;

    bool same(const SystemKey& o) const {
        if (dyn.kind != o.dyn.kind || dyn.rk4_substeps != o.dyn.rk4_substeps) return false;
        for (int i = 0; i < 8; ++i)
            if (dyn.param[i] != o.dyn.param[i]) return false;
        if (grid.ndim != o.grid.ndim) return false;
        for (int d = 0; d < grid.ndim; ++d)
            if (grid.n[d] != o.grid.n[d] || grid.lo[d] != o.grid.lo[d] || grid.hi[d] != o.grid.hi[d] ||
                (grid.periodic[d] != 0) != (o.grid.periodic[d] != 0))
                return false;
        return ninputs == o.ninputs && udim == o.udim && tau == o.tau && inputs == o.inputs;
    }
};

struct Cached {
    SystemKey key;
    bf_abstraction* a = nullptr;
    size_t bytes = 0;
};

struct Req {
    uint64_t id = 0;
    const bf_abstraction* abs = nullptr;     // caller-owned, or NULL
    bool has_system = false;
    SystemKey sys;
    std::vector<double> G, terminal;       // owned copies (unless borrowed)
    std::vector<uint8_t> target, avoid;
    const double* pG = nullptr;            // what the engine reads: copies or the caller's arrays
    const double* pT = nullptr;
    const uint8_t* pTg = nullptr;
    const uint8_t* pAv = nullptr;
    int64_t max_iters = 0;
    double* V = nullptr;
    uint8_t* mu = nullptr;
    bf_result res{};
    bfb::InstState* inst = nullptr;
    size_t need = 0;
};

}  // namespace

struct bf_server {
    size_t budget = 0, used = 0;
    int max_active = 0, passes = 8;
    int device = 0;
    cudaStream_t st = nullptr;
    std::mutex m;
    std::condition_variable cv_work, cv_done;
    std::deque<Req*> pending;
    std::vector<Req*> active;
    std::unordered_map<uint64_t, Req*> all;
    std::vector<Cached> cache;
    uint64_t next_id = 1;
    bool stop = false;
    std::unordered_set<const bf_abstraction*> direct;   // abstractions whose bf_solve workspace is counted
    std::thread th;
    bfb::Engine* eng = nullptr;
};

namespace {

size_t abs_bytes_estimate(const SystemKey& k, int mode) {
    size_t C = 1;
    for (int d = 0; d < k.grid.ndim; ++d) C *= (size_t)k.grid.n[d];
    const size_t D = (size_t)k.grid.ndim, U = (size_t)k.ninputs;
    size_t b = C * 2 * D * sizeof(short) + U * (size_t)k.udim * 8;   // pred index + inputs
    b += C * D * 8;                                                   // temporary pred bounds
    if (mode == BF_MODE_STORED) b += C * U * 4 * D;                  // boxes
    else if (D >= 3 && k.dyn.rk4_substeps <= bfk::kRkMaxSub)         // shared RK4 parts
        b += sizeof(double) * bfk::kRkEntry * U * (C / ((size_t)k.grid.n[0] * k.grid.n[1]));
    return b;
}

size_t state_bytes_estimate(const SystemKey& k) {
    long long C = 1;
    for (int d = 0; d < k.grid.ndim; ++d) C *= k.grid.n[d];
    return bfb::Engine::state_bytes_for(C, k.ninputs, true, true, true);   // as admission counts it
}

// Find or build the abstraction of a request's system.  Called with the lock
// held; builds outside it.  Returns the abstraction or NULL (*wait = true when
// it may fit later, false when it can never fit).
const bf_abstraction* resolve(bf_server* s, Req* r, std::unique_lock<std::mutex>& lk, bool* wait) {
    *wait = false;
    if (r->abs) return r->abs;
    for (Cached& c : s->cache)
        if (c.key.same(r->sys)) return c.a;
    const size_t need_state = state_bytes_estimate(r->sys);
    int mode = -1;
    size_t est = 0, box_budget = 0;
    const size_t base = abs_bytes_estimate(r->sys, BF_MODE_RECOMPUTE);
    if (s->used + abs_bytes_estimate(r->sys, BF_MODE_STORED) + need_state <= s->budget) {
        mode = BF_MODE_STORED;
        est = abs_bytes_estimate(r->sys, BF_MODE_STORED);
    } else if (s->used + base + need_state <= s->budget) {
        // store the records of as many inputs as the rest of the budget holds
        box_budget = s->budget - s->used - base - need_state;
        size_t C = 1;
        for (int d = 0; d < r->sys.grid.ndim; ++d) C *= (size_t)r->sys.grid.n[d];
        const size_t per_input = C * (r->sys.grid.ndim <= 2 ? 4 : 8);
        const size_t K = std::min<size_t>((size_t)r->sys.ninputs, box_budget / per_input);
        mode = K > 0 ? BF_MODE_HYBRID : BF_MODE_RECOMPUTE;
        est = base + K * per_input;
        box_budget = K * per_input;          // the stored records only (no frontier cache)
    }
    if (mode < 0) {
        // fits once other requests leave, unless nothing is running
        *wait = !s->active.empty();
        return nullptr;
    }
    s->used += est;                     // reserve while building
    lk.unlock();
    bf_inputs in;
    in.ninputs = r->sys.ninputs;
    in.udim = r->sys.udim;
    in.u = r->sys.inputs.data();
    bf_abstraction* a = nullptr;
    const int rc = mode == BF_MODE_HYBRID
                       ? abs_build_hybrid(&r->sys.dyn, &r->sys.grid, &in, r->sys.tau, (int64_t)box_budget, s->st, &a)
                       : abs_build(&r->sys.dyn, &r->sys.grid, &in, r->sys.tau, mode, s->st, &a);
    lk.lock();
    if (rc != BF_OK) {
        s->used -= est;
        r->res.error = rc;
        return nullptr;
    }
    Cached c;
    c.key = r->sys;
    c.a = a;
    c.bytes = est;
    s->cache.push_back(c);
    return a;
}

void engine_loop(bf_server* s) {
    cudaSetDevice(s->device);
    std::unordered_map<bfb::InstState*, Req*> owner;
    std::vector<bfk::Counters> ctrs;
    for (;;) {
        std::vector<std::pair<Req*, const bf_abstraction*>> admit;
        std::vector<Req*> failed;
        bool waiting = false;               // requests left in the queue after admission
        Req* solo = nullptr;                // a lone request on an idle engine: plain bf_solve
        const bf_abstraction* solo_a = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->m);
            s->cv_work.wait(lk, [&] { return s->stop || !s->pending.empty() || !s->active.empty(); });
            if (s->stop && s->pending.empty() && s->active.empty()) break;
            if (s->active.empty() && !s->pending.empty() && s->pending.size() <= (size_t)kDirectMax) {
                Req* r = s->pending.front();
                bool wait = false;
                const bf_abstraction* a = resolve(s, r, lk, &wait);
                if (a) {
                    const size_t ws = s->direct.count(a) ? 0 : solve_ws_bytes(a);
                    if (s->used + ws <= s->budget && s->pending.size() <= (size_t)kDirectMax &&
                        s->pending.front() == r) {
                        s->pending.pop_front();
                        if (ws) {
                            s->direct.insert(a);
                            s->used += ws;
                        }
                        solo = r;
                        solo_a = a;
                        r->res.mode = a->mode;
                        r->res.admit_s = now_s();
                    }
                }
            }
        }
        if (solo) {
            bf_solve_opts o;
            memset(&o, 0, sizeof o);
            o.terminal = solo->pT;
            o.max_iters = solo->max_iters;
            int64_t it = 0;
            int32_t stt = 0;
            const int rc = bf_solve(solo_a, solo->pG, solo->pT ? nullptr : solo->pTg, solo->pAv, &o, solo->V,
                                    solo->mu, &it, &stt, s->st);
            std::lock_guard<std::mutex> lk(s->m);
            solo->res.iters = it;
            solo->res.status = stt;
            solo->res.error = rc;
            solo->res.finish_s = now_s();
            solo->res.done = 1;
            s->cv_done.notify_all();
            continue;
        }
        {
            std::unique_lock<std::mutex> lk(s->m);
            if (s->stop && s->pending.empty() && s->active.empty()) break;
            while (!s->pending.empty() && (int)(s->active.size() + admit.size()) < s->max_active) {
                Req* r = s->pending.front();
                bool wait = false;
                const bf_abstraction* a = resolve(s, r, lk, &wait);
                if (!a) {
                    if (wait || (!admit.empty())) break;                 // retry after others leave
                    s->pending.pop_front();
                    if (r->res.error == BF_OK) r->res.error = BF_ERR_OOM;
                    failed.push_back(r);
                    continue;
                }
                const size_t need = s->eng->state_bytes(a, true, true, true);
                if (s->used + need > s->budget) {
                    if (!s->active.empty() || !admit.empty()) break;
                    s->pending.pop_front();
                    r->res.error = BF_ERR_OOM;
                    failed.push_back(r);
                    continue;
                }
                s->pending.pop_front();
                s->used += need;
                r->need = need;
                r->res.mode = a->mode;
                admit.push_back({r, a});
            }
            waiting = !s->pending.empty();
        }
        bool changed = false;
        for (auto& pa : admit) {
            Req* r = pa.first;
            const int rc = s->eng->add(pa.second, r->pG, r->pTg, r->pAv, r->pT, r->max_iters, r->V, r->mu,
                                       &r->inst);
            std::lock_guard<std::mutex> lk(s->m);
            r->res.admit_s = now_s();
            if (rc != BF_OK) {
                r->res.error = rc;
                s->used -= r->need;
                failed.push_back(r);
            } else {
                owner[r->inst] = r;
                s->active.push_back(r);
                changed = true;
            }
        }
        if (!failed.empty()) {
            std::lock_guard<std::mutex> lk(s->m);
            for (Req* r : failed) {
                r->res.done = 1;
                r->res.finish_s = now_s();
            }
            s->cv_done.notify_all();
        }
        if (changed) s->eng->rebuild();
        if (s->eng->list().empty()) continue;
        // with nobody waiting for a slot, longer steps cost no admission delay and
        // save host round trips; arrivals then wait at most one longer step
        if (waiting) s->eng->step(s->passes);        // the set changes often: host-launched passes
        else s->eng->step(4 * s->passes, true);    // light load: one graph launch per step
        if (s->eng->read_counters(ctrs) != BF_OK) {
            // a CUDA error: fail every active request
            std::lock_guard<std::mutex> lk(s->m);
            for (Req* r : s->active) {
                r->res.error = BF_ERR_CUDA;
                r->res.done = 1;
                r->res.finish_s = now_s();
            }
            s->active.clear();
            s->cv_done.notify_all();
            continue;
        }
        std::vector<bfb::InstState*> finished;
        for (size_t i = 0; i < ctrs.size(); ++i)
            if (ctrs[i].done) finished.push_back(s->eng->list()[i]);
        if (finished.empty()) continue;
        for (bfb::InstState* inst : finished) {
            Req* r = owner[inst];
            int64_t it = 0;
            int32_t stt = 0;
            int err = 0;
            const int rc = s->eng->finish_instance(inst, &it, &stt, &err);
            s->eng->remove(inst);
            owner.erase(inst);
            std::lock_guard<std::mutex> lk(s->m);
            r->res.iters = it;
            r->res.status = stt;
            r->res.error = rc != BF_OK ? rc : (err ? BF_ERR_INVALID : BF_OK);
            r->res.finish_s = now_s();
            r->res.done = 1;
            s->used -= r->need;
            s->active.erase(std::find(s->active.begin(), s->active.end(), r));
        }
        s->eng->rebuild();
        std::lock_guard<std::mutex> lk(s->m);
        s->cv_done.notify_all();
    }
}

}  // namespace

extern "C" int bf_serve_open(size_t hbm_budget, int32_t max_active, int32_t passes_per_step, bf_server** out) {
    if (!out || hbm_budget == 0 || max_active < 1 || max_active > 65536 || passes_per_step < 0) {
        bfh::set_error("bf_serve_open: need out, a budget, 1 <= max_active <= 65536, passes_per_step >= 0");
        return BF_ERR_INVALID;
    }
    bf_server* s = new bf_server;
    s->budget = hbm_budget;
    s->max_active = max_active;
    s->passes = passes_per_step ? passes_per_step : 8;
    cudaGetDevice(&s->device);
    cudaError_t e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete s;
        return bfh::cuda_fail(e, "bf_serve_open stream");
    }
    s->eng = new bfb::Engine(s->st);
    s->th = std::thread(engine_loop, s);
    *out = s;
    return BF_OK;
}

extern "C" int bf_serve_submit(bf_server* s, const bf_request* q, uint64_t* id) {
    if (!s || !q || !id || !q->G || !q->V || !q->mu || (!q->target && !q->terminal)) {
        bfh::set_error("bf_serve_submit: need G, V, mu and a target or terminal cost");
        return BF_ERR_INVALID;
    }
    if (!q->abs && (!q->dyn || !q->grid || !q->inputs || !q->inputs->u)) {
        bfh::set_error("bf_serve_submit: need an abstraction or a system (dyn, grid, inputs, tau)");
        return BF_ERR_INVALID;
    }
    Req* r = new Req;
    long long C = 1;
    int U = 0;
    if (q->abs) {
        r->abs = q->abs;
        int64_t nc = 0;
        int32_t nu = 0;
        abs_info(q->abs, &nc, &nu, nullptr, nullptr, nullptr, nullptr);
        C = nc;
        U = nu;
    } else {
        if (q->grid->ndim < 1 || q->grid->ndim > 4 || q->inputs->ninputs < 1 || q->inputs->udim < 1) {
            delete r;
            bfh::set_error("bf_serve_submit: invalid system");
            return BF_ERR_INVALID;
        }
        r->has_system = true;
        r->sys.dyn = *q->dyn;
        memset(&r->sys.grid, 0, sizeof r->sys.grid);
        r->sys.grid.ndim = q->grid->ndim;
        for (int d = 0; d < q->grid->ndim; ++d) {
            r->sys.grid.n[d] = q->grid->n[d];
            r->sys.grid.lo[d] = q->grid->lo[d];
            r->sys.grid.hi[d] = q->grid->hi[d];
            r->sys.grid.periodic[d] = q->grid->periodic[d] ? 1 : 0;
            C *= q->grid->n[d];
        }
        r->sys.ninputs = q->inputs->ninputs;
        r->sys.udim = q->inputs->udim;
        r->sys.inputs.assign(q->inputs->u, q->inputs->u + (size_t)q->inputs->ninputs * q->inputs->udim);
        r->sys.tau = q->tau;
        U = q->inputs->ninputs;
    }
    if (q->flags & BF_REQ_BORROW_INPUTS) {
        r->pG = q->G;
        r->pT = q->terminal;
        r->pTg = q->terminal ? nullptr : q->target;
        r->pAv = q->avoid;
    } else {
        r->G.assign(q->G, q->G + (size_t)C * U);
        if (q->terminal) r->terminal.assign(q->terminal, q->terminal + C);
        else r->target.assign(q->target, q->target + C);
        if (q->avoid) r->avoid.assign(q->avoid, q->avoid + C);
        r->pG = r->G.data();
        r->pT = r->terminal.empty() ? nullptr : r->terminal.data();
        r->pTg = r->target.empty() ? nullptr : r->target.data();
        r->pAv = r->avoid.empty() ? nullptr : r->avoid.data();
    }
    r->max_iters = q->max_iters;
    r->V = q->V;
    r->mu = q->mu;
    std::lock_guard<std::mutex> lk(s->m);
    r->id = s->next_id++;
    r->res.submit_s = now_s();
    s->all[r->id] = r;
    s->pending.push_back(r);
    *id = r->id;
    s->cv_work.notify_one();
    return BF_OK;
}

extern "C" int bf_serve_poll(bf_server* s, uint64_t id, int32_t wait, bf_result* out) {
    if (!s || !out) {
        bfh::set_error("bf_serve_poll: NULL argument");
        return BF_ERR_INVALID;
    }
    std::unique_lock<std::mutex> lk(s->m);
    auto it = s->all.find(id);
    if (it == s->all.end()) {
        bfh::set_error("bf_serve_poll: unknown request %llu", (unsigned long long)id);
        return BF_ERR_INVALID;
    }
    Req* r = it->second;
    if (wait) s->cv_done.wait(lk, [&] { return r->res.done != 0; });
    *out = r->res;
    if (r->res.done) {
        s->all.erase(it);
        delete r;
    }
    return BF_OK;
}

extern "C" void bf_serve_close(bf_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->m);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->th.joinable()) s->th.join();
    delete s->eng;
    for (Cached& c : s->cache) abs_free(c.a);
    for (auto& kv : s->all) delete kv.second;
    cudaStreamDestroy(s->st);
    delete s;
}
