// batch_engine.cuh -- the batched form of Algorithm 1: many independent
// instances (each with its own abstraction, costs, target and avoid set;
// uneven sizes) advanced together.  A pass is one relax launch per group of
// instances sharing dimension and storage mode, one planning launch, one
// propagate launch per group whose predecessor boxes are too large for relax
// to mark the next frontier itself, one compaction launch (which also commits
// W) and one finishing launch; each launch covers every unfinished instance,
// its warps pulling (instance, 32-cell chunk) or (instance, changed cell) work
// items through per-instance prefix offsets.
// Instances keep their own pass counters, frontiers and termination, so each
// result is identical to a solo bf_solve.
//
// bf_solve_batch runs the pass loop inside a CUDA graph WHILE node; the
// server (serve.cu) runs a bounded number of passes per engine step and lets
// instances join and leave between steps.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "solve_core.cuh"

namespace bfb {

using bfk::Counters;
using bfk::InstView;

constexpr int kMaxGroups = 16;  // D in 1..4 x {wide, compact, recompute, hybrid} boxes
constexpr double kFuseMarkRowsBatch = 64.0;   // mean predecessor-box rows up to which relax marks

// Device-side description of one batch (rebuilt when the instance set changes).
struct BatchDev {
    InstView* views;    // [n], ordered by group
    int* scan;          // [n + 1] exclusive prefix of the per-instance relax chunks
    int* scan_chg;      // [n + 1] exclusive prefix of the changed cells
    int* scan_cmp;      // [n + 1] exclusive prefix of the 256-word compaction chunks
    int* active;        // [1] unfinished instances
    int* step_left;     // [1] passes left in a bounded engine step (graph form)
    int n;
    int ngroups;
    int gbeg[kMaxGroups + 1];   // instances of group g are [gbeg[g], gbeg[g + 1])
};

// Per-instance device state, carved from one buffer.
struct InstState {
    const bf_abstraction* a = nullptr;
    InstView view;
    void* mem = nullptr;          // owned allocation (state + staging)
    double* G = nullptr;          // device copies or caller device pointers
    const unsigned char* target = nullptr;
    const unsigned char* avoid = nullptr;
    const double* terminal = nullptr;
    double* Vdev = nullptr;       // device V output (caller's or staging)
    double* V_host = nullptr;     // caller host V (copied back at the end) or NULL
    unsigned char* mu_host = nullptr;
    unsigned char* mu_dev_out = nullptr;
    long long cap = 0;
    int group = 0;
    bool done = false;
};

// Engine: owns the device batch description and launches passes.
class Engine {
public:
    explicit Engine(cudaStream_t st);
    ~Engine();
    // Set up an instance (allocate state, stage inputs, run lines 1-10 of
    // Algorithm 1).  Inputs may be host or device.  Returns BF_OK or an error.
    int add(const bf_abstraction* a, const double* G, const unsigned char* target,
            const unsigned char* avoid, const double* terminal, long long max_iters,
            double* V, unsigned char* mu, InstState** out);
    // Rebuild the device description for the current instance list (group order).
    int rebuild();
    // Run passes until every instance is done (graph with a WHILE node).
    int run_to_completion();
    // Run at most `passes` passes: host-launched, or (graph) one launch of a
    // WHILE node bounded by a device pass counter, kept until the instance set
    // changes (worth it when the set is stable for several steps).
    int step(int passes, bool graph = false);
    // Copy the results of finished instances out; fills *iters/*status.
    int finish_instance(InstState* s, int64_t* iters, int32_t* status, int* err);
    // Remove an instance (frees its state).
    void remove(InstState* s);
    // Read all counters (host copies, index = position in list()).
    int read_counters(std::vector<Counters>& out);
    std::vector<InstState*>& list() { return insts_; }
    // Device bytes add() allocates for an instance (upper bound when staging).
    size_t state_bytes(const bf_abstraction* a, bool stage_G, bool stage_T, bool stage_V) const;
    // the same for an instance of C cells and U inputs (before its abstraction exists)
    static size_t state_bytes_for(long long C, int U, bool stage_G, bool stage_T, bool stage_V);
    cudaStream_t stream() const { return st_; }

private:
    void launch_pass(cudaGraphConditionalHandle h, int use_graph);
    cudaStream_t st_;
    // stream-ordered pool of the per-instance state; it keeps freed memory
    // (release threshold: unbounded) so that instances joining later reuse it
    // instead of mapping new memory
    cudaMemPool_t pool_ = nullptr;
    int alloc(void** p, size_t bytes);
    std::vector<InstState*> insts_;
    std::vector<InstView> host_views_;   // kept alive until the async copy is done
    BatchDev dev_{};
    void* dev_mem_ = nullptr;
    size_t dev_mem_bytes_ = 0;
    int relax_blocks_ = 0, prop_blocks_ = 0, compact_blocks_ = 0;
    int group_D_[kMaxGroups] = {}, group_fmt_[kMaxGroups] = {};
    bool group_mark_[kMaxGroups] = {};   // relax marks the next frontier (no propagate launch)
    bool group_fixed_mark_[kMaxGroups] = {};   // ... as the first instance's batched schedule says
    bool group_plane_[kMaxGroups] = {};  // relax reads the plane lookup lists (plane kernel)
    bool group_pair_[kMaxGroups] = {};   // ... two inputs per iteration
    bool group_queue_[kMaxGroups] = {};  // ... by cell masks, pairs queued over the lanes
    bool group_wide_[kMaxGroups] = {};   // ... some instance has more than 16 inputs
    // bounded-step graphs of the current instance set, by pass count
    cudaGraphExec_t step_exec_[2] = {nullptr, nullptr};
    int step_passes_[2] = {0, 0};
    void drop_step_graphs();
    int build_step_graph(int passes, cudaGraphExec_t* out);
};

}  // namespace bfb
