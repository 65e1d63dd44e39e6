// solve_hybrid.cu -- the generic relax kernel of bf_solve (solve_core.cuh:
// relax_pass) for hybrid mode (the records of the first inputs stored, the
// other boxes regenerated inside the kernel), in its own translation unit so that the
// library's units compile side by side.
#include "solve_core.cuh"

using namespace bfk;

template <int D, int FMT, bool COUNT, bool MARK>
__global__ void __launch_bounds__(256, (FMT == kBoxRecompute || FMT == kBoxHybrid) ? 2 : 4) k_relax(InstView v) {
    relax_pass<D, FMT, COUNT, MARK, false>(v);
}

template <int D, int FMT>
static void launch_df(const InstView& v, bool count, bool mark, int blocks, cudaStream_t st) {
    if (mark) {
        if (count) k_relax<D, FMT, true, true><<<blocks, 256, 0, st>>>(v);
        else k_relax<D, FMT, false, true><<<blocks, 256, 0, st>>>(v);
    } else {
        if (count) k_relax<D, FMT, true, false><<<blocks, 256, 0, st>>>(v);
        else k_relax<D, FMT, false, false><<<blocks, 256, 0, st>>>(v);
    }
}

template <int D, int FMT>
static int wave_df() {
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_relax<D, FMT, false, true>, 256, 0);
    return (per_sm < 1 ? 1 : per_sm) * sms;
}

template <int FMT>
static void launch_f(const InstView& v, bool count, bool mark, int blocks, cudaStream_t st) {
    switch (v.g.D) {
        case 1: launch_df<1, FMT>(v, count, mark, blocks, st); break;
        case 2: launch_df<2, FMT>(v, count, mark, blocks, st); break;
        case 3: launch_df<3, FMT>(v, count, mark, blocks, st); break;
        default: launch_df<4, FMT>(v, count, mark, blocks, st); break;
    }
}

template <int FMT>
static int wave_f(int D) {
    switch (D) {
        case 1: return wave_df<1, FMT>();
        case 2: return wave_df<2, FMT>();
        case 3: return wave_df<3, FMT>();
        default: return wave_df<4, FMT>();
    }
}

// One launch of the generic relax in hybrid mode.
void launch_relax_hybrid(const InstView& v, bool count, bool mark, int blocks, cudaStream_t st) {
    launch_f<kBoxHybrid>(v, count, mark, blocks, st);
}

// One full wave of the hybrid-mode relax kernel of dimension D.
int relax_wave_hybrid(int D) { return wave_f<kBoxHybrid>(D); }
