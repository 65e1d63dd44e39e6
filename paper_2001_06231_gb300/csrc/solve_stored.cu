// solve_stored.cu -- the generic relax kernel of bf_solve (solve_core.cuh:
// relax_pass) for boxes stored as wide int16 or compact relative records, in its own translation unit so
// that it compiles beside solve.cu.
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

// One launch of the generic relax for format fmt (kBoxCompact, kBoxWide).
void launch_relax_stored(const InstView& v, int fmt, bool count, bool mark, int blocks, cudaStream_t st) {
    if (fmt == kBoxCompact) launch_f<kBoxCompact>(v, count, mark, blocks, st);
    else launch_f<kBoxWide>(v, count, mark, blocks, st);
}

// One full wave of the generic relax kernel of dimension D and format fmt.
int relax_wave_stored(int D, int fmt) {
    return fmt == kBoxCompact ? wave_f<kBoxCompact>(D) : wave_f<kBoxWide>(D);
}
