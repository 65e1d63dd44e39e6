// solve_cls.cu -- relax kernels of the single solve for a running cost that
// depends on the successor through a class (g2 of Sec. VI-A): g(x,y,u) =
// Gc(x,u) for y in the class, G(x,u) else.  Kept apart from solve.cu so the
// two sets of kernels compile in parallel.
#include "solve_core.cuh"

using namespace bfk;

template <int D, int FMT, bool MARK>
__global__ void __launch_bounds__(256, (FMT == kBoxRecompute || FMT == kBoxHybrid) ? 2 : 4) k_relax_cls(InstView v) {
    relax_pass<D, FMT, false, MARK, true>(v);
}

template <int D, int FMT>
static void launch_fmt(const InstView& v, bool mark, int blocks, cudaStream_t st) {
    if (mark) k_relax_cls<D, FMT, true><<<blocks, 256, 0, st>>>(v);
    else k_relax_cls<D, FMT, false><<<blocks, 256, 0, st>>>(v);
}

template <int D>
static void launch_d(const InstView& v, bool mark, int blocks, cudaStream_t st) {
    switch (v.box_fmt) {
        case kBoxCompact: launch_fmt<D, kBoxCompact>(v, mark, blocks, st); break;
        case kBoxRecompute: launch_fmt<D, kBoxRecompute>(v, mark, blocks, st); break;
        case kBoxHybrid: launch_fmt<D, kBoxHybrid>(v, mark, blocks, st); break;
        default: launch_fmt<D, kBoxWide>(v, mark, blocks, st); break;
    }
}

// Host: launch one class relax pass on the view's grid (blocks as for k_relax).
void launch_relax_cls(const InstView& v, bool mark, int blocks, cudaStream_t st) {
    switch (v.g.D) {
        case 1: launch_d<1>(v, mark, blocks, st); break;
        case 2: launch_d<2>(v, mark, blocks, st); break;
        case 3: launch_d<3>(v, mark, blocks, st); break;
        default: launch_d<4>(v, mark, blocks, st); break;
    }
}
