// relax_cls.cuh -- relax kernels of the single solve for a running cost that
// depends on the successor through a class (g2 of Sec. VI-A): g(x,y,u) =
// Gc(x,u) for y in the class, G(x,u) else.  Instantiated in two translation
// units (solve_cls.cu, solve_cls_count.cu) so they compile in parallel.
#pragma once
#include "solve_core.cuh"

namespace bfk {

template <int D, int FMT, bool COUNT, bool MARK>
__global__ void __launch_bounds__(256, (FMT == kBoxRecompute || FMT == kBoxHybrid) ? 2 : 4) k_relax_cls(InstView v) {
    relax_pass<D, FMT, COUNT, MARK, true>(v);
}

template <int D, int FMT, bool COUNT>
static void launch_cls_fmt(const InstView& v, bool mark, int blocks, cudaStream_t st) {
    if (mark) k_relax_cls<D, FMT, COUNT, true><<<blocks, 256, 0, st>>>(v);
    else k_relax_cls<D, FMT, COUNT, false><<<blocks, 256, 0, st>>>(v);
}

template <int D, bool COUNT>
static void launch_cls_d(const InstView& v, bool mark, int blocks, cudaStream_t st) {
    switch (v.box_fmt) {
        case kBoxCompact: launch_cls_fmt<D, kBoxCompact, COUNT>(v, mark, blocks, st); break;
        case kBoxRecompute: launch_cls_fmt<D, kBoxRecompute, COUNT>(v, mark, blocks, st); break;
        case kBoxHybrid: launch_cls_fmt<D, kBoxHybrid, COUNT>(v, mark, blocks, st); break;
        default: launch_cls_fmt<D, kBoxWide, COUNT>(v, mark, blocks, st); break;
    }
}

template <bool COUNT>
static void launch_cls(const InstView& v, bool mark, int blocks, cudaStream_t st) {
    switch (v.g.D) {
        case 1: launch_cls_d<1, COUNT>(v, mark, blocks, st); break;
        case 2: launch_cls_d<2, COUNT>(v, mark, blocks, st); break;
        case 3: launch_cls_d<3, COUNT>(v, mark, blocks, st); break;
        default: launch_cls_d<4, COUNT>(v, mark, blocks, st); break;
    }
}

}  // namespace bfk
