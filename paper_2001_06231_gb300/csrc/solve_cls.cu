// solve_cls.cu -- successor-class relax kernels (relax_cls.cuh), plain passes.
#include "relax_cls.cuh"

using namespace bfk;

// Host: launch one class relax pass on the view's grid (blocks as for k_relax).
void launch_relax_cls(const InstView& v, bool mark, int blocks, cudaStream_t st) {
    launch_cls<false>(v, mark, blocks, st);
}
