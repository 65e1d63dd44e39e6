// solve_cls_count.cu -- successor-class relax kernels (relax_cls.cuh) that also
// count the cells of the exact F1 (BF_FLAG_COUNT_EXACT).
#include "relax_cls.cuh"

using namespace bfk;

void launch_relax_cls_count(const InstView& v, bool mark, int blocks, cudaStream_t st) {
    launch_cls<true>(v, mark, blocks, st);
}
