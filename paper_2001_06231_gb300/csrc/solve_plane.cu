// solve_plane.cu -- the relax kernel of bf_solve for abstractions with plane
// lookup lists (solve_core.cuh: plane_offsets, relax_plane), in its own
// translation unit so that it compiles beside solve.cu.
//
// Two forms: one input per iteration (64 registers, 4 blocks of 256 threads
// per SM), or two inputs per iteration with the lookups of both in flight
// (3 blocks per SM); the schedule picks one.  The lists of the plane a warp is
// on are staged in dynamic shared memory (plane_smem_bytes() per block).
#include "solve_core.cuh"

using namespace bfk;

template <int D, bool COUNT, bool MARK, bool PAIR>
__global__ void __launch_bounds__(256, PAIR ? 3 : 4) k_relax_pl(InstView v) {
    relax_pass<D, kBoxCompact, COUNT, MARK, false, PAIR ? 2 : 1>(v);
}

size_t plane_smem_bytes() { return 8 * sizeof(PlaneStage); }

template <int D, bool PAIR>
static int wave_of() {
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_relax_pl<D, false, true, PAIR>, 256,
                                                  plane_smem_bytes());
    return (per_sm < 1 ? 1 : per_sm) * sms;
}

// One full wave of the plane relax kernel of dimension D (2..4).
int plane_relax_wave(int D, bool pair) {
    switch (D) {
        case 2: return pair ? wave_of<2, true>() : wave_of<2, false>();
        case 3: return pair ? wave_of<3, true>() : wave_of<3, false>();
        default: return pair ? wave_of<4, true>() : wave_of<4, false>();
    }
}

template <int D>
static void launch_d(const InstView& v, bool count, bool mark, bool pair, int blocks, cudaStream_t st) {
    const size_t sm = plane_smem_bytes();
    if (count) {                                   // counting mode: one form
        if (mark) k_relax_pl<D, true, true, false><<<blocks, 256, sm, st>>>(v);
        else k_relax_pl<D, true, false, false><<<blocks, 256, sm, st>>>(v);
    } else if (pair) {
        if (mark) k_relax_pl<D, false, true, true><<<blocks, 256, sm, st>>>(v);
        else k_relax_pl<D, false, false, true><<<blocks, 256, sm, st>>>(v);
    } else {
        if (mark) k_relax_pl<D, false, true, false><<<blocks, 256, sm, st>>>(v);
        else k_relax_pl<D, false, false, false><<<blocks, 256, sm, st>>>(v);
    }
}

void launch_relax_plane(const InstView& v, bool count, bool mark, bool pair, int blocks, cudaStream_t st) {
    switch (v.g.D) {
        case 2: launch_d<2>(v, count, mark, pair, blocks, st); break;
        case 3: launch_d<3>(v, count, mark, pair, blocks, st); break;
        default: launch_d<4>(v, count, mark, pair, blocks, st); break;
    }
}
