// solve_plane.cu -- the relax kernel of bf_solve for abstractions with plane
// lookup lists (solve_core.cuh: plane_offsets, relax_plane), in its own
// translation unit so that it compiles beside solve.cu.
//
// Two forms: one input per iteration (64 registers, 4 blocks of 256 threads
// per SM), or two inputs per iteration with the lookups of both in flight
// (3 blocks per SM); each also with one block per SM more; the schedule
// picks one.  The lists of the plane a warp is
// on are staged in dynamic shared memory (plane_smem_bytes() per block).
#include "solve_core.cuh"

using namespace bfk;

// OCC: one more block per SM than the registers the form wants would allow
// (5 blocks of the one-input form, 4 of the two-input form), at the price of
// some spilled registers; the schedule picks one.
template <int D, bool COUNT, bool MARK, bool PAIR, bool OCC>
__global__ void __launch_bounds__(256, PAIR ? (OCC ? 4 : 3) : (OCC ? 5 : 4)) k_relax_pl(InstView v) {
    relax_pass<D, kBoxCompact, COUNT, MARK, false, PAIR ? 2 : 1>(v);
}

size_t plane_smem_bytes() { return 8 * sizeof(PlaneStage); }

template <int D, bool PAIR, bool OCC>
static int wave_of() {
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_relax_pl<D, false, true, PAIR, OCC>, 256,
                                                  plane_smem_bytes());
    return (per_sm < 1 ? 1 : per_sm) * sms;
}

template <int D>
static int wave_d(bool pair, bool occ) {
    return pair ? (occ ? wave_of<D, true, true>() : wave_of<D, true, false>())
                : (occ ? wave_of<D, false, true>() : wave_of<D, false, false>());
}

// One full wave of the plane relax kernel of dimension D (2..4).
int plane_relax_wave(int D, bool pair, bool occ) {
    switch (D) {
        case 2: return wave_d<2>(pair, occ);
        case 3: return wave_d<3>(pair, occ);
        default: return wave_d<4>(pair, occ);
    }
}

template <int D, bool PAIR, bool OCC>
static void launch_po(const InstView& v, bool mark, int blocks, cudaStream_t st) {
    const size_t sm = plane_smem_bytes();
    if (mark) k_relax_pl<D, false, true, PAIR, OCC><<<blocks, 256, sm, st>>>(v);
    else k_relax_pl<D, false, false, PAIR, OCC><<<blocks, 256, sm, st>>>(v);
}

template <int D>
static void launch_d(const InstView& v, bool count, bool mark, bool pair, bool occ, int blocks, cudaStream_t st) {
    const size_t sm = plane_smem_bytes();
    if (count) {                                   // counting mode: one form
        if (mark) k_relax_pl<D, true, true, false, false><<<blocks, 256, sm, st>>>(v);
        else k_relax_pl<D, true, false, false, false><<<blocks, 256, sm, st>>>(v);
    } else if (pair) {
        if (occ) launch_po<D, true, true>(v, mark, blocks, st);
        else launch_po<D, true, false>(v, mark, blocks, st);
    } else {
        if (occ) launch_po<D, false, true>(v, mark, blocks, st);
        else launch_po<D, false, false>(v, mark, blocks, st);
    }
}

void launch_relax_plane(const InstView& v, bool count, bool mark, bool pair, bool occ, int blocks, cudaStream_t st) {
    switch (v.g.D) {
        case 2: launch_d<2>(v, count, mark, pair, occ, blocks, st); break;
        case 3: launch_d<3>(v, count, mark, pair, occ, blocks, st); break;
        default: launch_d<4>(v, count, mark, pair, occ, blocks, st); break;
    }
}
