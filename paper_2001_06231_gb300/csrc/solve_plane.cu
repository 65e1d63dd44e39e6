// solve_plane.cu -- the relax kernel of bf_solve for abstractions with plane
// lookup lists (solve_core.cuh: plane_offsets, relax_plane), in its own
// translation unit so that it compiles beside solve.cu.
//
// Two forms: one input per iteration (64 registers, 4 blocks of 256 threads
// per SM), or two inputs per iteration with the lookups of both in flight
// (3 blocks per SM); each also with one block per SM more; the schedule
// picks one.  A third kernel (k_relax_pm) reads the per-cell input masks
// (relax_plane_m) and takes two or four inputs per iteration; a fourth
// (k_relax_pq) queues the pairs over the lanes (relax_plane_q).  The lists of
// the plane a warp is on are staged in dynamic shared memory
// (plane_smem_bytes() per block).
#include "solve_core.cuh"

using namespace bfk;

// OCC: one more block per SM than the registers the form wants would allow
// (5 blocks of the one-input form, 4 of the two-input form), at the price of
// some spilled registers; the schedule picks one.
template <int D, bool COUNT, bool MARK, bool PAIR, bool OCC>
__global__ void __launch_bounds__(256, PAIR ? (OCC ? 4 : 3) : (OCC ? 5 : 4)) k_relax_pl(InstView v) {
    relax_pass<D, kBoxCompact, COUNT, MARK, false, PAIR ? 2 : 1>(v);
}

// Masked form (no counting mode): QUAD = four inputs per iteration, else two.
template <int D, bool MARK, bool QUAD>
__global__ void __launch_bounds__(256, QUAD ? 2 : 3) k_relax_pm(InstView v) {
    relax_pass<D, kBoxCompact, false, MARK, false, QUAD ? 4 : 3>(v);
}

// Pair-queue form (relax_plane_q): UM = the stage's inputs (16: U <= 16, 256
// threads; 32: U <= 32, 128 threads), R = pairs per lane per round.
template <int D, bool MARK, int UM, int R>
__global__ void __launch_bounds__(UM == 16 ? 256 : 128, 3) k_relax_pq(InstView v) {
    relax_pass<D, kBoxCompact, false, MARK, false, R == 2 ? 6 : 5, UM>(v);
}

size_t plane_smem_bytes() { return 8 * sizeof(PlaneStage); }

template <int UM>
static size_t pq_smem() { return (UM == 16 ? 8 : 4) * sizeof(PairStage<UM>); }

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

template <int D, bool QUAD>
static int wave_m() {
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_relax_pm<D, true, QUAD>, 256, plane_smem_bytes());
    return (per_sm < 1 ? 1 : per_sm) * sms;
}

// One full wave of the masked plane relax kernel of dimension D (2..4).
int masked_relax_wave(int D, bool quad) {
    switch (D) {
        case 2: return quad ? wave_m<2, true>() : wave_m<2, false>();
        case 3: return quad ? wave_m<3, true>() : wave_m<3, false>();
        default: return quad ? wave_m<4, true>() : wave_m<4, false>();
    }
}

template <int D>
static void launch_m(const InstView& v, bool mark, bool quad, int blocks, cudaStream_t st) {
    const size_t sm = plane_smem_bytes();
    if (quad) {
        if (mark) k_relax_pm<D, true, true><<<blocks, 256, sm, st>>>(v);
        else k_relax_pm<D, false, true><<<blocks, 256, sm, st>>>(v);
    } else {
        if (mark) k_relax_pm<D, true, false><<<blocks, 256, sm, st>>>(v);
        else k_relax_pm<D, false, false><<<blocks, 256, sm, st>>>(v);
    }
}

void launch_relax_masked(const InstView& v, bool mark, bool quad, int blocks, cudaStream_t st) {
    switch (v.g.D) {
        case 2: launch_m<2>(v, mark, quad, blocks, st); break;
        case 3: launch_m<3>(v, mark, quad, blocks, st); break;
        default: launch_m<4>(v, mark, quad, blocks, st); break;
    }
}

template <int D, bool MARK, int UM, int R>
static const void* pq_kernel() {
    static bool once = false;
    const void* k = (const void*)k_relax_pq<D, MARK, UM, R>;
    if (!once) {
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pq_smem<UM>());
        once = true;
    }
    return k;
}

template <int D, int UM, int R>
static int wave_q() {
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    pq_kernel<D, true, UM, R>();
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_relax_pq<D, true, UM, R>, UM == 16 ? 256 : 128,
                                                  pq_smem<UM>());
    return (per_sm < 1 ? 1 : per_sm) * sms;
}

template <int D>
static int wave_qd(bool wide, bool two) {
    if (wide) return two ? wave_q<D, 32, 2>() : wave_q<D, 32, 1>();
    return two ? wave_q<D, 16, 2>() : wave_q<D, 16, 1>();
}

// One full wave of the pair-queue relax kernel of dimension D (2..4) for U
// inputs (at most 32), R = two ? 2 : 1.
int queue_relax_wave(int D, int U, bool two) {
    const bool wide = U > 16;
    switch (D) {
        case 2: return wave_qd<2>(wide, two);
        case 3: return wave_qd<3>(wide, two);
        default: return wave_qd<4>(wide, two);
    }
}

template <int D, int UM, int R>
static void launch_q(const InstView& v, bool mark, int blocks, cudaStream_t st) {
    const int threads = UM == 16 ? 256 : 128;
    if (mark) {
        pq_kernel<D, true, UM, R>();
        k_relax_pq<D, true, UM, R><<<blocks, threads, pq_smem<UM>(), st>>>(v);
    } else {
        pq_kernel<D, false, UM, R>();
        k_relax_pq<D, false, UM, R><<<blocks, threads, pq_smem<UM>(), st>>>(v);
    }
}

template <int D>
static void launch_qd(const InstView& v, bool mark, bool two, int blocks, cudaStream_t st) {
    if (v.g.U > 16) {
        if (two) launch_q<D, 32, 2>(v, mark, blocks, st);
        else launch_q<D, 32, 1>(v, mark, blocks, st);
    } else {
        if (two) launch_q<D, 16, 2>(v, mark, blocks, st);
        else launch_q<D, 16, 1>(v, mark, blocks, st);
    }
}

void launch_relax_queue(const InstView& v, bool mark, bool two, int blocks, cudaStream_t st) {
    switch (v.g.D) {
        case 2: launch_qd<2>(v, mark, two, blocks, st); break;
        case 3: launch_qd<3>(v, mark, two, blocks, st); break;
        default: launch_qd<4>(v, mark, two, blocks, st); break;
    }
}
