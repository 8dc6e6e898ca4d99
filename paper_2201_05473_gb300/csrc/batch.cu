// Batched form: many independent instances of uneven grid sizes advanced by
// one persistent launch per phase (Faraday, fused fluid, Ampere) over a
// flattened work list of (instance, tile) items, replayed from a captured
// CUDA graph. Each tile is 128 nodes of one z-plane in the instance's
// autotuned shape (bx x by, bx * by = 128). CTAs take the items
// in contiguous chunks: no inter-CTA waits.
#include "lbm_batch.h"
#include "fields_node.cuh"
#include "fluid_node.cuh"

namespace pwfa {

namespace {

constexpr int kThreads = kBatchTile;

__device__ __forceinline__ int find_instance(const BatchEntry* ent, int ninst, int64_t item) {
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ent[mid].item_begin <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The instance table lives in constant memory: every thread of a CTA reads
// the same entry (broadcast), so no shared-memory copy and no barrier is
// needed anywhere in the kernel.
__constant__ BatchEntry c_entries[kMaxBatch];

// Resident blocks per SM: the fluid phase needs up to 128 registers (4 blocks
// of 128 threads); the light field phases run 8 blocks (64 registers).
template <int PHASE>
struct PhaseOcc {
    static constexpr int blocks = PHASE == 1 ? 4 : 8;
};

// Each CTA owns one contiguous chunk of the work list, so it crosses an
// instance boundary at most a few times; consecutive items of the same
// instance run back to back.
template <int ST, int COLL, bool PER, int PHASE>
__global__ void __launch_bounds__(kThreads, PhaseOcc<PHASE>::blocks) batch_kernel(int ninst, int64_t nitems,
                                                                                  int parity) {
    const int64_t per = (nitems + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * per;
    const int64_t i1 = i0 + per < nitems ? i0 + per : nitems;
    int inst = 0;
    int64_t end = 0;  // end of the current instance's items
    int tiles_x = 1, tiles_y = 1, bx = 1, by = 1, lx = 0, ly = 0;
    int tx = 0, ty = 0, z = 0;  // tile coordinates of the current item
    float zc = 0.0f;
    for (int64_t item = i0; item < i1; ++item) {
        if (item >= end) {
            // entering an instance: decode the item once (divisions only here)
            inst = find_instance(c_entries, ninst, item);
            const BatchEntry& e = c_entries[inst];
            end = inst + 1 < ninst ? c_entries[inst + 1].item_begin : nitems;
            tiles_x = e.tiles_x;
            tiles_y = e.tiles_y;
            bx = e.bx;
            by = kThreads / bx;
            lx = (int)threadIdx.x % bx;
            ly = (int)threadIdx.x / bx;
            const int64_t local = item - e.item_begin;
            const int64_t per_plane = (int64_t)tiles_x * tiles_y;
            z = (int)(local / per_plane);
            const int r = (int)(local - (int64_t)z * per_plane);
            ty = r / tiles_x;
            tx = r - ty * tiles_x;
            if (PHASE == 2) zc = (float)(e.z0 + (double)(*e.step + 1) * e.dt);
        }
        const StepArgs& a = c_entries[inst].args[parity];
        const int x = tx * bx + lx;
        const int y = ty * by + ly;
        if (x < a.g.nx && y < a.g.ny) {
            if (PHASE == 0) faraday_node<PER>(a, x, y, z);
            else if (PHASE == 1) fluid_node<ST, COLL, PER>(a, x, y, z);
            else ampere_node<PER>(a, x, y, z, zc);
        }
        // next item of the same instance: x tiles fastest, then y, then z
        if (++tx == tiles_x) {
            tx = 0;
            if (++ty == tiles_y) { ty = 0; ++z; }
        }
    }
}

__global__ void batch_advance_kernel(const BatchEntry* ent, int ninst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ninst) *ent[i].step += 1;
}

template <int ST, int COLL, bool PER>
cudaError_t launch_phase(const BatchLaunch& b, int phase, int parity, cudaStream_t s) {
    const int g1 = b.grid;                                     // fluid phase
    const int gf = b.grid / PhaseOcc<1>::blocks * PhaseOcc<0>::blocks;  // field phases
    switch (phase) {
        case 0: batch_kernel<ST, COLL, PER, 0><<<gf, kThreads, 0, s>>>(b.ninst, b.nitems, parity); break;
        case 1: batch_kernel<ST, COLL, PER, 1><<<g1, kThreads, 0, s>>>(b.ninst, b.nitems, parity); break;
        case 2: batch_kernel<ST, COLL, PER, 2><<<gf, kThreads, 0, s>>>(b.ninst, b.nitems, parity); break;
        default: batch_advance_kernel<<<(b.ninst + 127) / 128, 128, 0, s>>>(b.entries, b.ninst); break;
    }
    return cudaGetLastError();
}

template <int ST, int COLL>
cudaError_t launch_phase_p(const BatchLaunch& b, int phase, int parity, bool periodic, cudaStream_t s) {
    return periodic ? launch_phase<ST, COLL, true>(b, phase, parity, s)
                    : launch_phase<ST, COLL, false>(b, phase, parity, s);
}

template <int ST>
cudaError_t launch_phase_c(const BatchLaunch& b, int phase, int parity, int coll, bool periodic, cudaStream_t s) {
    switch (coll) {
        case 0: return launch_phase_p<ST, 0>(b, phase, parity, periodic, s);
        case 1: return launch_phase_p<ST, 1>(b, phase, parity, periodic, s);
        case 2: return launch_phase_p<ST, 2>(b, phase, parity, periodic, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_batch_phase(const BatchLaunch& b, int phase, int parity, int storage, int collision,
                               bool periodic, cudaStream_t s) {
    switch (storage) {
        case 0: return launch_phase_c<0>(b, phase, parity, collision, periodic, s);
        case 1: return launch_phase_c<1>(b, phase, parity, collision, periodic, s);
        case 2: return launch_phase_c<2>(b, phase, parity, collision, periodic, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t batch_upload_table(const BatchEntry* host, int n, cudaStream_t s) {
    if (n > kMaxBatch) return cudaErrorInvalidValue;
    return cudaMemcpyToSymbolAsync(c_entries, host, sizeof(BatchEntry) * n, 0, cudaMemcpyHostToDevice, s);
}

cudaError_t batch_grid_size(int storage, int collision, bool periodic, int* grid) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // occupancy of the heaviest phase (the fluid kernel) sets the persistent grid
    const void* fn = nullptr;
#define PWFA_BATCH_FN(ST_, C_)                                                          \
    fn = periodic ? (const void*)batch_kernel<ST_, C_, true, 1> : (const void*)batch_kernel<ST_, C_, false, 1>
    if (storage == 0) { if (collision == 0) PWFA_BATCH_FN(0, 0); else if (collision == 1) PWFA_BATCH_FN(0, 1); else PWFA_BATCH_FN(0, 2); }
    else if (storage == 1) { if (collision == 0) PWFA_BATCH_FN(1, 0); else if (collision == 1) PWFA_BATCH_FN(1, 1); else PWFA_BATCH_FN(1, 2); }
    else { if (collision == 0) PWFA_BATCH_FN(2, 0); else if (collision == 1) PWFA_BATCH_FN(2, 1); else PWFA_BATCH_FN(2, 2); }
#undef PWFA_BATCH_FN
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0);
    if (e != cudaSuccess) return e;
    *grid = sms * (per_sm > 0 ? per_sm : 1);
    return cudaSuccess;
}

}  // namespace pwfa
