// Batched form: many independent instances of uneven grid sizes advanced by
// one persistent launch per phase (Faraday, fused fluid, Ampere) over a
// flattened work list of (instance, tile) items, replayed from a captured
// CUDA graph. Each tile is 128 nodes of one z-plane in the instance's
// autotuned shape (bx x by, bx * by = 128). CTAs stride over the items
// (item = blockIdx.x, blockIdx.x + gridDim.x, ...): no inter-CTA waits.
#include "lbm_batch.h"
#include "fields_node.cuh"
#include "fluid_node.cuh"

namespace pwfa {

namespace {

constexpr int kThreads = kBatchTile;

// Copy one item's arguments into shared memory (all threads of the CTA work
// on the same item).
__device__ __forceinline__ void load_args(const BatchEntry& e, int parity, StepArgs& sa) {
    const int nwords = (int)(sizeof(StepArgs) / sizeof(int));
    const int* src = reinterpret_cast<const int*>(&e.args[parity]);
    int* dst = reinterpret_cast<int*>(&sa);
    for (int w = threadIdx.x; w < nwords; w += blockDim.x) dst[w] = src[w];
}

__device__ __forceinline__ int find_instance(const BatchEntry* ent, int ninst, int64_t item) {
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ent[mid].item_begin <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int ST, int COLL, bool PER, int PHASE>
__global__ void __launch_bounds__(kThreads, 4) batch_kernel(const BatchEntry* __restrict__ ent, int ninst,
                                                             int64_t nitems, int parity) {
    __shared__ StepArgs sa;
    __shared__ int s_inst;
    for (int64_t item = blockIdx.x; item < nitems; item += gridDim.x) {
        if (threadIdx.x == 0) s_inst = find_instance(ent, ninst, item);
        __syncthreads();
        const BatchEntry& e = ent[s_inst];
        load_args(e, parity, sa);
        __syncthreads();
        if (PHASE == 2) {
            if (threadIdx.x == 0) sa.zc = (float)(e.z0 + (double)(*e.step + 1) * e.dt);
            __syncthreads();
        }
        const int64_t local = item - e.item_begin;
        const int per_plane = e.tiles_x * e.tiles_y;
        const int z = (int)(local / per_plane);
        const int r = (int)(local - (int64_t)z * per_plane);
        const int ty = r / e.tiles_x;
        const int tx = r - ty * e.tiles_x;
        const int x = tx * e.bx + (int)threadIdx.x % e.bx;
        const int y = ty * e.by + (int)threadIdx.x / e.bx;
        if (x < sa.g.nx && y < sa.g.ny) {
            if (PHASE == 0) faraday_node<PER>(sa, x, y, z);
            else if (PHASE == 1) fluid_node<ST, COLL, PER>(sa, x, y, z);
            else ampere_node<PER>(sa, x, y, z);
        }
        __syncthreads();
    }
}

__global__ void batch_advance_kernel(const BatchEntry* ent, int ninst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ninst) *ent[i].step += 1;
}

template <int ST, int COLL, bool PER>
cudaError_t launch_phase(const BatchLaunch& b, int phase, int parity, cudaStream_t s) {
    switch (phase) {
        case 0: batch_kernel<ST, COLL, PER, 0><<<b.grid, kThreads, 0, s>>>(b.entries, b.ninst, b.nitems, parity); break;
        case 1: batch_kernel<ST, COLL, PER, 1><<<b.grid, kThreads, 0, s>>>(b.entries, b.ninst, b.nitems, parity); break;
        case 2: batch_kernel<ST, COLL, PER, 2><<<b.grid, kThreads, 0, s>>>(b.entries, b.ninst, b.nitems, parity); break;
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
