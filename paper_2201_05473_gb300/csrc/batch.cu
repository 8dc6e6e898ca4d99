// Batched form: many independent instances of uneven grid sizes advanced by
// one persistent launch per phase (Faraday, fused fluid, Ampere) over a
// flattened work list of (instance, tile) items, replayed from a captured
// CUDA graph. Each tile is 128 nodes of one z-plane in the instance's
// autotuned shape (bx x by, bx * by = 128). No inter-CTA waits.
#include "lbm_batch.h"
#include "lbm_kernels.h"
#include "fields_node.cuh"
#include "fluid_node.cuh"

namespace pwfa {

namespace {

constexpr int kThreads = kBatchTile;

// The instance table lives in constant memory: every thread of a CTA reads
// the same entry (broadcast), so no shared-memory copy and no barrier is
// needed anywhere in the kernel.
__constant__ BatchEntry c_entries[kMaxBatch];
static_assert(sizeof(BatchEntry) * kMaxBatch <= 60 * 1024, "instance table exceeds constant memory");

// Resident blocks per SM: the fluid phase as the single-instance fluid
// kernel (FluidOcc: 96 or 128 registers); the light field phases run 8
// blocks (64 registers).
template <int PHASE, int COLL>
struct PhaseOcc {
    static constexpr int blocks = PHASE == 1 ? FluidOcc<COLL>::blocks : 8;
};

// Work items are handed out in order by a global counter (one atomic per
// grab, prefetched one grab ahead), so the items in flight always form one
// short window of the work list, as with a hardware-scheduled grid: the
// planes pulled across (z - 1, z + 1) are still in L2 when their neighbours
// run, however unevenly the CTAs progress. Items only grow within a CTA, so
// each CTA walks the instance table forward. The fluid phase grabs one item
// at a time; the light field phases grab kFieldGrab consecutive items.
constexpr int kFieldGrab = 4;

template <int ST, int COLL, bool PER, int PHASE>
__global__ void __launch_bounds__(kThreads, PhaseOcc<PHASE, COLL>::blocks) batch_kernel(int ninst, int nitems,
                                                                                  int parity, int* counter) {
    constexpr int grab = PHASE == 1 ? 1 : kFieldGrab;
    __shared__ int s_next[2];
    if (threadIdx.x == 0) s_next[0] = atomicAdd(counter, grab);
    __syncthreads();
    // only the instance range is carried between items; the tile shape is
    // re-read from the (broadcast) constant table to keep registers free
    int inst = -1, begin = 0, end = 0;
    float zc = 0.0f;
    for (int buf = 0;; buf ^= 1) {
        const int first = s_next[buf];
        if (first >= nitems) break;
        if (threadIdx.x == 0) s_next[buf ^ 1] = atomicAdd(counter, grab);
        const int last = first + grab < nitems ? first + grab : nitems;
        for (int item = first; item < last; ++item) {
            if (item >= end) {
                do {
                    ++inst;
                    begin = (int)c_entries[inst].item_begin;
                    end = inst + 1 < ninst ? (int)c_entries[inst + 1].item_begin : nitems;
                } while (item >= end);
                if (PHASE == 2)
                    zc = (float)(c_entries[inst].z0 + (double)(*c_entries[inst].step + 1) * c_entries[inst].dt);
            }
            const BatchEntry& e = c_entries[inst];
            const int local = item - begin;
            const int per_plane = e.tiles_x * e.tiles_y;
            const int z = local / per_plane;
            const int r = local - z * per_plane;
            const int ty = r / e.tiles_x;
            const int bx = e.bx;
            const int x = (r - ty * e.tiles_x) * bx + (int)threadIdx.x % bx;
            const int y = ty * (kThreads / bx) + (int)threadIdx.x / bx;
            const StepArgs& a = c_entries[inst].args[parity];
            if (x < a.g.nx && y < a.g.ny) {
                if (PHASE == 0) faraday_node<PER>(a, x, y, z);
                else if (PHASE == 1) fluid_node<ST, COLL, PER>(a, x, y, z);
                else ampere_node<PER>(a, x, y, z, zc);
            }
        }
        // every thread has read s_next[buf]; the next grab is visible
        __syncthreads();
    }
}

// Advance the step counters and re-arm the phases' work counters.
__global__ void batch_advance_kernel(const BatchEntry* ent, int ninst, int* counters) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ninst) *ent[i].step += 1;
    if (i < kBatchCounters) counters[i] = 0;
}

template <int ST, int COLL, bool PER>
cudaError_t launch_phase(const BatchLaunch& b, int phase, int parity, cudaStream_t s) {
    const int g1 = b.grid;                                     // fluid phase
    const int gf = b.grid / PhaseOcc<1, COLL>::blocks * PhaseOcc<0, COLL>::blocks;  // field phases
    switch (phase) {
        case 0: batch_kernel<ST, COLL, PER, 0><<<gf, kThreads, 0, s>>>(b.ninst, (int)b.nitems, parity, b.counters); break;
        case 1: batch_kernel<ST, COLL, PER, 1><<<g1, kThreads, 0, s>>>(b.ninst, (int)b.nitems, parity, b.counters + 1); break;
        case 2: batch_kernel<ST, COLL, PER, 2><<<gf, kThreads, 0, s>>>(b.ninst, (int)b.nitems, parity, b.counters + 2); break;
        case 3: batch_advance_kernel<<<(b.ninst + 127) / 128, 128, 0, s>>>(b.entries, b.ninst, b.counters); break;
        default: return cudaErrorInvalidValue;
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
