// Batched form: many independent instances of uneven grid sizes advanced
// together, one launch per phase for all of them, two steps replayed from a
// captured CUDA graph. Each phase is one grid over the concatenated tiles of
// every instance (per-node phases: groups of tiles of 128 consecutive nodes;
// fused field step: the z-marching tiles of fields_fused.cuh); a 16-bit
// table maps each block to its instance. The hardware block
// scheduler hands the tiles out in order, so the tiles in flight form one
// short window of the list and the z +- 1 planes a pull reads are still in
// L2. No block waits on another.
#include "lbm_batch.h"
#include "fields_fused.cuh"
#include "fluid_node.cuh"

namespace pwfa {

namespace {

static_assert(sizeof(StepArgs) % 4 == 0 && sizeof(StepArgs) / 4 <= kBatchTile, "StepArgs copy");
static_assert(sizeof(FieldPair) % 4 == 0 && sizeof(FieldPair) / 4 <= kBatchTile, "FieldPair copy");
// the parked BGK values take one shared-memory column per thread of a block
static_assert(kBatchTile <= PWFA_FLUID_MAX_THREADS, "BGK park columns");

// The block's instance arguments, copied once into shared memory (every
// thread reads them).
template <int NT>
__device__ __forceinline__ void copy_words(void* dst, const void* src, int bytes, int tid) {
    for (int w = tid; w < bytes / 4; w += NT) static_cast<int*>(dst)[w] = __ldg(static_cast<const int*>(src) + w);
}

// Node (x, y, z) of thread tid in fluid tile t of an instance: tiles are
// 128 consecutive nodes of the instance's [z][y][x] order (four 32-node
// chunks of the population layout), so no lane idles on a narrow grid; false
// past the instance's last node.
__device__ __forceinline__ bool tile_node(const Grid& g, int64_t t, int tid, int& x, int& y, int& z) {
    const uint32_t node = (uint32_t)t * (uint32_t)kBatchTile + (uint32_t)tid;
    if (node >= (uint32_t)g.N) return false;
    const uint32_t nx = (uint32_t)g.nx, nxy = nx * (uint32_t)g.ny;
    const uint32_t zz = node / nxy, r = node - zz * nxy, yy = r / nx;
    z = (int)zz;
    y = (int)yy;
    x = (int)(r - yy * nx);
    return true;
}

// Driver time of the instance's Ampere launch of this parity, and the
// counter of the other parity advanced by the instance's first tile.
__device__ __forceinline__ float driver_centre(const BatchEntry& e, int parity, bool first) {
    const int64_t n = e.step[parity];
    if (first) e.step[parity ^ 1] = n + 1;
    return (float)(e.z0 + (double)(n + 1) * e.dt);
}

// Phases 0-2 on the fluid tiles: Faraday, the fluid step, Ampere. A block
// takes kBatchGroup consecutive tiles of one instance.
template <int ST, int COLL, bool PER, int PHASE>
__global__ void __launch_bounds__(kBatchTile, PHASE == 1 ? BatchFluidOcc<ST, COLL>::blocks : 8)
    batch_node_kernel(const BatchEntry* __restrict__ ent, const uint16_t* __restrict__ tile_inst, int parity) {
    __shared__ StepArgs sa;
    __shared__ float s_zc;
    const int tid = threadIdx.x;
    const int inst = __ldg(tile_inst + blockIdx.x);
    const BatchEntry& e = ent[inst];
    copy_words<kBatchTile>(&sa, &e.args[parity], sizeof(StepArgs), tid);
    const int64_t t0 = ((int64_t)blockIdx.x - e.tile_begin) * kBatchGroup;
    if (PHASE == 2 && tid == 0) s_zc = driver_centre(e, parity, t0 == 0);
    __syncthreads();
    const int64_t t1 = t0 + kBatchGroup < e.ntiles ? t0 + kBatchGroup : e.ntiles;
    for (int64_t t = t0; t < t1; ++t) {
        int x, y, z;
        if (!tile_node(sa.g, t, tid, x, y, z)) continue;
        if (PHASE == 0) faraday_node<PER>(sa, x, y, z);
        else if (PHASE == 1) fluid_node<ST, COLL, PER, false, false, BatchFluidOcc<ST, COLL>::park>(sa, x, y, z);
        else ampere_node<PER>(sa, x, y, z, s_zc);
    }
}

// Phase 3 on the fused-field tiles: Ampere of this step with Faraday of the
// next.
template <bool PER>
__global__ void __launch_bounds__(kAFX * kAFY, PWFA_AF_MIN_BLOCKS)
    batch_fields_kernel(const BatchEntry* __restrict__ ent, const uint16_t* __restrict__ ftile_inst, int parity) {
    __shared__ StepArgs sa;
    __shared__ FieldPair so;
    __shared__ float s_zc;
    const int tid = threadIdx.y * kAFX + threadIdx.x;
    const int inst = __ldg(ftile_inst + blockIdx.x);
    const BatchEntry& e = ent[inst];
    copy_words<kAFX * kAFY>(&sa, &e.args[parity], sizeof(StepArgs), tid);
    copy_words<kAFX * kAFY>(&so, &e.out[parity], sizeof(FieldPair), tid);
    const int64_t local = (int64_t)blockIdx.x - e.ftile_begin;
    if (tid == 0) s_zc = driver_centre(e, parity, local == 0);
    __syncthreads();
    const int per_slab = e.ftiles_x * e.ftiles_y;
    const int tbz = (int)(local / per_slab);
    const int r = (int)(local - (int64_t)tbz * per_slab);
    const int tby = r / e.ftiles_x;
    ampere_faraday_tile<PER>(sa, so, r - tby * e.ftiles_x, tby, tbz, s_zc);
}

template <int ST, int COLL, bool PER>
cudaError_t launch_phase(const BatchLaunch& b, int phase, int parity, cudaStream_t s) {
    const unsigned nt = (unsigned)b.ntiles;
    switch (phase) {
        case 0: batch_node_kernel<ST, COLL, PER, 0><<<nt, kBatchTile, 0, s>>>(b.entries, b.tile_inst, parity); break;
        case 1: batch_node_kernel<ST, COLL, PER, 1><<<nt, kBatchTile, 0, s>>>(b.entries, b.tile_inst, parity); break;
        case 2: batch_node_kernel<ST, COLL, PER, 2><<<nt, kBatchTile, 0, s>>>(b.entries, b.tile_inst, parity); break;
        case 3:
            batch_fields_kernel<PER><<<(unsigned)b.nftiles, dim3(kAFX, kAFY, 1), 0, s>>>(b.entries, b.ftile_inst, parity);
            break;
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
    if (b.ntiles > INT32_MAX || b.nftiles > INT32_MAX) return cudaErrorInvalidConfiguration;
    switch (storage) {
        case 0: return launch_phase_c<0>(b, phase, parity, collision, periodic, s);
        case 1: return launch_phase_c<1>(b, phase, parity, collision, periodic, s);
        case 2: return launch_phase_c<2>(b, phase, parity, collision, periodic, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace pwfa
