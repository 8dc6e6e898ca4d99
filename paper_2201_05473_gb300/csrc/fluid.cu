// Fused fluid kernel of one time step: the hot path of the method (the
// per-node body is in fluid_node.cuh).
//
// Memory traffic per node: 76 population reads + 76 writes (FP32: 608 B),
// E (one edge per component) + two B time levels (36 B) read, J (12 B)
// written; neighbouring edge/face reads hit L1/L2.
#include "lbm_kernels.h"
#include "fluid_node.cuh"

namespace pwfa {

namespace {

#ifndef PWFA_FLUID_MAX_THREADS
#define PWFA_FLUID_MAX_THREADS 256
#endif
#ifndef PWFA_FLUID_MIN_BLOCKS
#define PWFA_FLUID_MIN_BLOCKS 2
#endif

template <int ST, int COLL, bool PER>
__global__ void __launch_bounds__(PWFA_FLUID_MAX_THREADS, PWFA_FLUID_MIN_BLOCKS) fluid_kernel(const StepArgs a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.g.nx || y >= a.g.ny) return;
    fluid_node<ST, COLL, PER>(a, x, y, blockIdx.z);
}

template <int ST, int COLL>
cudaError_t launch_fluid_t(const StepArgs& a, cudaStream_t s) {
    const int bx = a.bx, by = a.by;
    if (bx * by > PWFA_FLUID_MAX_THREADS || bx <= 0 || by <= 0) return cudaErrorInvalidConfiguration;
    dim3 block(bx, by, 1);
    dim3 grid((a.g.nx + bx - 1) / bx, (a.g.ny + by - 1) / by, a.g.nz);
    if (a.g.periodic) fluid_kernel<ST, COLL, true><<<grid, block, 0, s>>>(a);
    else fluid_kernel<ST, COLL, false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

template <int ST>
cudaError_t launch_fluid_s(const StepArgs& a, int collision, cudaStream_t s) {
    switch (collision) {
        case 0: return launch_fluid_t<ST, 0>(a, s);
        case 1: return launch_fluid_t<ST, 1>(a, s);
        case 2: return launch_fluid_t<ST, 2>(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_fluid(const StepArgs& a, int storage, int collision, cudaStream_t s) {
    switch (storage) {
        case 0: return launch_fluid_s<0>(a, collision, s);
        case 1: return launch_fluid_s<1>(a, collision, s);
        case 2: return launch_fluid_s<2>(a, collision, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace pwfa
