// The fluid step of the adjoint's recompute: the fused fluid kernel of
// fluid.cu that also stores each node's lattice sums A_l for the reverse
// step (a translation unit of its own, so that the production kernels'
// build is unchanged).
#include "lbm_kernels.h"
#include "fluid_node.cuh"

namespace pwfa {

namespace {

template <int ST, int COLL, bool PER>
__global__ void __launch_bounds__(PWFA_FLUID_MAX_THREADS, FluidOcc<ST, COLL>::blocks) fluid_mom_kernel(const StepArgs a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.g.nx || y >= a.g.ny) return;
    fluid_node<ST, COLL, PER, false, true>(a, x, y, blockIdx.z);
}

template <int ST, int COLL>
cudaError_t launch_t(const StepArgs& a, cudaStream_t s) {
    const int bx = a.bx, by = a.by;
    if (bx * by > PWFA_FLUID_MAX_THREADS || bx <= 0 || by <= 0 || (bx * by) % 32 || !a.mom)
        return cudaErrorInvalidConfiguration;
    dim3 block(bx, by, 1);
    dim3 grid((a.g.nx + bx - 1) / bx, (a.g.ny + by - 1) / by, a.g.nz);
    if (a.g.periodic) fluid_mom_kernel<ST, COLL, true><<<grid, block, 0, s>>>(a);
    else fluid_mom_kernel<ST, COLL, false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

template <int ST>
cudaError_t launch_s(const StepArgs& a, int collision, cudaStream_t s) {
    switch (collision) {
        case 0: return launch_t<ST, 0>(a, s);
        case 1: return launch_t<ST, 1>(a, s);
        case 2: return launch_t<ST, 2>(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_fluid_mom(const StepArgs& a, int storage, int collision, cudaStream_t s) {
    switch (storage) {
        case 0: return launch_s<0>(a, collision, s);
        case 1: return launch_s<1>(a, collision, s);
        case 2: return launch_s<2>(a, collision, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace pwfa
