// Adjoint kernels of one time step (internal; see adjoint.cu).
#pragma once

#include "lbm_kernels.h"

namespace pwfa {

// Driver-gradient accumulation slots: each warp of the Ampere adjoint adds
// its three partial sums to FP64 slot (warp % kGradSlots), which spreads the
// atomics over 3 kGradSlots addresses; the slots are summed into grad[0..2]
// once, after the sweep.
constexpr int kGradSlots = 1024;

struct AdjArgs {
    StepArgs f;           // forward state of the reversed step: fin = S^{n-1},
                          // E = E^n, Bc = B(t_n), Bn = B(t_{n+1}), driver at t_{n+1}
    const float* Sbar_in; // adjoint of the stored populations S^n, population layout (FP32)
    float* Sbar_out;      // adjoint of S^{n-1}, population layout (FP32)
    float* Ebar[3];       // in: adjoint of E^{n+1}; out: adjoint of E^n
    float* Bbar[3];       // in: adjoint of B(t_{n+1}); out: adjoint of B(t_n)
    float* Bnp[3];        // scratch: adjoint of Bn at faces
    float* Jbar[3];       // scratch: adjoint of the node current
    float* ebar[3];       // scratch: adjoint of the node-averaged E
    float* bbar[3];       // scratch: adjoint of the node-averaged B (each time level)
    float* Abnd[4];       // scratch: moment adjoints of Eq. 14 boundary nodes
    double* grad;         // d/d(alpha, sigma_r, sigma_z), then the profile gradient
    double* gslots;       // [kGradSlots][3] partial sums of d/d(alpha, sigma_r, sigma_z)
    float sr, sz;         // driver sigma_r, sigma_z
    float csr, csz;       // alpha / sigma_r^3, alpha / sigma_z^3 (set by the launchers)
};

// R1..R4 of one reversed step on stream s: R1 (launch_adjoint_ampere), R2a
// and R2 (launch_adjoint_fluid), R3 and R4 (launch_adjoint_fields: one fused
// kernel, or two separate ones when fused is false; the same results bit
// for bit), in that order.
cudaError_t launch_adjoint_ampere(const AdjArgs& a, cudaStream_t s);
cudaError_t launch_adjoint_fluid(const AdjArgs& a, int storage, int collision, cudaStream_t s);
cudaError_t launch_adjoint_fields(const AdjArgs& a, bool fused, cudaStream_t s);
cudaError_t launch_adjoint_step(const AdjArgs& a, int storage, int collision, cudaStream_t s);

// grad[0..2] = the sums of the driver-gradient slots.
cudaError_t launch_adjoint_grad_finish(const double* gslots, double* grad, cudaStream_t s);

// Profile gradient from the adjoint of the initial stored populations
// (lattice 0 block of Sbar, population layout); n_profile <= 256.
cudaError_t launch_adjoint_profile(const Grid& g, const float* Sbar, float n0, int n_profile, double rmax,
                                   double dx, double* grad_profile, cudaStream_t s);

}  // namespace pwfa
