// 2D-axisymmetric (z, r) form (internal; kernels in axi.cu, host side in
// axi_api.cu). Three D2Q9 lattices for A = (n, n p_z, n p_r) with the
// cylindrical terms of Eq. 13, and cylindrical Yee TM fields (E_z, E_r,
// B_theta).
//
// Grid: nodes (z_k, r_j), z_k = k dx, r_j = (j - 1/2) dx, node index
// k nr + j (r fastest). Row 0 is the mirror image of row 1 (the axis lies
// between them), rows 1..nr-2 hold the plasma, row nr-1 is the outer
// boundary row. E_z at (z_{k+1/2}, r_j), E_r at (z_k, j dx), B_theta at
// (z_{k+1/2}, j dx). Populations: [lattice][q][Np] planes (Np = N rounded up
// to 32), the stored post-collision values that the next step pulls.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pwfa {
namespace axi {

constexpr int kQ = 9;
constexpr int kL = 3;

struct Args {
    int nz, nr;
    int64_t N, Np;
    const float* fin;    // streaming source of this step
    float* fout;         // post-collision populations written by this step
    float* Am;           // [3][N] node moments (exports)
    const float* Ez;     // E_z, E_r at t_{n+1/2} (updated in place by Ampere)
    const float* Er;
    const float* Bt;     // B_theta at t_n
    float* Btn;          // B_theta at t_{n+1}
    float* EzO;
    float* ErO;
    float* Jz;           // node current of the step
    float* Jr;
    float omega;         // 1 / tau
    float lat;           // dt / dx
    float dt, cdt, dx;
    float D;             // physical diffusivity (tau - 1/2)/3 dx^2/dt (Eq. 12)
    float n_floor, n0;
    int couple, collision;  // collision: 0 BGK, 2 stream only
    float alpha, inv2sr2, inv2sz2, zc;  // driver at t_{n+1}
};

// a.Am := pre-collision node moments (for exports; the step's fluid kernel
// takes its neighbours' moments from adjacent lanes)
cudaError_t launch_moments(const Args& a, cudaStream_t s);
cudaError_t launch_fluid(const Args& a, cudaStream_t s);
cudaError_t launch_ampere(const Args& a, cudaStream_t s);
// plasma at rest: w_i n0 on lattice 0, zero on the momentum lattices
cudaError_t launch_init(const Args& a, float* f, cudaStream_t s);
// out[3][N] = n, beta_z, beta_r from the moments in a.Am
cudaError_t launch_export_moments(const Args& a, float* out, cudaStream_t s);

}  // namespace axi
}  // namespace pwfa
