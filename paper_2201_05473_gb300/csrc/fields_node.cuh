// Per-node bodies of the Yee FDTD field updates (Eq. 5 in normalised units,
// Faraday with Maxwell's sign): dB/dt = -curl E, dE/dt = curl B - J. One
// thread per node updates the three components stored at that node's index.
// Shared by the single-instance kernels (fields.cu) and the batched kernels
// (batch.cu).
//
// Staggering: E_x (i+1/2, j, k), E_y (i, j+1/2, k), E_z (i, j, k+1/2);
// B_x (i, j+1/2, k+1/2), B_y (i+1/2, j, k+1/2), B_z (i+1/2, j+1/2, k).
// Open grids are closed by perfectly conducting walls: tangential E and
// normal B on the six outer planes (and components outside the grid) stay 0.
#pragma once

#include "lbm_device.cuh"

namespace pwfa {

template <bool PER>
__device__ __forceinline__ float yee_ld(const Grid& g, const float* a, int i, int j, int k) {
    if (PER) { i = wrapi(i, g.nx); j = wrapi(j, g.ny); k = wrapi(k, g.nz); }
    return __ldg(a + ((int64_t)k * g.ny + j) * g.nx + i);
}

// Bn = Bc - (dt/dx) curl_h E, curl at the face centres.
template <bool PER>
__device__ __forceinline__ void faraday_node(const StepArgs& a, int i, int j, int k) {
    const Grid& g = a.g;
    const int64_t o = ((int64_t)k * g.ny + j) * g.nx + i;
    const float c = a.cdt;
    const float *Ex = a.E[0], *Ey = a.E[1], *Ez = a.E[2];
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    float bx = 0.0f, by = 0.0f, bz = 0.0f;
    if (PER || (i >= 1 && i <= nx - 2 && j <= ny - 2 && k <= nz - 2)) {
        const float ez0 = yee_ld<PER>(g, Ez, i, j, k), ez1 = yee_ld<PER>(g, Ez, i, j + 1, k);
        const float ey0 = yee_ld<PER>(g, Ey, i, j, k), ey1 = yee_ld<PER>(g, Ey, i, j, k + 1);
        bx = __ldg(a.Bc[0] + o) - c * ((ez1 - ez0) - (ey1 - ey0));
    }
    if (PER || (i <= nx - 2 && j >= 1 && j <= ny - 2 && k <= nz - 2)) {
        const float ex0 = yee_ld<PER>(g, Ex, i, j, k), ex1 = yee_ld<PER>(g, Ex, i, j, k + 1);
        const float ez0 = yee_ld<PER>(g, Ez, i, j, k), ez1 = yee_ld<PER>(g, Ez, i + 1, j, k);
        by = __ldg(a.Bc[1] + o) - c * ((ex1 - ex0) - (ez1 - ez0));
    }
    if (PER || (i <= nx - 2 && j <= ny - 2 && k >= 1 && k <= nz - 2)) {
        const float ey0 = yee_ld<PER>(g, Ey, i, j, k), ey1 = yee_ld<PER>(g, Ey, i + 1, j, k);
        const float ex0 = yee_ld<PER>(g, Ex, i, j, k), ex1 = yee_ld<PER>(g, Ex, i, j + 1, k);
        bz = __ldg(a.Bc[2] + o) - c * ((ey1 - ey0) - (ex1 - ex0));
    }
    a.Bn[0][o] = bx;
    a.Bn[1][o] = by;
    a.Bn[2][o] = bz;
}

// E += (dt/dx) curl_h Bn - dt (J_e,edge + J_b), J_e,edge the mean of the two
// node currents of the edge, J_b,z = -n_b of the rigid driver at t_{n+1}.
template <bool PER>
__device__ __forceinline__ void ampere_node(const StepArgs& a, int i, int j, int k, float zc) {
    const Grid& g = a.g;
    const int64_t o = ((int64_t)k * g.ny + j) * g.nx + i;
    const float c = a.cdt, dt = a.dt;
    const float *Bx = a.Bn[0], *By = a.Bn[1], *Bz = a.Bn[2];
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    if (PER || (i <= nx - 2 && j >= 1 && j <= ny - 2 && k >= 1 && k <= nz - 2)) {
        const float curl = (yee_ld<PER>(g, Bz, i, j, k) - yee_ld<PER>(g, Bz, i, j - 1, k))
                         - (yee_ld<PER>(g, By, i, j, k) - yee_ld<PER>(g, By, i, j, k - 1));
        float je = 0.5f * (yee_ld<PER>(g, a.J[0], i, j, k) + yee_ld<PER>(g, a.J[0], i + 1, j, k));
        if (a.Jb[0]) je += a.Jb[0][o];
        a.Eout[0][o] = a.Eout[0][o] + c * curl - dt * je;
    }
    if (PER || (i >= 1 && i <= nx - 2 && j <= ny - 2 && k >= 1 && k <= nz - 2)) {
        const float curl = (yee_ld<PER>(g, Bx, i, j, k) - yee_ld<PER>(g, Bx, i, j, k - 1))
                         - (yee_ld<PER>(g, Bz, i, j, k) - yee_ld<PER>(g, Bz, i - 1, j, k));
        float je = 0.5f * (yee_ld<PER>(g, a.J[1], i, j, k) + yee_ld<PER>(g, a.J[1], i, j + 1, k));
        if (a.Jb[1]) je += a.Jb[1][o];
        a.Eout[1][o] = a.Eout[1][o] + c * curl - dt * je;
    }
    if (PER || (i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2 && k <= nz - 2)) {
        const float curl = (yee_ld<PER>(g, By, i, j, k) - yee_ld<PER>(g, By, i - 1, j, k))
                         - (yee_ld<PER>(g, Bx, i, j, k) - yee_ld<PER>(g, Bx, i, j - 1, k));
        const float je = 0.5f * (yee_ld<PER>(g, a.J[2], i, j, k) + yee_ld<PER>(g, a.J[2], i, j, k + 1));
        float jb = 0.0f;
        if (a.Jb[2]) {
            jb = a.Jb[2][o];
        } else if (a.alpha != 0.0f) {
            const float xr = ((float)i - 0.5f * (float)(nx - 1)) * a.dx;
            const float yr = ((float)j - 0.5f * (float)(ny - 1)) * a.dx;
            const float zeta = ((float)k + 0.5f) * a.dx - zc;
            jb = -a.alpha * expf(-(xr * xr + yr * yr) * a.inv2sr2 - zeta * zeta * a.inv2sz2);
        }
        a.Eout[2][o] = a.Eout[2][o] + c * curl - dt * (je + jb);
    }
}

}  // namespace pwfa
