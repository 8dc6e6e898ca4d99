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

// Neighbour indices: wrapped by yee_ld on periodic grids, clamped into the
// grid on open ones (where the wall conditions then discard the result), so
// that every load of a node is issued before any of them is used. Loads
// inside the per-component wall branches had left one round trip to memory
// per branch in sequence.
template <bool PER>
__device__ __forceinline__ int up1(int i, int n) { return PER ? i + 1 : min(i + 1, n - 1); }
template <bool PER>
__device__ __forceinline__ int dn1(int i) { return PER ? i - 1 : max(i - 1, 0); }

// Bn = Bc - (dt/dx) curl_h E, curl at the face centres.
template <bool PER>
__device__ __forceinline__ void faraday_node(const StepArgs& a, int i, int j, int k) {
    const Grid& g = a.g;
    const int64_t o = ((int64_t)k * g.ny + j) * g.nx + i;
    const float c = a.cdt;
    const float *Ex = a.E[0], *Ey = a.E[1], *Ez = a.E[2];
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int ip = up1<PER>(i, nx), jp = up1<PER>(j, ny), kp = up1<PER>(k, nz);
    const float ex = yee_ld<PER>(g, Ex, i, j, k), ey = yee_ld<PER>(g, Ey, i, j, k), ez = yee_ld<PER>(g, Ez, i, j, k);
    const float ez_j = yee_ld<PER>(g, Ez, i, jp, k), ey_k = yee_ld<PER>(g, Ey, i, j, kp);
    const float ex_k = yee_ld<PER>(g, Ex, i, j, kp), ez_i = yee_ld<PER>(g, Ez, ip, j, k);
    const float ey_i = yee_ld<PER>(g, Ey, ip, j, k), ex_j = yee_ld<PER>(g, Ex, i, jp, k);
    const float b0 = __ldg(a.Bc[0] + o), b1 = __ldg(a.Bc[1] + o), b2 = __ldg(a.Bc[2] + o);
    const bool cx = PER || (i >= 1 && i <= nx - 2 && j <= ny - 2 && k <= nz - 2);
    const bool cy = PER || (i <= nx - 2 && j >= 1 && j <= ny - 2 && k <= nz - 2);
    const bool cz = PER || (i <= nx - 2 && j <= ny - 2 && k >= 1 && k <= nz - 2);
    a.Bn[0][o] = cx ? b0 - c * ((ez_j - ez) - (ey_k - ey)) : 0.0f;
    a.Bn[1][o] = cy ? b1 - c * ((ex_k - ex) - (ez_i - ez)) : 0.0f;
    a.Bn[2][o] = cz ? b2 - c * ((ey_i - ey) - (ex_j - ex)) : 0.0f;
}

// E += (dt/dx) curl_h Bn - dt (J_e,edge + J_b), J_e,edge the mean of the two
// node currents of the edge, J_b,z = -n_b of the rigid driver at t_{n+1}.
// Components on the walls of an open grid are left as they are (zero).
template <bool PER>
__device__ __forceinline__ void ampere_node(const StepArgs& a, int i, int j, int k, float zc) {
    const Grid& g = a.g;
    const int64_t o = ((int64_t)k * g.ny + j) * g.nx + i;
    const float c = a.cdt, dt = a.dt;
    const float *Bx = a.Bn[0], *By = a.Bn[1], *Bz = a.Bn[2];
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int im = dn1<PER>(i), jm = dn1<PER>(j), km = dn1<PER>(k);
    const int ip = up1<PER>(i, nx), jp = up1<PER>(j, ny), kp = up1<PER>(k, nz);
    const float bx = yee_ld<PER>(g, Bx, i, j, k), by = yee_ld<PER>(g, By, i, j, k), bz = yee_ld<PER>(g, Bz, i, j, k);
    const float bz_j = yee_ld<PER>(g, Bz, i, jm, k), by_k = yee_ld<PER>(g, By, i, j, km);
    const float bx_k = yee_ld<PER>(g, Bx, i, j, km), bz_i = yee_ld<PER>(g, Bz, im, j, k);
    const float by_i = yee_ld<PER>(g, By, im, j, k), bx_j = yee_ld<PER>(g, Bx, i, jm, k);
    const float j0 = yee_ld<PER>(g, a.J[0], i, j, k), j0_i = yee_ld<PER>(g, a.J[0], ip, j, k);
    const float j1 = yee_ld<PER>(g, a.J[1], i, j, k), j1_j = yee_ld<PER>(g, a.J[1], i, jp, k);
    const float j2 = yee_ld<PER>(g, a.J[2], i, j, k), j2_k = yee_ld<PER>(g, a.J[2], i, j, kp);
    const float e0 = a.Eout[0][o], e1 = a.Eout[1][o], e2 = a.Eout[2][o];
    // PIC deposit: read (and clear for the next step) only inside its box
    const bool inbox = a.Jb[0] && i >= a.jbox[0] && j >= a.jbox[1] && k >= a.jbox[2] && i <= a.jbox[3] &&
                       j <= a.jbox[4] && k <= a.jbox[5];
    const float jb0 = inbox ? a.Jb[0][o] : 0.0f, jb1 = inbox ? a.Jb[1][o] : 0.0f;
    const float jb2 = inbox ? a.Jb[2][o] : 0.0f;
    if (inbox) {
        a.Jb[0][o] = 0.0f;
        a.Jb[1][o] = 0.0f;
        a.Jb[2][o] = 0.0f;
    }
    const bool cx = PER || (i <= nx - 2 && j >= 1 && j <= ny - 2 && k >= 1 && k <= nz - 2);
    const bool cy = PER || (i >= 1 && i <= nx - 2 && j <= ny - 2 && k >= 1 && k <= nz - 2);
    const bool cz = PER || (i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2 && k <= nz - 2);
    if (cx) {
        float je = 0.5f * (j0 + j0_i);
        if (a.Jb[0]) je += jb0;
        a.Eout[0][o] = e0 + c * ((bz - bz_j) - (by - by_k)) - dt * je;
    }
    if (cy) {
        float je = 0.5f * (j1 + j1_j);
        if (a.Jb[1]) je += jb1;
        a.Eout[1][o] = e1 + c * ((bx - bx_k) - (bz - bz_i)) - dt * je;
    }
    if (cz) {
        const float je = 0.5f * (j2 + j2_k);
        float jb = 0.0f;
        if (a.Jb[2]) {
            jb = jb2;
        } else if (a.alpha != 0.0f) {
            const float xr = ((float)i - 0.5f * (float)(nx - 1)) * a.dx;
            const float yr = ((float)j - 0.5f * (float)(ny - 1)) * a.dx;
            const float zeta = ((float)k + 0.5f) * a.dx - zc;
            jb = -a.alpha * expf(-(xr * xr + yr * yr) * a.inv2sr2 - zeta * zeta * a.inv2sz2);
        }
        a.Eout[2][o] = e2 + c * ((by - by_i) - (bx - bx_j)) - dt * (je + jb);
    }
}

}  // namespace pwfa
