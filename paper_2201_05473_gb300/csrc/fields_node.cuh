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

// Faraday's arithmetic for the three B components stored at one index, given
// the E values it reads (own index and the +1 neighbours), the old B and
// which components are active: Bn = Bc - (dt/dx) curl_h E, zero on the walls.
// Every Faraday kernel goes through it, so they agree bit for bit.
__device__ __forceinline__ void faraday_arith(float c, const float (&b)[3], float ex, float ey, float ez, float ez_j,
                                              float ey_k, float ex_k, float ez_i, float ey_i, float ex_j, bool cx,
                                              bool cy, bool cz, float (&bn)[3]) {
    bn[0] = cx ? b[0] - c * ((ez_j - ez) - (ey_k - ey)) : 0.0f;
    bn[1] = cy ? b[1] - c * ((ex_k - ex) - (ez_i - ez)) : 0.0f;
    bn[2] = cz ? b[2] - c * ((ey_i - ey) - (ex_j - ex)) : 0.0f;
}

// Faraday's update of the three B components stored at node (i, j, k) from
// the E values it reads and the old B; B_x is active on the faces with
// 1 <= i <= nx-2, j <= ny-2, k <= nz-2 of an open grid (cyclically for B_y,
// B_z), every face of a periodic one.
template <bool PER>
__device__ __forceinline__ void faraday_values(const Grid& g, float c, int i, int j, int k, const float (&b)[3],
                                               float ex, float ey, float ez, float ez_j, float ey_k, float ex_k,
                                               float ez_i, float ey_i, float ex_j, float (&bn)[3]) {
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const bool cx = PER || (i >= 1 && i <= nx - 2 && j <= ny - 2 && k <= nz - 2);
    const bool cy = PER || (i <= nx - 2 && j >= 1 && j <= ny - 2 && k <= nz - 2);
    const bool cz = PER || (i <= nx - 2 && j <= ny - 2 && k >= 1 && k <= nz - 2);
    faraday_arith(c, b, ex, ey, ez, ez_j, ey_k, ex_k, ez_i, ey_i, ex_j, cx, cy, cz, bn);
}

// The rigid driver's density n_b = alpha exp(-r^2/(2 sigma_r^2))
// exp(-(z - zc)^2/(2 sigma_z^2)) at the E_z edge (i, j, k + 1/2), as the
// product of a transverse factor (alpha included) and a longitudinal one:
// the fused field kernel takes the first once per (x, y) column and the
// second once per plane, and every kernel that evaluates J_b = -n_b forms
// the same product.
__device__ __forceinline__ float driver_transverse(const StepArgs& a, int i, int j) {
    const float xr = ((float)i - 0.5f * (float)(a.g.nx - 1)) * a.dx;
    const float yr = ((float)j - 0.5f * (float)(a.g.ny - 1)) * a.dx;
    return a.alpha * expf(-(xr * xr + yr * yr) * a.inv2sr2);
}
__device__ __forceinline__ float driver_longitudinal(const StepArgs& a, int k, float zc) {
    const float zeta = ((float)k + 0.5f) * a.dx - zc;
    return expf(-zeta * zeta * a.inv2sz2);
}

// Ampere's arithmetic for one E component: e + (dt/dx) (curl_h B) - dt j,
// the curl given as its two differences.
__device__ __forceinline__ float ampere_arith(float c, float dt, float e, float d1, float d2, float j) {
    return e + c * (d1 - d2) - dt * j;
}

// Bn = Bc - (dt/dx) curl_h E, curl at the face centres.
template <bool PER>
__device__ __forceinline__ void faraday_node(const StepArgs& a, int i, int j, int k) {
    const Grid& g = a.g;
    const int64_t o = PWFA_CHECK(a.dbg, ((int64_t)k * g.ny + j) * g.nx + i, 0, g.N, 4u);
    const float *Ex = a.E[0], *Ey = a.E[1], *Ez = a.E[2];
    // +1 neighbours: wrapped (periodic) or clamped into the grid as offsets
    int64_t pi, pj, pk;
    if (PER) {
        pi = wrapi(i + 1, g.nx) - i;
        pj = (int64_t)(wrapi(j + 1, g.ny) - j) * g.nx;
        pk = (int64_t)(wrapi(k + 1, g.nz) - k) * g.nx * g.ny;
    } else {
        pi = i < g.nx - 1 ? 1 : 0;
        pj = j < g.ny - 1 ? (int64_t)g.nx : 0;
        pk = k < g.nz - 1 ? (int64_t)g.nx * g.ny : 0;
    }
#ifdef PWFA_DEBUG
    pi = PWFA_CHECK(a.dbg, o + pi, 0, g.N, 4u) - o;
    pj = PWFA_CHECK(a.dbg, o + pj, 0, g.N, 4u) - o;
    pk = PWFA_CHECK(a.dbg, o + pk, 0, g.N, 4u) - o;
#endif
    const float ex = __ldg(Ex + o), ey = __ldg(Ey + o), ez = __ldg(Ez + o);
    const float ez_j = __ldg(Ez + o + pj), ey_k = __ldg(Ey + o + pk);
    const float ex_k = __ldg(Ex + o + pk), ez_i = __ldg(Ez + o + pi);
    const float ey_i = __ldg(Ey + o + pi), ex_j = __ldg(Ex + o + pj);
    const float b[3] = {__ldg(a.Bc[0] + o), __ldg(a.Bc[1] + o), __ldg(a.Bc[2] + o)};
    float bn[3];
    faraday_values<PER>(g, a.cdt, i, j, k, b, ex, ey, ez, ez_j, ey_k, ex_k, ez_i, ey_i, ex_j, bn);
    a.Bn[0][o] = bn[0];
    a.Bn[1][o] = bn[1];
    a.Bn[2][o] = bn[2];
}

// Ampere's update of the three E components stored at node (i, j, k):
// E += (dt/dx) curl_h Bn - dt (J_e,edge + J_b), J_e,edge the mean of the two
// node currents of the edge, J_b the PIC deposit jb (when a.Jb is set) or
// J_b,z = -n_b of the rigid driver at t_{n+1}. Split into the node's loads
// (AmpereIn) and the arithmetic (ampere_compute: en holds the new values, act
// which components are active; the others, on the walls of an open grid,
// keep their value, zero), shared by the plain and the fused kernels.
struct AmpereIn {
    float bx, by, bz, bz_j, by_k, bx_k, bz_i, by_i, bx_j, j0, j0_i, j1, j1_j, j2, j2_k, e0, e1, e2;
};

template <bool PER>
__device__ __forceinline__ AmpereIn ampere_loads(const StepArgs& a, int i, int j, int k) {
    const Grid& g = a.g;
    const int64_t o = PWFA_CHECK(a.dbg, ((int64_t)k * g.ny + j) * g.nx + i, 0, g.N, 5u);
    const float *Bx = a.Bn[0], *By = a.Bn[1], *Bz = a.Bn[2];
    AmpereIn v;
    if (PER) {
        const int im = dn1<PER>(i), jm = dn1<PER>(j), km = dn1<PER>(k);
        const int ip = up1<PER>(i, g.nx), jp = up1<PER>(j, g.ny), kp = up1<PER>(k, g.nz);
        v.bz_j = yee_ld<PER>(g, Bz, i, jm, k);
        v.by_k = yee_ld<PER>(g, By, i, j, km);
        v.bx_k = yee_ld<PER>(g, Bx, i, j, km);
        v.bz_i = yee_ld<PER>(g, Bz, im, j, k);
        v.by_i = yee_ld<PER>(g, By, im, j, k);
        v.bx_j = yee_ld<PER>(g, Bx, i, jm, k);
        v.j0_i = yee_ld<PER>(g, a.J[0], ip, j, k);
        v.j1_j = yee_ld<PER>(g, a.J[1], i, jp, k);
        v.j2_k = yee_ld<PER>(g, a.J[2], i, j, kp);
    } else {
        // neighbours clamped into the grid as index offsets from o
        const int64_t sx = g.nx, sxy = (int64_t)g.nx * g.ny;
        int64_t di = i > 0 ? 1 : 0, dj = j > 0 ? sx : 0, dk = k > 0 ? sxy : 0;
        int64_t ui = i < g.nx - 1 ? 1 : 0, uj = j < g.ny - 1 ? sx : 0, uk = k < g.nz - 1 ? sxy : 0;
#ifdef PWFA_DEBUG
        dk = o - PWFA_CHECK(a.dbg, o - dk, 0, g.N, 5u);
        uk = PWFA_CHECK(a.dbg, o + uk, 0, g.N, 5u) - o;
        (void)di; (void)dj; (void)ui; (void)uj;
#endif
        v.bz_j = __ldg(Bz + o - dj);
        v.by_k = __ldg(By + o - dk);
        v.bx_k = __ldg(Bx + o - dk);
        v.bz_i = __ldg(Bz + o - di);
        v.by_i = __ldg(By + o - di);
        v.bx_j = __ldg(Bx + o - dj);
        v.j0_i = __ldg(a.J[0] + o + ui);
        v.j1_j = __ldg(a.J[1] + o + uj);
        v.j2_k = __ldg(a.J[2] + o + uk);
    }
    v.bx = __ldg(Bx + o);
    v.by = __ldg(By + o);
    v.bz = __ldg(Bz + o);
    v.j0 = __ldg(a.J[0] + o);
    v.j1 = __ldg(a.J[1] + o);
    v.j2 = __ldg(a.J[2] + o);
    v.e0 = a.E[0][o];
    v.e1 = a.E[1][o];
    v.e2 = a.E[2][o];
    return v;
}

template <bool PER>
__device__ __forceinline__ void ampere_compute(const StepArgs& a, int i, int j, int k, float zc, const AmpereIn& v,
                                               const float (&jbv)[3], float (&en)[3], bool (&act)[3]) {
    const float c = a.cdt, dt = a.dt;
    const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
    act[0] = PER || (i <= nx - 2 && j >= 1 && j <= ny - 2 && k >= 1 && k <= nz - 2);
    act[1] = PER || (i >= 1 && i <= nx - 2 && j <= ny - 2 && k >= 1 && k <= nz - 2);
    act[2] = PER || (i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2 && k <= nz - 2);
    en[0] = v.e0;
    en[1] = v.e1;
    en[2] = v.e2;
    if (act[0]) {
        float je = 0.5f * (v.j0 + v.j0_i);
        if (a.Jb[0]) je += jbv[0];
        en[0] = ampere_arith(c, dt, v.e0, v.bz - v.bz_j, v.by - v.by_k, je);
    }
    if (act[1]) {
        float je = 0.5f * (v.j1 + v.j1_j);
        if (a.Jb[1]) je += jbv[1];
        en[1] = ampere_arith(c, dt, v.e1, v.bx - v.bx_k, v.bz - v.bz_i, je);
    }
    if (act[2]) {
        const float je = 0.5f * (v.j2 + v.j2_k);
        float jb = 0.0f;
        if (a.Jb[2]) jb = jbv[2];
        else if (a.alpha != 0.0f) jb = -(driver_transverse(a, i, j) * driver_longitudinal(a, k, zc));
        en[2] = ampere_arith(c, dt, v.e2, v.by - v.by_i, v.bx - v.bx_j, je + jb);
    }
}

// Ampere at node (i, j, k) from a.E into a.Eout (in place when they are the
// same arrays); the PIC deposit is read (and cleared for the next step) only
// inside its box.
template <bool PER>
__device__ __forceinline__ void ampere_node(const StepArgs& a, int i, int j, int k, float zc) {
    const Grid& g = a.g;
    const int64_t o = ((int64_t)k * g.ny + j) * g.nx + i;
    const bool inbox = a.Jb[0] && i >= a.jbox[0] && j >= a.jbox[1] && k >= a.jbox[2] && i <= a.jbox[3] &&
                       j <= a.jbox[4] && k <= a.jbox[5];
    const float jbv[3] = {inbox ? a.Jb[0][o] : 0.0f, inbox ? a.Jb[1][o] : 0.0f, inbox ? a.Jb[2][o] : 0.0f};
    const AmpereIn v = ampere_loads<PER>(a, i, j, k);
    float en[3];
    bool act[3];
    ampere_compute<PER>(a, i, j, k, zc, v, jbv, en, act);
    // in place (a.Eout = a.E) only the active components change; out of place
    // every component is written (the inactive ones keep their value)
#pragma unroll
    for (int c = 0; c < 3; ++c)
        if (act[c] || a.Eout[c] != a.E[c]) a.Eout[c][o] = en[c];
    if (inbox) {
        a.Jb[0][o] = 0.0f;
        a.Jb[1][o] = 0.0f;
        a.Jb[2][o] = 0.0f;
    }
}

}  // namespace pwfa
