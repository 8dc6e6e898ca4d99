// Per-node device functions shared by the step, export and diagnostics
// kernels: pull gather (Eq. 6), moments (Eq. 8 first line + Eq. 2), the
// shared equilibrium factors of Eq. 9 and the node-averaged Yee fields.
#pragma once

#include "lbm_device.cuh"

namespace pwfa {

template <bool PER>
__device__ __forceinline__ int64_t src_index(const Grid& g, int x, int y, int z, int q) {
    int sx = x - xi_x(q), sy = y - xi_y(q), sz = z - xi_z(q);
    if (PER) { sx = wrapi(sx, g.nx); sy = wrapi(sy, g.ny); sz = wrapi(sz, g.nz); }
    return ((int64_t)sz * g.ny + sy) * g.nx + sx;
}

// Pull the 76 populations f^n(x) = f*(x - xi_i) of node (x,y,z). Open grids
// gather at the clamped interior node instead and flag the node as a boundary
// node: its state is then f^eq of those moments (Eq. 14). Each lattice's
// block of 19 Np elements is addressed with 32-bit offsets (the host limits
// the grid so that 19 Np < 2^32). src_shift (open grids) moves every source
// node by that many nodes: nx*ny pulls from one plane up, which is how a
// moving-window step reads the moved streaming source (the plane above the
// box holds fresh plasma).
// RAW (16-bit storage): the values are left in stored units (the
// deviation, scaled for FP16) for a caller that works in those units.
template <int ST, bool PER, bool RAW = false>
__device__ __forceinline__ void gather(const Grid& g, const typename Codec<ST>::T* __restrict__ fin,
                                       float n0, int x, int y, int z, float f[kL][kQ], bool& bnd,
                                       uint32_t src_shift = 0, unsigned* dbg = nullptr) {
    using T = typename Codec<ST>::T;
    int xs = x, ys = y, zs = z;
    bnd = false;
    if (!PER) {
        xs = min(max(x, 1), g.nx - 2);
        ys = min(max(y, 1), g.ny - 2);
        zs = min(max(z, 1), g.nz - 2);
        bnd = (xs != x) | (ys != y) | (zs != z);
    }
    const int64_t LS = lattice_stride(g);
    // per-lattice (FP32) or per-pair (16-bit) base pointers; 32-bit offsets
    const T* __restrict__ fl[kL] = {fin, fin + LS, fin + 2 * LS, fin + 3 * LS};
    const T* __restrict__ fp[2] = {fin, fin + 2 * LS};
    const uint32_t sxy = (uint32_t)g.nx * (uint32_t)g.ny;
    const uint32_t nodec =
        ((uint32_t)zs * (uint32_t)g.ny + (uint32_t)ys) * (uint32_t)g.nx + (uint32_t)xs + (PER ? 0u : src_shift);
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        uint32_t src;
        if (PER) {
            src = (uint32_t)src_index<true>(g, xs, ys, zs, q);
        } else {
            const int d = xi_x(q) + xi_y(q) * g.nx;
            src = nodec - (uint32_t)d - (uint32_t)(xi_z(q)) * sxy;
        }
        src = PWFA_CHECK(dbg, src, 0, g.Np, 1u);
        const uint32_t off = pop_off(q, src);
        if constexpr (ST == 0) {
#pragma unroll
            for (int l = 0; l < kL; ++l) f[l][q] = Codec<ST>::load(fl[l] + off, l, q, n0);
        } else if constexpr (RAW) {
            Codec<ST>::load2raw(fp[0] + 2 * off, f[0][q], f[1][q]);
            Codec<ST>::load2raw(fp[1] + 2 * off, f[2][q], f[3][q]);
        } else {
            Codec<ST>::load2(fp[0] + 2 * off, 0, q, n0, f[0][q], f[1][q]);
            Codec<ST>::load2(fp[1] + 2 * off, 2, q, n0, f[2][q], f[3][q]);
        }
    }
}

// From the lattice sums A_l: the reciprocal inn of the floored density and
// beta = p / sqrt(1 + p^2), p = A_{1..3} / max(n, n_floor). One division and
// one reciprocal square root per node (six IEEE divisions and a square root
// were ~5 % of the fluid kernel's instructions).
__device__ __forceinline__ void node_velocity(const float A[kL], float n_floor, float& inn, float beta[3]) {
    inn = 1.0f / (A[0] > n_floor ? A[0] : n_floor);
    const float p0 = A[1] * inn, p1 = A[2] * inn, p2 = A[3] * inn;
    const float ig = rsqrtf(1.0f + p0 * p0 + p1 * p1 + p2 * p2);
    beta[0] = p0 * ig;
    beta[1] = p1 * ig;
    beta[2] = p2 * ig;
}

// Lattice sums A_l of the pulled values, then node_velocity.
__device__ __forceinline__ void node_moments(const float f[kL][kQ], float n_floor, float A[kL],
                                             float& inn, float beta[3]) {
#pragma unroll
    for (int l = 0; l < kL; ++l) {
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < kQ; ++q) s += f[l][q];
        A[l] = s;
    }
    node_velocity(A, n_floor, inn, beta);
}

// phi_i = w_i (1 + 3 xi.u + 4.5 (xi.u)^2 - 1.5 u.u): f^eq_{l,i} = A_l phi_i,
// shared by the four lattices (one advecting velocity, Eq. 4).
// WEIGHTED = false leaves out the weight: phi_i / w_i.
template <bool WEIGHTED = true>
__device__ __forceinline__ void eq_factors(const float u[3], float phi[kQ]) {
    const float base = 1.0f - 1.5f * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        const float xu = (float)xi_x(q) * u[0] + (float)xi_y(q) * u[1] + (float)xi_z(q) * u[2];
        const float b = base + 3.0f * xu + 4.5f * xu * xu;
        phi[q] = WEIGHTED ? wq(q) * b : b;
    }
}

// E at node (x,y,z): mean of its two edges per component. B: mean over the
// four adjacent faces of the two time levels Bc (t_n) and Bn (t_{n+1}).
template <bool PER>
__device__ __forceinline__ float yat(const Grid& g, const float* a, int i, int j, int k) {
    if (PER) {
        i = wrapi(i, g.nx); j = wrapi(j, g.ny); k = wrapi(k, g.nz);
    } else if (i < 0 || j < 0 || k < 0) {
        return 0.0f;
    }
    return __ldg(a + ((int64_t)k * g.ny + j) * g.nx + i);
}

// Open grids keep a zero guard in front of every Yee array (one plane, one
// row and one element) and every component outside the conducting box at
// zero, so the indices just below the grid (x-1, y-1, z-1 and their
// combinations, wrapping into the previous row/plane or the guard) read 0.
template <bool PER>
__device__ __forceinline__ void node_E(const Grid& g, const float* const E[3], int x, int y, int z, float e[3],
                                       unsigned* dbg = nullptr) {
    if (PER) {
        e[0] = 0.5f * (yat<PER>(g, E[0], x - 1, y, z) + yat<PER>(g, E[0], x, y, z));
        e[1] = 0.5f * (yat<PER>(g, E[1], x, y - 1, z) + yat<PER>(g, E[1], x, y, z));
        e[2] = 0.5f * (yat<PER>(g, E[2], x, y, z - 1) + yat<PER>(g, E[2], x, y, z));
    } else {
        const int64_t o = PWFA_CHECK(dbg, ((int64_t)z * g.ny + y) * g.nx + x, 0, g.N, 3u);
        const int64_t sxy = (int64_t)g.nx * g.ny;
#ifdef PWFA_DEBUG
        PWFA_CHECK(dbg, o - sxy, -guard_elems(g), g.N, 3u);
#endif
        e[0] = 0.5f * (__ldg(E[0] + o - 1) + __ldg(E[0] + o));
        e[1] = 0.5f * (__ldg(E[1] + o - g.nx) + __ldg(E[1] + o));
        e[2] = 0.5f * (__ldg(E[2] + o - sxy) + __ldg(E[2] + o));
    }
}

// Sum over the four faces around the node for one B array.
template <bool PER>
__device__ __forceinline__ void node_B_sum(const Grid& g, const float* const B[3], int x, int y, int z, float b[3],
                                           unsigned* dbg = nullptr) {
    if (PER) {
        b[0] = yat<PER>(g, B[0], x, y, z) + yat<PER>(g, B[0], x, y - 1, z) + yat<PER>(g, B[0], x, y, z - 1)
             + yat<PER>(g, B[0], x, y - 1, z - 1);
        b[1] = yat<PER>(g, B[1], x, y, z) + yat<PER>(g, B[1], x - 1, y, z) + yat<PER>(g, B[1], x, y, z - 1)
             + yat<PER>(g, B[1], x - 1, y, z - 1);
        b[2] = yat<PER>(g, B[2], x, y, z) + yat<PER>(g, B[2], x - 1, y, z) + yat<PER>(g, B[2], x, y - 1, z)
             + yat<PER>(g, B[2], x - 1, y - 1, z);
    } else {
        const int64_t o = PWFA_CHECK(dbg, ((int64_t)z * g.ny + y) * g.nx + x, 0, g.N, 3u);
        const int64_t sx = g.nx, sxy = (int64_t)g.nx * g.ny;
#ifdef PWFA_DEBUG
        // the lowest index read: the -y, -z corner of B_x
        PWFA_CHECK(dbg, o - sx - sxy, -guard_elems(g), g.N, 3u);
#endif
        const float* b0 = B[0] + o;
        const float* b1 = B[1] + o;
        const float* b2 = B[2] + o;
        b[0] = __ldg(b0) + __ldg(b0 - sx) + __ldg(b0 - sxy) + __ldg(b0 - sx - sxy);
        b[1] = __ldg(b1) + __ldg(b1 - 1) + __ldg(b1 - sxy) + __ldg(b1 - 1 - sxy);
        b[2] = __ldg(b2) + __ldg(b2 - 1) + __ldg(b2 - sx) + __ldg(b2 - 1 - sx);
    }
}

}  // namespace pwfa
