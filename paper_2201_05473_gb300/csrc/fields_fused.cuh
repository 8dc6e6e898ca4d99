// The fused field step: Ampere of step n with Faraday of step n + 1 over one
// tile, shared by the single-instance kernel (fields.cu) and the batched
// field phase (batch.cu). Bodies of the separate updates: fields_node.cuh.
#pragma once

#include "fields_node.cuh"

namespace pwfa {

// Ampere of step n fused with Faraday of step n+1 (rigid driver):
// E_{n+3/2} = E_{n+1/2} + (dt/dx) curl_h B_{n+1} - dt (J + J_b) into out.E
// (the other E buffer), then B_{n+2} = B_{n+1} - (dt/dx) curl_h E_{n+3/2}
// into out.B (the buffer of B_n, which no later kernel reads). B_{n+1} is
// read once for both, so the pair moves 60 B per node instead of 84.
//
// A block of 32 x kAFY threads owns a tile of 31 x (kAFY - 1) nodes and
// marches up kAFZ planes. Each thread evaluates E_{n+3/2} at its (x, y)
// column, plane by plane; the last lane and row are the +x / +y neighbours
// the tile's Faraday reads (evaluated again by their owner). Faraday of plane
// k - 1 runs once plane k is evaluated: the +x neighbour's E comes from the
// next lane by a shuffle, the +y neighbour's from shared memory (one barrier
// per plane, two buffers), the +z value from the thread's own registers. The
// march also keeps B_{n+1} of plane k - 1 (Ampere's -z neighbour) and J_z of
// plane k + 1 (the next plane's own value) in registers, and the column's
// neighbour offsets, wall masks and the driver's transverse factor are
// computed once: per plane a thread loads 15 values. The driver's
// longitudinal factor of plane kz0 + l is evaluated once per warp, by lane l,
// and each plane takes it by a shuffle. Open-grid neighbours
// below index 0 read the zero guard in front of each array; +1 neighbours
// are clamped into the grid (the conducting walls discard what they feed).
#ifndef PWFA_AF_Y
#define PWFA_AF_Y 8
#endif
#ifndef PWFA_AF_Z
#define PWFA_AF_Z 16
#endif
#ifndef PWFA_AF_MIN_BLOCKS
#define PWFA_AF_MIN_BLOCKS 4
#endif
#ifndef PWFA_AF_UNROLL
#define PWFA_AF_UNROLL 1
#endif
constexpr int kAFX = 32, kAFY = PWFA_AF_Y, kAFZ = PWFA_AF_Z, kAFUnroll = PWFA_AF_UNROLL;
// one lane per plane of a slab, the plane above it included
static_assert(kAFZ < kAFX, "the driver's per-plane factors are held one per lane");

// The 15 values a thread loads for one plane of its column.
struct AFPlane {
    float e0, e1, e2, bx, by, bz, bz_i, by_i, bz_j, bx_j, j0, j0_i, j1, j1_j, j2k;
};

template <bool PER>
__device__ __forceinline__ void af_load(const StepArgs& a, int o, int zp, int xm, int ym, int xp, int yp,
                                        AFPlane& v) {
    const float *Bx = a.Bn[0], *By = a.Bn[1], *Bz = a.Bn[2];
#ifdef PWFA_DEBUG
    // the extremes of the plane's reads: own index, the -y (lowest) and the
    // +y / +z (highest) neighbours
    o = PWFA_CHECK(a.dbg, o, 0, a.g.N, 6u);
    ym = PWFA_CHECK(a.dbg, o + ym, -guard_elems(a.g), a.g.N, 6u) - o;
    yp = PWFA_CHECK(a.dbg, o + yp, 0, a.g.N, 6u) - o;
    zp = PWFA_CHECK(a.dbg, o + zp, 0, a.g.N, 6u) - o;
#endif
    v.e0 = __ldg(a.E[0] + o);
    v.e1 = __ldg(a.E[1] + o);
    v.e2 = __ldg(a.E[2] + o);
    v.bx = __ldg(Bx + o);
    v.by = __ldg(By + o);
    v.bz = __ldg(Bz + o);
    v.bz_i = __ldg(Bz + o + xm);
    v.by_i = __ldg(By + o + xm);
    v.bz_j = __ldg(Bz + o + ym);
    v.bx_j = __ldg(Bx + o + ym);
    v.j0 = __ldg(a.J[0] + o);
    v.j0_i = __ldg(a.J[0] + o + xp);
    v.j1 = __ldg(a.J[1] + o);
    v.j1_j = __ldg(a.J[1] + o + yp);
    v.j2k = __ldg(a.J[2] + o + zp);
}

// The fused step over one tile (tile coordinates tbx, tby, tbz): called by
// the single-instance kernel (fields.cu) and the batched field phase
// (batch.cu) with blocks of kAFX x kAFY threads; zc is the driver centre at
// t_{n+1}.
template <bool PER>
__device__ __forceinline__ void ampere_faraday_tile(const StepArgs& a, const FieldPair& out, int tbx, int tby,
                                                    int tbz, float zc) {
    const Grid& g = a.g;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int nxy = nx * ny;
    __shared__ float sEz[2][kAFY][kAFX], sEx[2][kAFY][kAFX];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x = tbx * (kAFX - 1) + tx, y = tby * (kAFY - 1) + ty;
    const bool own = tx < kAFX - 1 && ty < kAFY - 1 && x < nx && y < ny;
    // the evaluated column: wrapped (periodic) or clamped into the grid (an
    // open grid's clamped halo columns feed only wall components)
    const int xe = PER ? x % nx : min(x, nx - 1);
    const int ye = PER ? y % ny : min(y, ny - 1);
    // neighbour offsets of the column (open: -1 neighbours read the guard
    // plane or a wall component, +1 neighbours are clamped)
    const int xm = PER && xe == 0 ? nx - 1 : -1;
    const int ym = PER && ye == 0 ? nxy - nx : -nx;
    const int xp = xe < nx - 1 ? 1 : (PER ? 1 - nx : 0);
    const int yp = ye < ny - 1 ? nx : (PER ? nx - nxy : 0);
    // wall masks of the column (the plane's part is added per plane)
    const bool mEx = PER || (xe <= nx - 2 && ye >= 1 && ye <= ny - 2);  // E_x and B_y
    const bool mEy = PER || (xe >= 1 && xe <= nx - 2 && ye <= ny - 2);  // E_y and B_x
    const bool mEz = PER || (xe >= 1 && xe <= nx - 2 && ye >= 1 && ye <= ny - 2);
    const bool mBz = PER || (xe <= nx - 2 && ye <= ny - 2);
    const float gT = a.alpha != 0.0f ? driver_transverse(a, xe, ye) : 0.0f;
    const float c = a.cdt, dt = a.dt;

    const int kz0 = tbz * kAFZ, kend = min(kz0 + kAFZ, nz);
    // lane l holds the longitudinal factor of plane kz0 + l (same function,
    // same arguments as everywhere else: the same value)
    const float glane = a.alpha != 0.0f && tx <= kAFZ ? driver_longitudinal(a, kz0 + tx, zc) : 0.0f;
    // plane offsets: o of plane k (wrapped on a periodic grid), zp its +z
    // neighbour offset (clamped on an open grid)
    // (k runs to kend <= nz: on a periodic grid plane nz is plane 0 again)
    auto wrapk = [&](int k) { return PER && k >= nz ? k - nz : k; };
    auto plane_o = [&](int k) { return (wrapk(k) * ny + ye) * nx + xe; };
    auto plane_zp = [&](int k) { return wrapk(k) < nz - 1 ? nxy : (PER ? -(nz - 1) * nxy : 0); };
    // carried from plane k - 1: own E_{n+3/2}, the +x and +y neighbours' E,
    // own B_{n+1}; J_z of plane k
    float ep0 = 0.0f, ep1 = 0.0f, ep2 = 0.0f, ezx = 0.0f, eyx = 0.0f, ezy = 0.0f, exy = 0.0f;
    float bp0, bp1, bp2 = 0.0f, j2n;
    int o = plane_o(kz0);
    {
        int zm = PER && kz0 == 0 ? (nz - 1) * nxy : -nxy;
#ifdef PWFA_DEBUG
        zm = PWFA_CHECK(a.dbg, o + zm, -guard_elems(g), g.N, 6u) - o;
#endif
        bp0 = __ldg(a.Bn[0] + o + zm);
        bp1 = __ldg(a.Bn[1] + o + zm);
        j2n = __ldg(a.J[2] + o);
    }
    // the loads of the first plane; each iteration issues the next plane's
    // before it works on its own
    AFPlane nxt;
    af_load<PER>(a, o, plane_zp(kz0), xm, ym, xp, yp, nxt);
    int oprev = o;
#pragma unroll kAFUnroll
    for (int k = kz0; k <= kend; ++k) {
        const int buf = (k - kz0) & 1;
        const bool valid = PER || k < nz;
        const AFPlane v = nxt;
        // plane_o(k + 1), one plane up from o (wrapped on a periodic grid)
        const int onext = PER && wrapk(k) + 1 >= nz ? o + nxy - nz * nxy : o + nxy;
        if (k < kend && (PER || k + 1 < nz)) af_load<PER>(a, onext, plane_zp(k + 1), xm, ym, xp, yp, nxt);
        float e0 = valid ? v.e0 : 0.0f, e1 = valid ? v.e1 : 0.0f, e2 = valid ? v.e2 : 0.0f;
        const float gl = __shfl_sync(0xffffffffu, glane, k - kz0);
        if (valid) {
            const bool kin = PER || (k >= 1 && k <= nz - 2), klo = PER || k <= nz - 2;
            if (mEx && kin) e0 = ampere_arith(c, dt, e0, v.bz - v.bz_j, v.by - bp1, 0.5f * (v.j0 + v.j0_i));
            if (mEy && kin) e1 = ampere_arith(c, dt, e1, v.bx - bp0, v.bz - v.bz_i, 0.5f * (v.j1 + v.j1_j));
            if (mEz && klo) {
                const float jb = a.alpha != 0.0f ? -(gT * gl) : 0.0f;
                e2 = ampere_arith(c, dt, e2, v.by - v.by_i, v.bx - v.bx_j, 0.5f * (j2n + v.j2k) + jb);
            }
            if (own && k < kend) {
#ifdef PWFA_DEBUG
                o = PWFA_CHECK(a.dbg, o, 0, g.N, 6u);
#endif
                out.E[0][o] = e0;
                out.E[1][o] = e1;
                out.E[2][o] = e2;
            }
        }
        // the +x neighbour's E_z, E_y of this plane (lane + 1) and, after
        // the barrier, the +y neighbour's E_z, E_x (row + 1)
        const float ezx_k = __shfl_down_sync(0xffffffffu, e2, 1);
        const float eyx_k = __shfl_down_sync(0xffffffffu, e1, 1);
        sEz[buf][ty][tx] = e2;
        sEx[buf][ty][tx] = e0;
        __syncthreads();
        if (k > kz0 && own) {
            // Faraday of plane k - 1 (B_{n+2} at the own index)
            const int kb = k - 1;
            const bool kbl = PER || kb <= nz - 2, kbi = PER || (kb >= 1 && kb <= nz - 2);
            const float bprev[3] = {bp0, bp1, bp2};
            float bn[3];
            faraday_arith(c, bprev, ep0, ep1, ep2, ezy, e1, e0, ezx, eyx, exy, mEy && kbl, mEx && kbl, mBz && kbi, bn);
#ifdef PWFA_DEBUG
            oprev = PWFA_CHECK(a.dbg, oprev, 0, g.N, 6u);
#endif
            out.B[0][oprev] = bn[0];
            out.B[1][oprev] = bn[1];
            out.B[2][oprev] = bn[2];
        }
        const int tyn = ty + 1 < kAFY ? ty + 1 : ty;
        ezy = sEz[buf][tyn][tx];
        exy = sEx[buf][tyn][tx];
        ezx = ezx_k;
        eyx = eyx_k;
        ep0 = e0;
        ep1 = e1;
        ep2 = e2;
        bp0 = v.bx;
        bp1 = v.by;
        bp2 = v.bz;
        j2n = v.j2k;
        oprev = o;
        o = onext;
    }
}


}  // namespace pwfa
