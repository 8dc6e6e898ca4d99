// PIC driver (Eq. 1): macro-electrons pushed in E + beta x B and their
// current deposited on the Yee grid, in place of the rigid bunch.
//
// Positions live at t_{n+1/2} (the time level of E), momenta at t_n (that of
// B). One thread per particle: E(t_{n+1/2}) and the mean of B(t_n),
// B(t_{n+1}) interpolated trilinearly from each component's own Yee lattice
// at x_{n+1/2}; Boris push (charge/mass -1) to p_{n+1}; move to
// x_{n+3/2} = x_{n+1/2} + dt p_{n+1}/gamma; the current of the move added to
// J_b on the E edges by Esirkepov's charge-conserving scheme (Comput. Phys.
// Commun. 135, 2001) for the linear shape, with FP32 atomics. Particles
// outside an open grid see no field and deposit only on in-grid edges. Each
// block also grows the step's deposit box, so that Ampere's law reads (and
// clears) J_b only where particles deposited instead of over the whole grid.
#include "lbm_kernels.h"

namespace pwfa {

namespace {

__device__ __forceinline__ int wrapc(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// Yee value at (i, j, k): wrapped when periodic, zero outside an open grid
__device__ __forceinline__ float yv(const Grid& g, const float* a, int i, int j, int k) {
    if (g.periodic) {
        i = wrapc(i, g.nx); j = wrapc(j, g.ny); k = wrapc(k, g.nz);
    } else if (i < 0 || j < 0 || k < 0 || i >= g.nx || j >= g.ny || k >= g.nz) {
        return 0.0f;
    }
    return __ldg(a + ((int64_t)k * g.ny + j) * g.nx + i);
}

// component at grid coordinates of its own lattice, trilinear
__device__ __forceinline__ float interp(const Grid& g, const float* a, float gx, float gy, float gz) {
    const float fx0 = floorf(gx), fy0 = floorf(gy), fz0 = floorf(gz);
    const int i0 = (int)fx0, j0 = (int)fy0, k0 = (int)fz0;
    const float fx = gx - fx0, fy = gy - fy0, fz = gz - fz0;
    float r = 0.0f;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a2 = 0; a2 < 2; ++a2) {
                const float w = (a2 ? fx : 1.0f - fx) * (b ? fy : 1.0f - fy) * (c ? fz : 1.0f - fz);
                r += w * yv(g, a, i0 + a2, j0 + b, k0 + c);
            }
    return r;
}

__device__ __forceinline__ float hat(float t) {
    const float at = fabsf(t);
    return at < 1.0f ? 1.0f - at : 0.0f;
}

__device__ __forceinline__ void add_edge(const Grid& g, float* a, int i, int j, int k, float v) {
    if (g.periodic) {
        i = wrapc(i, g.nx); j = wrapc(j, g.ny); k = wrapc(k, g.nz);
    } else if (i < 0 || j < 0 || k < 0 || i >= g.nx || j >= g.ny || k >= g.nz) {
        return;
    }
    atomicAdd(a + ((int64_t)k * g.ny + j) * g.nx + i, v);
}

// Node box of the block's deposits, merged into a.jbox: per axis the 3-node
// stencil [base, base + 2] of every particle, clamped to the grid (the whole
// grid when periodic, where the stencil may wrap). Warp reductions, then
// shared-memory atomics, then six global atomics per block.
__device__ __forceinline__ void merge_box(const StepArgs& a, bool valid, const int base[3]) {
    __shared__ int sbox[6];
    if (threadIdx.x < 6) sbox[threadIdx.x] = threadIdx.x < 3 ? 0x7fffffff : -1;
    __syncthreads();
    const int n[3] = {a.g.nx, a.g.ny, a.g.nz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        int lo = 0x7fffffff, hi = -1;
        if (valid) {
            lo = a.g.periodic ? 0 : max(base[d], 0);
            hi = a.g.periodic ? n[d] - 1 : min(base[d] + 2, n[d] - 1);
        }
        lo = __reduce_min_sync(0xffffffffu, lo);
        hi = __reduce_max_sync(0xffffffffu, hi);
        if ((threadIdx.x & 31) == 0 && lo <= hi) {
            atomicMin(sbox + d, lo);
            atomicMax(sbox + 3 + d, hi);
        }
    }
    __syncthreads();
    if (threadIdx.x < 3 && sbox[threadIdx.x] <= sbox[3 + threadIdx.x]) {
        atomicMin(a.jbox + threadIdx.x, sbox[threadIdx.x]);
        atomicMax(a.jbox + 3 + threadIdx.x, sbox[3 + threadIdx.x]);
    }
}

// Particle m: push, move, deposit; base = the lower corner of its deposit
// stencil.
__device__ __forceinline__ void push_deposit(const StepArgs& a, float* xp, int64_t np, float coef, float* jx,
                                             float* jy, float* jz, int64_t m, int base[3]) {
    const Grid& g = a.g;
    float* px = xp;
    float* py = xp + np;
    float* pzp = xp + 2 * np;
    const float inv_dx = 1.0f / a.dx;
    const float g0[3] = {px[m] * inv_dx, py[m] * inv_dx, pzp[m] * inv_dx};
    const float e[3] = {interp(g, a.E[0], g0[0] - 0.5f, g0[1], g0[2]), interp(g, a.E[1], g0[0], g0[1] - 0.5f, g0[2]),
                        interp(g, a.E[2], g0[0], g0[1], g0[2] - 0.5f)};
    const float b[3] = {
        0.5f * (interp(g, a.Bc[0], g0[0], g0[1] - 0.5f, g0[2] - 0.5f) + interp(g, a.Bn[0], g0[0], g0[1] - 0.5f, g0[2] - 0.5f)),
        0.5f * (interp(g, a.Bc[1], g0[0] - 0.5f, g0[1], g0[2] - 0.5f) + interp(g, a.Bn[1], g0[0] - 0.5f, g0[1], g0[2] - 0.5f)),
        0.5f * (interp(g, a.Bc[2], g0[0] - 0.5f, g0[1] - 0.5f, g0[2]) + interp(g, a.Bn[2], g0[0] - 0.5f, g0[1] - 0.5f, g0[2]))};
    // Boris, q/m = -1: half kick, rotation, half kick
    const float hdt = 0.5f * a.dt;
    float um[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) um[c] = xp[(3 + c) * np + m] - hdt * e[c];
    const float gm = sqrtf(1.0f + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    float tv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) tv[c] = -hdt * b[c] / gm;
    const float t2 = tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2];
    float sv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) sv[c] = 2.0f * tv[c] / (1.0f + t2);
    const float w1[3] = {um[0] + (um[1] * tv[2] - um[2] * tv[1]), um[1] + (um[2] * tv[0] - um[0] * tv[2]),
                         um[2] + (um[0] * tv[1] - um[1] * tv[0])};
    float pn[3];
    pn[0] = um[0] + (w1[1] * sv[2] - w1[2] * sv[1]) - hdt * e[0];
    pn[1] = um[1] + (w1[2] * sv[0] - w1[0] * sv[2]) - hdt * e[1];
    pn[2] = um[2] + (w1[0] * sv[1] - w1[1] * sv[0]) - hdt * e[2];
    const float gn = sqrtf(1.0f + pn[0] * pn[0] + pn[1] * pn[1] + pn[2] * pn[2]);
    float xn[3], g1[3];
    const float pos[3] = {px[m], py[m], pzp[m]};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        xn[c] = pos[c] + a.dt * pn[c] / gn;
        g1[c] = xn[c] * inv_dx;
    }
    // Esirkepov deposit on a 3-node stencil per axis
    float s0[3][3], ds[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        base[d] = (int)floorf(fminf(g0[d], g1[d]));
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float node = (float)(base[d] + q);
            s0[d][q] = hat(g0[d] - node);
            ds[d][q] = hat(g1[d] - node) - s0[d][q];
        }
    }
    const float third = 1.0f / 3.0f;
#pragma unroll
    for (int bb = 0; bb < 3; ++bb)
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            float run = 0.0f;
#pragma unroll
            for (int aa = 0; aa < 2; ++aa) {
                run += ds[0][aa] * (s0[1][bb] * s0[2][cc] + 0.5f * ds[1][bb] * s0[2][cc] + 0.5f * s0[1][bb] * ds[2][cc] +
                                    third * ds[1][bb] * ds[2][cc]);
                if (run != 0.0f) add_edge(g, jx, base[0] + aa, base[1] + bb, base[2] + cc, coef * run);
            }
        }
#pragma unroll
    for (int aa = 0; aa < 3; ++aa)
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            float run = 0.0f;
#pragma unroll
            for (int bb = 0; bb < 2; ++bb) {
                run += ds[1][bb] * (s0[0][aa] * s0[2][cc] + 0.5f * ds[0][aa] * s0[2][cc] + 0.5f * s0[0][aa] * ds[2][cc] +
                                    third * ds[0][aa] * ds[2][cc]);
                if (run != 0.0f) add_edge(g, jy, base[0] + aa, base[1] + bb, base[2] + cc, coef * run);
            }
        }
#pragma unroll
    for (int aa = 0; aa < 3; ++aa)
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) {
            float run = 0.0f;
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                run += ds[2][cc] * (s0[0][aa] * s0[1][bb] + 0.5f * ds[0][aa] * s0[1][bb] + 0.5f * s0[0][aa] * ds[1][bb] +
                                    third * ds[0][aa] * ds[1][bb]);
                if (run != 0.0f) add_edge(g, jz, base[0] + aa, base[1] + bb, base[2] + cc, coef * run);
            }
        }
    // periodic grids keep the positions in the box
    const float L[3] = {g.nx * a.dx, g.ny * a.dx, g.nz * a.dx};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float v = xn[c];
        if (g.periodic) {
            if (v < 0.0f) v += L[c];
            else if (v >= L[c]) v -= L[c];
        }
        xp[c * np + m] = v;
        xp[(3 + c) * np + m] = pn[c];
    }
}

__global__ void __launch_bounds__(128) push_deposit_kernel(const StepArgs a, float* xp, int64_t np, float coef,
                                                           float* jx, float* jy, float* jz) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int base[3] = {0, 0, 0};
    const bool valid = m < np;
    if (valid) push_deposit(a, xp, np, coef, jx, jy, jz, m, base);
    if (a.jbox) merge_box(a, valid, base);
}

}  // namespace

cudaError_t launch_push_deposit(const StepArgs& a, float* xp, int64_t np, double weight, float* const Jb[3],
                                cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    const float coef = (float)(weight / ((double)a.dx * a.dx * a.dt));
    const unsigned blocks = (unsigned)((np + 127) / 128);
    push_deposit_kernel<<<blocks, 128, 0, s>>>(a, xp, np, coef, Jb[0], Jb[1], Jb[2]);
    return cudaGetLastError();
}

}  // namespace pwfa
