// Kernels of the 2D-axisymmetric (z, r) form: the fused step (Faraday's law,
// pull, node moments, the cylindrical terms of Eq. 13, collision), Ampere
// with the driver, and the node moments for exports. One thread per node,
// warps along r (coalesced rows).
#include "axi.h"

namespace pwfa {
namespace axi {

namespace {

constexpr int kBR = 32;  // threads along r
constexpr int kBZ = 4;   // threads along z

// D2Q9 in (z, r) components: rest, +z, -z, +r, -r, (+z,+r), (-z,-r), (+z,-r), (-z,+r)
__host__ __device__ constexpr int xz(int q) {
    return (q == 1 || q == 5 || q == 7) ? 1 : ((q == 2 || q == 6 || q == 8) ? -1 : 0);
}
__host__ __device__ constexpr int xr(int q) {
    return (q == 3 || q == 5 || q == 8) ? 1 : ((q == 4 || q == 6 || q == 7) ? -1 : 0);
}
__host__ __device__ constexpr float w9(int q) { return q == 0 ? 4.0f / 9.0f : (q <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f); }
// the direction with the r component reversed
__host__ __device__ constexpr int rrefl(int q) {
    return q == 3 ? 4 : (q == 4 ? 3 : (q == 5 ? 7 : (q == 7 ? 5 : (q == 6 ? 8 : (q == 8 ? 6 : q)))));
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// f^eq of Eq. 9 in lattice units (c_s^2 = 1/3)
__device__ __forceinline__ float feq(int q, float A, float uz, float ur) {
    const float xu = (float)xz(q) * uz + (float)xr(q) * ur;
    return w9(q) * A * (1.0f + 3.0f * xu + 4.5f * xu * xu - 1.5f * (uz * uz + ur * ur));
}

__device__ __forceinline__ float yee(const float* a, const Args& g, int k, int j) {
    if (k < 0 || j < 0 || k >= g.nz || j >= g.nr) return 0.0f;
    return a[(int64_t)k * g.nr + j];
}

// Faraday on one face: B_theta(t_{n+1}) = B_theta(t_n) + dt (dE_z/dr - dE_r/dz)
// on the active faces, zero elsewhere (axis, outer wall, outside the grid)
__device__ __forceinline__ float faraday_bt(const Args& a, int k, int j) {
    if (k < 0 || k > a.nz - 2 || j < 1 || j > a.nr - 2) return 0.0f;
    const int64_t o = (int64_t)k * a.nr + j;
    return a.Bt[o] - a.cdt * ((a.Er[o + a.nr] - a.Er[o]) - (a.Ez[o + 1] - a.Ez[o]));
}


// Pre-collision moments of every node: interior nodes sum their pulled
// populations; the z walls and the outer row take their clamped interior
// node's moments (their state is its equilibrium, Eq. 14); the axis row
// mirrors row 1 (n p_r changes sign).
__global__ void __launch_bounds__(kBR * kBZ) moments_kernel(const Args a) {
    const int j = blockIdx.x * kBR + threadIdx.x;
    const int k = blockIdx.y * kBZ + threadIdx.y;
    if (j >= a.nr || k >= a.nz) return;
    const int kc = clampi(k, 1, a.nz - 2);
    const int jc = clampi(j, 1, a.nr - 2);
    const int64_t base = (int64_t)kc * a.nr + jc;
    float A[kL];
#pragma unroll
    for (int l = 0; l < kL; ++l) {
        const float* fl = a.fin + (int64_t)l * kQ * a.Np;
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < kQ; ++q) s += __ldg(fl + (int64_t)q * a.Np + base - (int64_t)xz(q) * a.nr - xr(q));
        A[l] = s;
    }
    if (j == 0) A[2] = -A[2];
    const int64_t o = (int64_t)k * a.nr + j;
#pragma unroll
    for (int l = 0; l < kL; ++l) a.Am[(int64_t)l * a.N + o] = A[l];
}

// One fused step of every node of rows 1..nr-1. A warp takes 30 consecutive
// nodes of one z row plus a halo node on each side (lanes 0 and 31); every
// lane gathers the pulled populations of its clamped node (its own node when
// interior; the clamped interior node for the z walls, the outer row and the
// mirror row, which negates n p_r), so the radial neighbours' moments of
// dA/dr come from the neighbouring lanes (warp shuffles) without a separate
// moments pass. Faraday's law runs here too: each node evaluates B_theta at
// t_{n+1} on the four faces around it and stores the one it owns (rows
// 1..nr-1; the axis row's B_theta stays zero). Then: the equilibrium of the
// clamped node on boundary nodes (Eq. 14), Lorentz source with the node
// fields, the cylindrical terms
// D (1/r) dA/dr - A u_r / r of Eq. 13 on interior nodes, BGK collision
// (Eq. 7) with S_i = w_i S dt, store; row 1 also writes the axis row as its
// mirror image. Node current J = -n* beta(p*) of the post-collision moments.
constexpr int kOut = 30;  // output nodes per warp

// Seven blocks of 128 threads per SM (a 72-register budget, no spills): the
// kernel waits on its loads, and 28 resident warps instead of 24 (80
// registers) cut it from 0.064 to 0.054 ms on the 2400 x 402 grid.
#ifndef PWFA_AXI_MIN_BLOCKS
#define PWFA_AXI_MIN_BLOCKS 7
#endif
__global__ void __launch_bounds__(kBR * kBZ, PWFA_AXI_MIN_BLOCKS) fluid_kernel(const Args a) {
    const int lane = (int)threadIdx.x;
    const int j = (int)blockIdx.x * kOut + lane - 1;
    const int k = (int)(blockIdx.y * kBZ + threadIdx.y);
    const bool row_ok = k < a.nz;
    const bool valid = row_ok && j >= 0 && j < a.nr;
    const bool out = valid && lane >= 1 && lane <= kOut && j >= 1;
    const int kc = clampi(k, 1, a.nz - 2);
    const int jc = clampi(j, 1, a.nr - 2);
    const bool bnd = k == 0 || k == a.nz - 1 || j == a.nr - 1;
    float f[kL][kQ];
    float A[kL] = {0.0f, 0.0f, 0.0f};
    if (valid) {
        const int64_t c = (int64_t)kc * a.nr + jc;
#pragma unroll
        for (int l = 0; l < kL; ++l) {
            const float* fl = a.fin + (int64_t)l * kQ * a.Np;
            float s = 0.0f;
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                f[l][q] = __ldg(fl + (int64_t)q * a.Np + c - (int64_t)xz(q) * a.nr - xr(q));
                s += f[l][q];
            }
            A[l] = s;
        }
        if (j == 0) A[2] = -A[2];
    }
    // radial neighbours' moments (pre-collision, every node's own rule)
    float Am1[kL], Ap1[kL];
#pragma unroll
    for (int l = 0; l < kL; ++l) {
        Am1[l] = __shfl_up_sync(0xffffffffu, A[l], 1);
        Ap1[l] = __shfl_down_sync(0xffffffffu, A[l], 1);
    }
    if (!out) return;
    const int64_t o = (int64_t)k * a.nr + j;
    // one division and one reciprocal square root (p = A_k / n, beta = p / gamma)
    const float inn = 1.0f / (A[0] > a.n_floor ? A[0] : a.n_floor);
    const float pz = A[1] * inn, pr = A[2] * inn;
    const float ig = rsqrtf(1.0f + pz * pz + pr * pr);
    const float bz = pz * ig, br = pr * ig;
    const float uz = bz * a.lat, ur = br * a.lat;
    // equilibrium factors shared by the three lattices: f^eq_l,i = A_l phi_i
    float phi[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) phi[q] = feq(q, 1.0f, uz, ur);
    if (bnd) {
        // Eq. 14: the equilibrium of the clamped node
#pragma unroll
        for (int l = 0; l < kL; ++l)
#pragma unroll
            for (int q = 0; q < kQ; ++q) f[l][q] = A[l] * phi[q];
#pragma unroll
        for (int l = 0; l < kL; ++l) {
            float s = 0.0f;
#pragma unroll
            for (int q = 0; q < kQ; ++q) s += f[l][q];
            A[l] = s;
        }
    }
    float S[kL] = {0.0f, 0.0f, 0.0f};
    float nst = A[0], pzs = A[1], prs = A[2];  // post-collision moments
    if (a.collision != 2) {
        if (a.couple) {
            // node fields: E_z of its two z edges, E_r of its two r edges,
            // B_theta over the four surrounding faces of both time levels
            const float ez = 0.5f * (yee(a.Ez, a, k - 1, j) + yee(a.Ez, a, k, j));
            const float er = 0.5f * (yee(a.Er, a, k, j - 1) + yee(a.Er, a, k, j));
            float bs = 0.0f;
#pragma unroll
            for (int dk = -1; dk <= 0; ++dk)
#pragma unroll
                for (int dj = -1; dj <= 0; ++dj) bs += yee(a.Bt, a, k + dk, j + dj) + faraday_bt(a, k + dk, j + dj);
            const float bt = bs * 0.125f;
            // F_z = -n (E_z + beta_r B_theta), F_r = -n (E_r - beta_z B_theta)
            S[1] = -A[0] * (ez + br * bt);
            S[2] = -A[0] * (er - bz * bt);
        }
        if (!bnd) {
            // D (1/r) dA/dr - A u_r / r, dA/dr = (A(r + dx) - A(r - dx)) / 2 dx
            const float inv_r = 1.0f / (((float)j - 0.5f) * a.dx);
            const float c = 0.5f * a.D / a.dx;
#pragma unroll
            for (int l = 0; l < kL; ++l) S[l] += (c * (Ap1[l] - Am1[l]) - A[l] * br) * inv_r;
        }
        nst = A[0] + S[0] * a.dt;
        pzs = A[1] + S[1] * a.dt;
        prs = A[2] + S[2] * a.dt;
    }
    // collide and store (row 1 also writes its mirror image into the axis row)
    const int64_t om = (int64_t)k * a.nr;  // axis row node of this column
    const float omc = 1.0f - a.omega;
#pragma unroll
    for (int l = 0; l < kL; ++l) {
        float* fo = a.fout + (int64_t)l * kQ * a.Np;
        const float sg = l == 2 ? -1.0f : 1.0f;
        // f* = (1 - omega) f + omega A phi_i + w_i S dt, the weights applied
        // once per lattice
        const float oA = a.omega * A[l], sdt = S[l] * a.dt;
        const float sw[3] = {sdt * w9(0), sdt * w9(1), sdt * w9(5)};
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            float fs = f[l][q];
            if (a.collision != 2) fs = fmaf(fs, omc, fmaf(oA, phi[q], sw[q == 0 ? 0 : (q <= 4 ? 1 : 2)]));
            fo[(int64_t)q * a.Np + o] = fs;
            if (j == 1) fo[(int64_t)rrefl(q) * a.Np + om] = sg * fs;
        }
    }
    const float insn = 1.0f / (nst > a.n_floor ? nst : a.n_floor);
    const float qz = pzs * insn, qr = prs * insn;
    const float ngs = -nst * rsqrtf(1.0f + qz * qz + qr * qr);
    const float jz = ngs * qz, jr = ngs * qr;
    if (a.couple) a.Btn[o] = faraday_bt(a, k, j);
    a.Jz[o] = jz;
    a.Jr[o] = jr;
    if (j == 1) {
        a.Jz[om] = jz;
        a.Jr[om] = -jr;
    }
}

// Ampere: dE_r/dt = -dB_theta/dz - J_r, dE_z/dt = (1/r) d(r B_theta)/dr - J_z - J_b
__global__ void __launch_bounds__(kBR * kBZ) ampere_kernel(const Args a) {
    const int j = blockIdx.x * kBR + threadIdx.x;
    const int k = blockIdx.y * kBZ + threadIdx.y;
    if (j >= a.nr || k >= a.nz) return;
    const int64_t o = (int64_t)k * a.nr + j;
    if (k >= 1 && k <= a.nz - 2 && j >= 1 && j <= a.nr - 2) {
        const float je = 0.5f * (a.Jr[o] + a.Jr[o + 1]);
        a.ErO[o] = a.ErO[o] - a.cdt * (a.Btn[o] - a.Btn[o - a.nr]) - a.dt * je;
    }
    if (k <= a.nz - 2 && j >= 1 && j <= a.nr - 2) {
        const float curl = ((float)j * a.Btn[o] - (float)(j - 1) * a.Btn[o - 1]) / ((float)j - 0.5f);
        const float je = 0.5f * (a.Jz[o] + a.Jz[o + a.nr]);
        float jb = 0.0f;
        if (a.alpha != 0.0f) {
            const float r = ((float)j - 0.5f) * a.dx;
            const float zeta = ((float)k + 0.5f) * a.dx - a.zc;
            jb = -a.alpha * expf(-r * r * a.inv2sr2 - zeta * zeta * a.inv2sz2);
        }
        a.EzO[o] = a.EzO[o] + a.cdt * curl - a.dt * (je + jb);
    }
}

__global__ void init_kernel(const Args a, float* f) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)kL * kQ * a.Np) return;
    const int lq = (int)(i / a.Np);
    const int l = lq / kQ, q = lq - l * kQ;
    f[i] = l == 0 ? w9(q) * a.n0 : 0.0f;
}

__global__ void export_kernel(const Args a, float* out) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= a.N) return;
    const float n = a.Am[o], A1 = a.Am[a.N + o], A2 = a.Am[2 * a.N + o];
    const float nn = n > a.n_floor ? n : a.n_floor;
    const float pz = A1 / nn, pr = A2 / nn;
    const float g = sqrtf(1.0f + pz * pz + pr * pr);
    out[o] = n;
    out[a.N + o] = pz / g;
    out[2 * a.N + o] = pr / g;
}

dim3 grid_of(const Args& a) { return dim3((a.nr + kBR - 1) / kBR, (a.nz + kBZ - 1) / kBZ, 1); }

}  // namespace

cudaError_t launch_moments(const Args& a, cudaStream_t s) {
    moments_kernel<<<grid_of(a), dim3(kBR, kBZ), 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_fluid(const Args& a, cudaStream_t s) {
    const dim3 grid((unsigned)((a.nr + kOut - 1) / kOut), (unsigned)((a.nz + kBZ - 1) / kBZ), 1);
    fluid_kernel<<<grid, dim3(kBR, kBZ), 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_ampere(const Args& a, cudaStream_t s) {
    ampere_kernel<<<grid_of(a), dim3(kBR, kBZ), 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_init(const Args& a, float* f, cudaStream_t s) {
    const int64_t n = (int64_t)kL * kQ * a.Np;
    init_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, f);
    return cudaGetLastError();
}
cudaError_t launch_export_moments(const Args& a, float* out, cudaStream_t s) {
    export_kernel<<<(unsigned)((a.N + 255) / 256), 256, 0, s>>>(a, out);
    return cudaGetLastError();
}

}  // namespace axi
}  // namespace pwfa
