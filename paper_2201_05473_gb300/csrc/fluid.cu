// Fused fluid kernel of one time step: the hot path of the method.
//
// One thread per node. It pulls the 76 populations of the four advection-
// diffusion lattices (Eq. 6), takes their moments (Eq. 8) and the relativistic
// velocity beta(p) (Eq. 2), evaluates the Lorentz source F = -n (E + beta x B)
// (Eq. 4) with the Yee fields averaged to the node, collides every lattice
// towards the shared equilibrium of Eq. 9 (BGK Eq. 7, or the regularized
// variant) adding S_i = w_i F dt (Eq. 10), and stores f* at its own node for
// the next step's pull. Boundary nodes of open grids take f^eq of their
// clamped interior node (Eq. 14). It also writes the node current
// J = -n beta(p*) from the post-collision momentum p* = (A_k + F_k dt)/n,
// which Ampere's law consumes.
//
// Memory traffic per node: 76 population reads + 76 writes (FP32: 608 B),
// E (one edge per component) + two B time levels (36 B) read, J (12 B)
// written; neighbouring edge/face reads hit L1/L2.
#include "lbm_kernels.h"
#include "lbm_node.cuh"

namespace pwfa {

namespace {

constexpr int kBX = 32;
constexpr int kBY = 4;

template <int ST, int COLL, bool PER>
__global__ void __launch_bounds__(kBX * kBY) fluid_kernel(const StepArgs a) {
    using T = typename Codec<ST>::T;
    const Grid& g = a.g;
    const int x = blockIdx.x * kBX + threadIdx.x;
    const int y = blockIdx.y * kBY + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const int64_t node = ((int64_t)z * g.ny + y) * g.nx + x;

    float f[kL][kQ];
    bool bnd;
    gather<ST, PER>(g, static_cast<const T*>(a.fin), a.n0, x, y, z, f, bnd);

    float A[kL], nn, beta[3];
    node_moments(f, a.n_floor, A, nn, beta);
    const float n = A[0];

    // Lorentz source (Eq. 4): F_0 = 0, F_k = -n (E + beta x B)_k.
    float F[3] = {0.0f, 0.0f, 0.0f};
    if (COLL != 2 && a.couple) {
        float e[3], bc[3], bn[3];
        node_E<PER>(g, a.E, x, y, z, e);
        node_B_sum<PER>(g, a.Bc, x, y, z, bc);
        node_B_sum<PER>(g, a.Bn, x, y, z, bn);
        const float b0 = 0.125f * (bc[0] + bn[0]);
        const float b1 = 0.125f * (bc[1] + bn[1]);
        const float b2 = 0.125f * (bc[2] + bn[2]);
        F[0] = -n * (e[0] + beta[1] * b2 - beta[2] * b1);
        F[1] = -n * (e[1] + beta[2] * b0 - beta[0] * b2);
        F[2] = -n * (e[2] + beta[0] * b1 - beta[1] * b0);
    }

    T* fout = static_cast<T*>(a.fout);
    const float u[3] = {beta[0] * a.lat, beta[1] * a.lat, beta[2] * a.lat};
    float phi[kQ];
    eq_factors(u, phi);
    if (!PER && bnd) {
        // Eq. 14: a boundary node holds the equilibrium of the clamped node.
#pragma unroll
        for (int l = 0; l < kL; ++l)
#pragma unroll
            for (int q = 0; q < kQ; ++q) f[l][q] = A[l] * phi[q];
    }
    if (COLL == 2) {
        // streaming only: f* = f
#pragma unroll
        for (int l = 0; l < kL; ++l)
#pragma unroll
            for (int q = 0; q < kQ; ++q)
                Codec<ST>::store(fout + (int64_t)(l * kQ + q) * g.N + node, f[l][q], l == 0 ? wq(q) * a.n0 : 0.0f);
    } else {
        const float om = a.omega;
#pragma unroll
        for (int l = 0; l < kL; ++l) {
            const float Fl = l == 0 ? 0.0f : F[l - 1] * a.dt;
            if (COLL == 0) {
                // BGK, Eq. 7 + source Eq. 10
#pragma unroll
                for (int q = 0; q < kQ; ++q) {
                    const float fe = A[l] * phi[q];
                    const float fs = f[l][q] + om * (fe - f[l][q]) + wq(q) * Fl;
                    Codec<ST>::store(fout + (int64_t)(l * kQ + q) * g.N + node, fs, l == 0 ? wq(q) * a.n0 : 0.0f);
                }
            } else {
                // Regularized: relax only Pi = sum_i xi_i (f_i - f^eq_i).
                float P0 = 0.0f, P1 = 0.0f, P2 = 0.0f;
#pragma unroll
                for (int q = 0; q < kQ; ++q) {
                    const float d = f[l][q] - A[l] * phi[q];
                    if (xi_x(q)) P0 += (float)xi_x(q) * d;
                    if (xi_y(q)) P1 += (float)xi_y(q) * d;
                    if (xi_z(q)) P2 += (float)xi_z(q) * d;
                }
                const float k3 = 3.0f * (1.0f - om);
#pragma unroll
                for (int q = 0; q < kQ; ++q) {
                    const float xp = (float)xi_x(q) * P0 + (float)xi_y(q) * P1 + (float)xi_z(q) * P2;
                    const float fs = A[l] * phi[q] + k3 * wq(q) * xp + wq(q) * Fl;
                    Codec<ST>::store(fout + (int64_t)(l * kQ + q) * g.N + node, fs, l == 0 ? wq(q) * a.n0 : 0.0f);
                }
            }
        }
    }

    // Node current for Ampere: J = -n beta(p*), p* = (A_k + F_k dt) / nn.
    const float ps0 = (A[1] + F[0] * a.dt) / nn;
    const float ps1 = (A[2] + F[1] * a.dt) / nn;
    const float ps2 = (A[3] + F[2] * a.dt) / nn;
    const float gs = sqrtf(1.0f + ps0 * ps0 + ps1 * ps1 + ps2 * ps2);
    __stcs(a.J[0] + node, -n * ps0 / gs);
    __stcs(a.J[1] + node, -n * ps1 / gs);
    __stcs(a.J[2] + node, -n * ps2 / gs);
}

template <int ST, int COLL>
cudaError_t launch_fluid_t(const StepArgs& a, cudaStream_t s) {
    dim3 block(kBX, kBY, 1);
    dim3 grid((a.g.nx + kBX - 1) / kBX, (a.g.ny + kBY - 1) / kBY, a.g.nz);
    if (a.g.periodic) fluid_kernel<ST, COLL, true><<<grid, block, 0, s>>>(a);
    else fluid_kernel<ST, COLL, false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

template <int ST>
cudaError_t launch_fluid_s(const StepArgs& a, int collision, cudaStream_t s) {
    switch (collision) {
        case 0: return launch_fluid_t<ST, 0>(a, s);
        case 1: return launch_fluid_t<ST, 1>(a, s);
        case 2: return launch_fluid_t<ST, 2>(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_fluid(const StepArgs& a, int storage, int collision, cudaStream_t s) {
    switch (storage) {
        case 0: return launch_fluid_s<0>(a, collision, s);
        case 1: return launch_fluid_s<1>(a, collision, s);
        case 2: return launch_fluid_s<2>(a, collision, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace pwfa
