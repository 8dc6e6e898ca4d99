// Per-node body of the fused fluid step, shared by the single-instance
// kernel (fluid.cu) and the batched persistent kernel (batch.cu).
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
#pragma once

#include "lbm_node.cuh"

namespace pwfa {

// Node quantities handed to the fused diagnostics (state entering the step).
struct NodeDiag {
    float n, a1, a2, a3, beta2;
};

// m = sum_i xi_i f_i over one lattice's 19 values (signed adds, q ascending).
__device__ __forceinline__ void first_moments(const float (&fl)[kQ], float (&m)[3]) {
    float m0 = 0.0f, m1 = 0.0f, m2 = 0.0f;
#pragma unroll
    for (int q = 1; q < kQ; ++q) {
        if (xi_x(q) > 0) m0 += fl[q]; else if (xi_x(q) < 0) m0 -= fl[q];
        if (xi_y(q) > 0) m1 += fl[q]; else if (xi_y(q) < 0) m1 -= fl[q];
        if (xi_z(q) > 0) m2 += fl[q]; else if (xi_z(q) < 0) m2 -= fl[q];
    }
    m[0] = m0;
    m[1] = m1;
    m[2] = m2;
}

// Lattice sums and first moments of one lattice from values s in stored
// units of a 16-bit form, f = kappa_i s + w_i n0 delta_l0: the rest, axis and
// diagonal directions are summed apart and weighted once (kappa is 1 for
// BF16, w_i / 1024 for FP16; sum_i w_i = 1 and sum_i xi_i w_i = 0 give the
// base terms).
template <int ST>
__device__ __forceinline__ void raw_moments(const float (&s)[kQ], float base, float& A, float (&m)[3]) {
    float sa = 0.0f, sd = 0.0f, ma[3] = {0.0f, 0.0f, 0.0f}, md[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int q = 1; q < kQ; ++q) {
        float* mc = q <= 6 ? ma : md;
        if (q <= 6) sa += s[q]; else sd += s[q];
        if (xi_x(q) > 0) mc[0] += s[q]; else if (xi_x(q) < 0) mc[0] -= s[q];
        if (xi_y(q) > 0) mc[1] += s[q]; else if (xi_y(q) < 0) mc[1] -= s[q];
        if (xi_z(q) > 0) mc[2] += s[q]; else if (xi_z(q) < 0) mc[2] -= s[q];
    }
    constexpr float k0 = Codec<ST>::kappa(0), ka = Codec<ST>::kappa(1), kd = Codec<ST>::kappa(7);
    A = base + (k0 * s[0] + ka * sa + kd * sd);
#pragma unroll
    for (int c = 0; c < 3; ++c) m[c] = ka * ma[c] + kd * md[c];
}

// The moments a node's step needs from its pulled populations: the lattice
// sums A_l, 1/max(n, n_floor), beta, and for the regularized collision the
// first moments m_l = sum_i xi_i f_l,i (taken here so that the 76 pulled
// values are dead before the fields are read; a boundary node recomputes
// them from its equilibrium in fluid_rest).
struct NodeMoments {
    float A[kL], inn, beta[3], m[kL][3];
};

template <int ST, int COLL, bool RAW>
__device__ __forceinline__ void fluid_moments(const StepArgs& a, const float (&f)[kL][kQ], NodeMoments& s) {
    constexpr bool RAWR = RAW && ST != 0 && COLL == 1;
    if constexpr (RAWR) {
#pragma unroll
        for (int l = 0; l < kL; ++l) raw_moments<ST>(f[l], l == 0 ? a.n0 : 0.0f, s.A[l], s.m[l]);
        node_velocity(s.A, a.n_floor, s.inn, s.beta);
    } else {
        node_moments(f, a.n_floor, s.A, s.inn, s.beta);
        if (COLL == 1) {
#pragma unroll
            for (int l = 0; l < kL; ++l) first_moments(f[l], s.m[l]);
        }
    }
}

// Shared-memory words of one thread's parked BGK values (lattices 2 and 3),
// thread index fastest: a warp's 32 accesses of one value hit 32 banks. The
// accesses are opaque to the compiler, so the parked registers are free
// until the collision reads the words back.
constexpr int kStashVals = 2 * kQ;
__device__ __forceinline__ void stash_st(uint32_t a, float v) {
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v));
}
__device__ __forceinline__ float stash_ld(uint32_t a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}

// Everything after the moments: source, collision, stores, current. f holds
// the pulled populations f^n(x) (of the clamped node when bnd; BGK and
// stream-only read them, the regularized form only uses f as its output
// scratch); with RAW (16-bit storage, regularized collision) in stored units,
// and the post-collision values are formed in stored units too, so that
// neither the decode nor the encode of the deviations costs a per-value
// operation.
template <int ST, int COLL, bool PER, bool DIAG = false, bool RAW = false, bool MOM = false, bool PARK = false>
__device__ __forceinline__ void fluid_rest(const StepArgs& a, int x, int y, int z, float (&f)[kL][kQ], bool bnd,
                                           NodeMoments& s, NodeDiag* nd = nullptr) {
    using T = typename Codec<ST>::T;
    constexpr bool RAWR = RAW && ST != 0 && COLL == 1;
    const Grid& g = a.g;
    const uint32_t node =
        PWFA_CHECK(a.dbg, ((uint32_t)z * (uint32_t)g.ny + (uint32_t)y) * (uint32_t)g.nx + (uint32_t)x, 0, g.N, 2u);
    float(&A)[kL] = s.A;
    float& inn = s.inn;
    float(&beta)[3] = s.beta;
    float(&m)[kL][3] = s.m;
    const float n = A[0];
    // PARK (BGK): lattices 2 and 3 wait in shared memory while the fields are
    // read and the source is formed (128 threads per block at most)
    constexpr bool STASH = PARK && COLL == 0;
    __shared__ float stash[STASH ? kStashVals : 1][PWFA_FLUID_MAX_THREADS];
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(&stash[0][threadIdx.y * blockDim.x + threadIdx.x]);
    constexpr uint32_t kSRow = 4u * PWFA_FLUID_MAX_THREADS;
    if constexpr (STASH) {
#pragma unroll
        for (int l = 2; l < kL; ++l)
#pragma unroll
            for (int q = 0; q < kQ; ++q) stash_st(sbase + kSRow * ((l - 2) * kQ + q), f[l][q]);
    }
    if (MOM) {
        // the adjoint's recompute keeps the lattice sums (the reverse step
        // needs nothing else of the populations)
#pragma unroll
        for (int l = 0; l < kL; ++l) __stcs(a.mom + (int64_t)l * g.N + node, A[l]);
    }
    if (DIAG) {
        nd->n = A[0];
        nd->a1 = A[1];
        nd->a2 = A[2];
        nd->a3 = A[3];
        nd->beta2 = beta[0] * beta[0] + beta[1] * beta[1] + beta[2] * beta[2];
    }

    // Lorentz source (Eq. 4): F_0 = 0, F_k = -n (E + beta x B)_k, with B the
    // mean of its two time levels.
    float F[3] = {0.0f, 0.0f, 0.0f};
    if (COLL != 2 && a.couple) {
        float e[3], bc[3], bn[3];
        node_E<PER>(g, a.E, x, y, z, e, a.dbg);
        node_B_sum<PER>(g, a.Bc, x, y, z, bc, a.dbg);
        node_B_sum<PER>(g, a.Bn, x, y, z, bn, a.dbg);
        const float b0 = 0.125f * (bc[0] + bn[0]);
        const float b1 = 0.125f * (bc[1] + bn[1]);
        const float b2 = 0.125f * (bc[2] + bn[2]);
        F[0] = -n * (e[0] + beta[1] * b2 - beta[2] * b1);
        F[1] = -n * (e[1] + beta[2] * b0 - beta[0] * b2);
        F[2] = -n * (e[2] + beta[0] * b1 - beta[1] * b0);
    }

    const int64_t LS = lattice_stride(g);
    T* const fo0 = static_cast<T*>(a.fout);
    // per-lattice (FP32) or per-pair (16-bit) base pointers, 32-bit offsets
    T* const fo[kL] = {fo0, fo0 + LS, fo0 + 2 * LS, fo0 + 3 * LS};
    const float u[3] = {beta[0] * a.lat, beta[1] * a.lat, beta[2] * a.lat};
    // (the FP16 stored-unit path keeps phi_i / w_i)
    constexpr bool UNW = RAWR && ST == 2;
    float phi[kQ];
    eq_factors<!UNW>(u, phi);
    if (!PER && bnd) {
        // Eq. 14: a boundary node holds the equilibrium of the clamped node.
#pragma unroll
        for (int l = 0; l < kL; ++l) {
            float fe[kQ];
#pragma unroll
            for (int q = 0; q < kQ; ++q) fe[q] = UNW ? A[l] * (wq(q) * phi[q]) : A[l] * phi[q];
            if (COLL == 1) first_moments(fe, m[l]);
            if constexpr (!RAWR) {
#pragma unroll
                for (int q = 0; q < kQ; ++q) f[l][q] = fe[q];
            }
            if constexpr (STASH) {
                if (l >= 2) {
#pragma unroll
                    for (int q = 0; q < kQ; ++q) stash_st(sbase + kSRow * ((l - 2) * kQ + q), fe[q]);
                }
            }
        }
    }
    // Collide in place, lattice pair by lattice pair; FP32 stores each value
    // as it is made, the 16-bit forms store each pair of lattices as 32-bit
    // words (pop_elem).
    const float om = a.omega;
#pragma unroll
    for (int pr = 0; pr < kL / 2; ++pr) {
#pragma unroll
        for (int l = 2 * pr; l < 2 * pr + 2; ++l) {
            const float Fl = l == 0 ? 0.0f : F[l - 1] * a.dt;
            if (COLL == 0) {
                // BGK, Eq. 7, plus the source of Eq. 10
                if constexpr (STASH) {
                    if (l >= 2) {
#pragma unroll
                        for (int q = 0; q < kQ; ++q) f[l][q] = stash_ld(sbase + kSRow * ((l - 2) * kQ + q));
                    }
                }
#pragma unroll
                for (int q = 0; q < kQ; ++q) f[l][q] = f[l][q] + om * (A[l] * phi[q] - f[l][q]) + wq(q) * Fl;
            } else if (COLL == 1) {
                // Regularized: relax only the first Hermite moment of f - f^eq,
                // Pi = sum_i xi_i (f_i - A phi_i) = sum_i xi_i f_i - A u
                // (sum_i xi_i phi_i = u exactly for the D3Q19 weights).
                const float m0 = m[l][0], m1 = m[l][1], m2 = m[l][2];
                // w_i (xi_i . P + F dt) with the two weights of the moving
                // directions (1/18 axis, 1/36 diagonal) folded into P and F:
                // f = A phi_i + one or two adds of +-P_k w + F w.
                const float k3 = 3.0f * (1.0f - om);
                const float P[3] = {k3 * (m0 - A[l] * u[0]), k3 * (m1 - A[l] * u[1]), k3 * (m2 - A[l] * u[2])};
                if constexpr (RAWR && ST == 2) {
                    // FP16 stores (f - w_i n0 delta_l0) 1024 / w_i
                    //   = 1024 (A phi_i / w_i + xi_i . P + F dt - n0 delta_l0)
                    const float A1 = kF16Scale * A[l];
                    const float P1[3] = {kF16Scale * P[0], kF16Scale * P[1], kF16Scale * P[2]};
                    const float G1 = kF16Scale * (Fl - (l == 0 ? a.n0 : 0.0f));
#pragma unroll
                    for (int q = 0; q < kQ; ++q) {
                        float s = G1;
                        if (xi_x(q) > 0) s += P1[0]; else if (xi_x(q) < 0) s -= P1[0];
                        if (xi_y(q) > 0) s += P1[1]; else if (xi_y(q) < 0) s -= P1[1];
                        if (xi_z(q) > 0) s += P1[2]; else if (xi_z(q) < 0) s -= P1[2];
                        f[l][q] = fmaf(A1, phi[q], s);
                    }
                } else {
                    // FP32 / BF16 (BF16 stores f - w_i n0 delta_l0: the base
                    // enters with the source)
                    const float G = RAWR ? Fl - (l == 0 ? a.n0 : 0.0f) : Fl;
                    const float Pa[3] = {P[0] * (1.0f / 18.0f), P[1] * (1.0f / 18.0f), P[2] * (1.0f / 18.0f)};
                    const float Pd[3] = {P[0] * (1.0f / 36.0f), P[1] * (1.0f / 36.0f), P[2] * (1.0f / 36.0f)};
                    const float Ga = G * (1.0f / 18.0f), Gd = G * (1.0f / 36.0f);
#pragma unroll
                    for (int q = 0; q < kQ; ++q) {
                        const int nz = (xi_x(q) != 0) + (xi_y(q) != 0) + (xi_z(q) != 0);
                        const float* Pw = nz == 2 ? Pd : Pa;
                        float s = nz == 0 ? G * (1.0f / 3.0f) : (nz == 2 ? Gd : Ga);
                        if (xi_x(q) > 0) s += Pw[0]; else if (xi_x(q) < 0) s -= Pw[0];
                        if (xi_y(q) > 0) s += Pw[1]; else if (xi_y(q) < 0) s -= Pw[1];
                        if (xi_z(q) > 0) s += Pw[2]; else if (xi_z(q) < 0) s -= Pw[2];
                        f[l][q] = fmaf(A[l], phi[q], s);
                    }
                }
            }
            // (stream only: f* = f)
            if constexpr (ST == 0) {
#pragma unroll
                for (int q = 0; q < kQ; ++q) Codec<ST>::store(fo[l] + pop_off(q, node), f[l][q], l, q, a.n0);
            }
        }
        if constexpr (RAWR) {
#pragma unroll
            for (int q = 0; q < kQ; ++q)
                Codec<ST>::store2raw(fo[2 * pr] + 2 * pop_off(q, node), f[2 * pr][q], f[2 * pr + 1][q]);
        } else if constexpr (ST != 0) {
#pragma unroll
            for (int q = 0; q < kQ; ++q)
                Codec<ST>::store2(fo[2 * pr] + 2 * pop_off(q, node), f[2 * pr][q], f[2 * pr + 1][q], 2 * pr, q, a.n0);
        }
    }

    // Node current for Ampere: J = -n beta(p*), p* = (A_k + F_k dt) / nn.
    const float ps0 = (A[1] + F[0] * a.dt) * inn;
    const float ps1 = (A[2] + F[1] * a.dt) * inn;
    const float ps2 = (A[3] + F[2] * a.dt) * inn;
    const float ngs = -n * rsqrtf(1.0f + ps0 * ps0 + ps1 * ps1 + ps2 * ps2);
    __stcs(a.J[0] + node, ngs * ps0);
    __stcs(a.J[1] + node, ngs * ps1);
    __stcs(a.J[2] + node, ngs * ps2);
}

// Everything after the gather: moments, then fluid_rest.
template <int ST, int COLL, bool PER, bool DIAG = false, bool RAW = false, bool MOM = false, bool PARK = false>
__device__ __forceinline__ void fluid_compute(const StepArgs& a, int x, int y, int z, float (&f)[kL][kQ], bool bnd,
                                              NodeDiag* nd = nullptr) {
    NodeMoments s;
    fluid_moments<ST, COLL, RAW>(a, f, s);
    fluid_rest<ST, COLL, PER, DIAG, RAW, MOM, PARK>(a, x, y, z, f, bnd, s, nd);
}

template <int ST, int COLL, bool PER, bool DIAG = false, bool MOM = false, bool PARK = false>
__device__ __forceinline__ void fluid_node(const StepArgs& a, int x, int y, int z, NodeDiag* nd = nullptr) {
    using T = typename Codec<ST>::T;
    float f[kL][kQ];
    bool bnd;
    // the 16-bit regularized form works in stored units (see fluid_compute)
    constexpr bool RAW = ST != 0 && COLL == 1;
    gather<ST, PER, RAW>(a.g, static_cast<const T*>(a.fin), a.n0, x, y, z, f, bnd, a.src_shift, a.dbg);
    fluid_compute<ST, COLL, PER, DIAG, RAW, MOM, PARK>(a, x, y, z, f, bnd, nd);
}

}  // namespace pwfa
