// Hand-written discrete adjoint of one time step (the paper has no adjoint;
// this differentiates the discrete scheme of the forward kernels exactly).
//
// Forward step n (see fluid.cu / fields.cu):
//   Bn     = Bc - c curl E                              (Faraday, active faces)
//   S^n, J = fluid(S^{n-1}, E, Bc, Bn)                  (stream+collide+source)
//   E'     = E + c curl Bn - dt (avg J + J_b(theta))    (Ampere, active edges)
// Reverse step n, given the adjoints of (S^n, E', Bn as the next B):
//   R1  adj_ampere:   Bn_bar += c curl^T(E'_bar); J_bar = -dt avg^T(E'_bar);
//                     theta_bar += dt E'_z,bar dJ_b/dtheta (FP64)
//   R2a adj_fluid (boundary nodes): A_bar of each Eq. 14 boundary node
//   R2  adj_fluid (interior nodes): S^{n-1}_bar by the transposed pull
//                     (a scatter to x - xi_i), node E_bar and B_bar
//   R3  adj_faces:    Bn_bar += avg4^T(b_bar)/8; Bc_bar = Bn_bar + avg4^T(b_bar)/8
//   R4  adj_edges:    E_bar = E'_bar + avg2^T(e_bar)/2 - c curl_F^T(Bn_bar)
// with c = dt/dx. All adjoint state is FP32; parameter gradients are FP64.
#include "lbm_adjoint.h"
#include "lbm_node.cuh"

namespace pwfa {

namespace {

constexpr int kBX = 32;
constexpr int kBY = 8;

__device__ __forceinline__ bool in_grid(const Grid& g, int i, int j, int k) {
    return i >= 0 && j >= 0 && k >= 0 && i < g.nx && j < g.ny && k < g.nz;
}

// Open-grid activity of each Yee component (conducting walls).
__device__ __forceinline__ bool act_E(const Grid& g, int c, int i, int j, int k) {
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    if (c == 0) return i <= nx - 2 && j >= 1 && j <= ny - 2 && k >= 1 && k <= nz - 2;
    if (c == 1) return i >= 1 && i <= nx - 2 && j <= ny - 2 && k >= 1 && k <= nz - 2;
    return i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2 && k <= nz - 2;
}
__device__ __forceinline__ bool act_B(const Grid& g, int c, int i, int j, int k) {
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    if (c == 0) return i >= 1 && i <= nx - 2 && j <= ny - 2 && k <= nz - 2;
    if (c == 1) return i <= nx - 2 && j >= 1 && j <= ny - 2 && k <= nz - 2;
    return i <= nx - 2 && j <= ny - 2 && k >= 1 && k <= nz - 2;
}

// Read a[c] at (i,j,k): wraps on periodic grids; on open grids zero outside
// the grid and, when mask_e / mask_b, at inactive Yee components.
template <bool PER>
__device__ __forceinline__ float rd(const Grid& g, const float* a, int i, int j, int k) {
    if (PER) {
        i = wrapi(i, g.nx); j = wrapi(j, g.ny); k = wrapi(k, g.nz);
    } else if (!in_grid(g, i, j, k)) {
        return 0.0f;
    }
    return a[((int64_t)k * g.ny + j) * g.nx + i];
}
template <bool PER>
__device__ __forceinline__ float rdE(const Grid& g, const float* a, int c, int i, int j, int k) {
    if (!PER && (!in_grid(g, i, j, k) || !act_E(g, c, i, j, k))) return 0.0f;
    return rd<PER>(g, a, i, j, k);
}

// ------------------------------------------------------------------- R1
template <bool PER>
__global__ void __launch_bounds__(kBX * kBY) adj_ampere_kernel(const AdjArgs a) {
    const Grid& g = a.f.g;
    const int i = blockIdx.x * kBX + threadIdx.x;
    const int j = blockIdx.y * kBY + threadIdx.y;
    const int k = blockIdx.z;
    double g3[3] = {0.0, 0.0, 0.0};
    if (i < g.nx && j < g.ny) {
        const int64_t o = ((int64_t)k * g.ny + j) * g.nx + i;
        const float c = a.f.cdt, dt = a.f.dt;
        const float* Ex = a.Ebar[0];
        const float* Ey = a.Ebar[1];
        const float* Ez = a.Ebar[2];
        const float ex = rdE<PER>(g, Ex, 0, i, j, k);
        const float ey = rdE<PER>(g, Ey, 1, i, j, k);
        const float ez = rdE<PER>(g, Ez, 2, i, j, k);
        float bx = 0.0f, by = 0.0f, bz = 0.0f;
        if (PER || act_B(g, 0, i, j, k))
            bx = a.Bbar[0][o] + c * (ey - rdE<PER>(g, Ey, 1, i, j, k + 1) - ez + rdE<PER>(g, Ez, 2, i, j + 1, k));
        if (PER || act_B(g, 1, i, j, k))
            by = a.Bbar[1][o] + c * (-ex + rdE<PER>(g, Ex, 0, i, j, k + 1) + ez - rdE<PER>(g, Ez, 2, i + 1, j, k));
        if (PER || act_B(g, 2, i, j, k))
            bz = a.Bbar[2][o] + c * (ex - rdE<PER>(g, Ex, 0, i, j + 1, k) - ey + rdE<PER>(g, Ey, 1, i + 1, j, k));
        a.Bnp[0][o] = bx;
        a.Bnp[1][o] = by;
        a.Bnp[2][o] = bz;
        a.Jbar[0][o] = -0.5f * dt * (ex + rdE<PER>(g, Ex, 0, i - 1, j, k));
        a.Jbar[1][o] = -0.5f * dt * (ey + rdE<PER>(g, Ey, 1, i, j - 1, k));
        a.Jbar[2][o] = -0.5f * dt * (ez + rdE<PER>(g, Ez, 2, i, j, k - 1));
        // driver: E_z += dt alpha gauss  =>  d/d(alpha, sigma_r, sigma_z)
        if (ez != 0.0f) {
            const double xr = ((double)i - 0.5 * (g.nx - 1)) * a.f.dx;
            const double yr = ((double)j - 0.5 * (g.ny - 1)) * a.f.dx;
            const double zeta = ((double)k + 0.5) * a.f.dx - a.f.zc;
            const double r2 = xr * xr + yr * yr;
            const double ga = exp(-r2 * a.f.inv2sr2 - zeta * zeta * a.f.inv2sz2);
            const double w = (double)dt * ez * ga;
            g3[0] = w;
            g3[1] = w * a.f.alpha * r2 / ((double)a.sr * a.sr * a.sr);
            g3[2] = w * a.f.alpha * zeta * zeta / ((double)a.sz * a.sz * a.sz);
        }
    }
    // block reduction of the three driver partials, one FP64 atomic each
    __shared__ double sh[3][kBX * kBY / 32];
    for (int c3 = 0; c3 < 3; ++c3)
        for (int off = 16; off > 0; off >>= 1) g3[c3] += __shfl_down_sync(0xffffffffu, g3[c3], off);
    const int t = threadIdx.y * kBX + threadIdx.x;
    if ((t & 31) == 0)
        for (int c3 = 0; c3 < 3; ++c3) sh[c3][t >> 5] = g3[c3];
    __syncthreads();
    if (t < 3) {
        double s = 0.0;
        for (int w = 0; w < kBX * kBY / 32; ++w) s += sh[t][w];
        if (s != 0.0) atomicAdd(a.grad + t, s);
    }
}

// ------------------------------------------------------------------- R2
// Boundary nodes clamping to interior node x: for each axis the candidates
// are x itself and the wall node when x sits next to the wall.
__device__ __forceinline__ int wall_candidates(int v, int n, int out[3]) {
    int m = 0;
    out[m++] = v;
    if (v == 1) out[m++] = 0;
    if (v == n - 2) out[m++] = n - 1;
    return m;
}

template <int ST, int COLL, bool PER, bool BPASS>
#ifndef PWFA_ADJ_MIN_BLOCKS
#define PWFA_ADJ_MIN_BLOCKS 2
#endif
__global__ void __launch_bounds__(256, PWFA_ADJ_MIN_BLOCKS) adj_fluid_kernel(const AdjArgs a) {
    using T = typename Codec<ST>::T;
    const StepArgs& s = a.f;
    const Grid& g = s.g;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const uint32_t N = (uint32_t)g.N;
    const uint32_t node = ((uint32_t)z * (uint32_t)g.ny + (uint32_t)y) * (uint32_t)g.nx + (uint32_t)x;
    const bool bnd = !PER && (x == 0 || y == 0 || z == 0 || x == g.nx - 1 || y == g.ny - 1 || z == g.nz - 1);
    if (BPASS != bnd) {
        if (!BPASS) {
            // A boundary node's own pull slots are never read by the forward
            // step: their adjoint is zero.
            for (int q = 0; q < kQ; ++q) {
                const int sx = x - xi_x(q), sy = y - xi_y(q), sz = z - xi_z(q);
                if (!in_grid(g, sx, sy, sz)) continue;
                const uint32_t so = ((uint32_t)sz * (uint32_t)g.ny + (uint32_t)sy) * (uint32_t)g.nx + (uint32_t)sx;
                for (int l = 0; l < kL; ++l) a.Sbar_out[(size_t)l * kQ * N + ((uint32_t)q * N + so)] = 0.0f;
            }
        }
        return;
    }
    // ---- forward recompute: moments at the (clamped) node
    int xs = x, ys = y, zs = z;
    if (!PER) {
        xs = min(max(x, 1), g.nx - 2);
        ys = min(max(y, 1), g.ny - 2);
        zs = min(max(z, 1), g.nz - 2);
    }
    const T* fin = static_cast<const T*>(s.fin);
    const int64_t LS = lattice_stride(g);
    const T* finl[kL] = {fin, fin + LS, fin + 2 * LS, fin + 3 * LS};
    const float* Sinl[kL] = {a.Sbar_in, a.Sbar_in + (size_t)kQ * N, a.Sbar_in + (size_t)2 * kQ * N,
                             a.Sbar_in + (size_t)3 * kQ * N};
    // (the regularized projection's first moments are not needed: the
    // transpose of P = k3 (m - A u) with respect to m does not involve m)
    float A[kL] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        const uint32_t src = (uint32_t)src_index<PER>(g, xs, ys, zs, q);
#pragma unroll
        for (int l = 0; l < kL; ++l) A[l] += Codec<ST>::load(finl[l] + pop_off(q, src), l, q, s.n0);
    }
    const float n = A[0];
    const float nn = n > s.n_floor ? n : s.n_floor;
    const float p[3] = {A[1] / nn, A[2] / nn, A[3] / nn};
    const float gam = sqrtf(1.0f + p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    const float beta[3] = {p[0] / gam, p[1] / gam, p[2] / gam};
    const float u[3] = {beta[0] * s.lat, beta[1] * s.lat, beta[2] * s.lat};
    float phi[kQ];
    eq_factors(u, phi);
    float e[3] = {0.0f, 0.0f, 0.0f}, b[3] = {0.0f, 0.0f, 0.0f}, F[3] = {0.0f, 0.0f, 0.0f};
    const bool forced = (COLL != 2) && s.couple;
    if (forced) {
        float bc[3], bn[3];
        node_E<PER>(g, s.E, x, y, z, e);
        node_B_sum<PER>(g, s.Bc, x, y, z, bc);
        node_B_sum<PER>(g, s.Bn, x, y, z, bn);
        for (int c = 0; c < 3; ++c) b[c] = 0.125f * (bc[c] + bn[c]);
        F[0] = -n * (e[0] + beta[1] * b[2] - beta[2] * b[1]);
        F[1] = -n * (e[1] + beta[2] * b[0] - beta[0] * b[2]);
        F[2] = -n * (e[2] + beta[0] * b[1] - beta[1] * b[0]);
    }
    const float ps[3] = {(A[1] + F[0] * s.dt) / nn, (A[2] + F[1] * s.dt) / nn, (A[3] + F[2] * s.dt) / nn};
    const float gs = sqrtf(1.0f + ps[0] * ps[0] + ps[1] * ps[1] + ps[2] * ps[2]);
    const float bs[3] = {ps[0] / gs, ps[1] / gs, ps[2] / gs};

    // ---- reverse
    float Ab[kL] = {0.0f, 0.0f, 0.0f, 0.0f};
    float Fb[3] = {0.0f, 0.0f, 0.0f};
    float nb = 0.0f, nnb = 0.0f;
    // J = -n beta(p*)
    {
        const float Jb[3] = {a.Jbar[0][node], a.Jbar[1][node], a.Jbar[2][node]};
        nb -= Jb[0] * bs[0] + Jb[1] * bs[1] + Jb[2] * bs[2];
        const float v[3] = {-n * Jb[0], -n * Jb[1], -n * Jb[2]};
        const float bv = bs[0] * v[0] + bs[1] * v[1] + bs[2] * v[2];
        for (int c = 0; c < 3; ++c) {
            const float psb = (v[c] - bs[c] * bv) / gs;
            Ab[c + 1] += psb / nn;
            Fb[c] += psb * s.dt / nn;
            nnb -= psb * ps[c] / nn;
        }
    }
    // collision (and the Eq. 14 replacement f := A phi on boundary nodes)
    float phib[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) phib[q] = 0.0f;
    float ub[3] = {0.0f, 0.0f, 0.0f};
    float mb[kL][3];
    const float om = s.omega;
    const float k3 = 3.0f * (1.0f - om);
#pragma unroll
    for (int l = 0; l < kL; ++l) {
        mb[l][0] = mb[l][1] = mb[l][2] = 0.0f;
        float Gb = 0.0f, sphi = 0.0f, P0 = 0.0f, P1 = 0.0f, P2 = 0.0f;
        // weight of d fs / d(A phi): omega for interior BGK, 1 otherwise
        const float wA = (COLL == 0 && !bnd) ? om : ((COLL == 2 && !bnd) ? 0.0f : 1.0f);
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const float fsb = Sinl[l][(uint32_t)q * N + node];
            Gb += wq(q) * fsb;
            sphi += phi[q] * fsb;
            phib[q] += wA * A[l] * fsb;
            if (COLL == 1 && !bnd) {
                P0 += wq(q) * (float)xi_x(q) * fsb;
                P1 += wq(q) * (float)xi_y(q) * fsb;
                P2 += wq(q) * (float)xi_z(q) * fsb;
            }
        }
        Ab[l] += wA * sphi;
        if (l > 0 && COLL != 2) Fb[l - 1] += Gb * s.dt;
        if (COLL == 1 && !bnd) {
            mb[l][0] = k3 * P0;
            mb[l][1] = k3 * P1;
            mb[l][2] = k3 * P2;
            Ab[l] -= k3 * (P0 * u[0] + P1 * u[1] + P2 * u[2]);
            ub[0] -= k3 * A[l] * P0;
            ub[1] -= k3 * A[l] * P1;
            ub[2] -= k3 * A[l] * P2;
        }
    }
    // phi_i = w_i (1 - 1.5 u.u + 3 xi.u + 4.5 (xi.u)^2)
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        const float xu = (float)xi_x(q) * u[0] + (float)xi_y(q) * u[1] + (float)xi_z(q) * u[2];
        const float c1 = wq(q) * phib[q];
        const float cx = c1 * (3.0f + 9.0f * xu);
        ub[0] += cx * (float)xi_x(q) - 3.0f * c1 * u[0];
        ub[1] += cx * (float)xi_y(q) - 3.0f * c1 * u[1];
        ub[2] += cx * (float)xi_z(q) - 3.0f * c1 * u[2];
    }
    float betab[3] = {s.lat * ub[0], s.lat * ub[1], s.lat * ub[2]};
    float eb[3] = {0.0f, 0.0f, 0.0f}, bb[3] = {0.0f, 0.0f, 0.0f};
    if (forced) {
        // F = -n (e + beta x b)
        const float bxb[3] = {beta[1] * b[2] - beta[2] * b[1], beta[2] * b[0] - beta[0] * b[2],
                              beta[0] * b[1] - beta[1] * b[0]};
        nb -= Fb[0] * (e[0] + bxb[0]) + Fb[1] * (e[1] + bxb[1]) + Fb[2] * (e[2] + bxb[2]);
        for (int c = 0; c < 3; ++c) eb[c] = -n * Fb[c];
        // d/dbeta [Fb . (beta x b)] = b x Fb ;  d/db = Fb x beta
        betab[0] += -n * (b[1] * Fb[2] - b[2] * Fb[1]);
        betab[1] += -n * (b[2] * Fb[0] - b[0] * Fb[2]);
        betab[2] += -n * (b[0] * Fb[1] - b[1] * Fb[0]);
        bb[0] = -n * (Fb[1] * beta[2] - Fb[2] * beta[1]);
        bb[1] = -n * (Fb[2] * beta[0] - Fb[0] * beta[2]);
        bb[2] = -n * (Fb[0] * beta[1] - Fb[1] * beta[0]);
    }
    // beta = p / gamma
    {
        const float bbv = beta[0] * betab[0] + beta[1] * betab[1] + beta[2] * betab[2];
        for (int c = 0; c < 3; ++c) {
            const float pb = (betab[c] - beta[c] * bbv) / gam;
            Ab[c + 1] += pb / nn;
            nnb -= pb * p[c] / nn;
        }
    }
    if (n > s.n_floor) nb += nnb;
    Ab[0] += nb;

    for (int c = 0; c < 3; ++c) {
        a.ebar[c][node] = eb[c];
        a.bbar[c][node] = bb[c];
    }
    if (BPASS) {
        for (int l = 0; l < kL; ++l) a.Abnd[l][node] = Ab[l];
        return;
    }
    // Boundary nodes that gathered at this node add their A_bar to every
    // population of the corresponding lattice.
    if (!PER && (x == 1 || y == 1 || z == 1 || x == g.nx - 2 || y == g.ny - 2 || z == g.nz - 2)) {
        int cx_[3], cy_[3], cz_[3];
        const int mx = wall_candidates(x, g.nx, cx_), my = wall_candidates(y, g.ny, cy_),
                  mz = wall_candidates(z, g.nz, cz_);
        for (int iz = 0; iz < mz; ++iz)
            for (int iy = 0; iy < my; ++iy)
                for (int ix = 0; ix < mx; ++ix) {
                    if (ix == 0 && iy == 0 && iz == 0) continue;
                    const uint32_t bo =
                        ((uint32_t)cz_[iz] * (uint32_t)g.ny + (uint32_t)cy_[iy]) * (uint32_t)g.nx + (uint32_t)cx_[ix];
                    for (int l = 0; l < kL; ++l) Ab[l] += a.Abnd[l][bo];
                }
    }
    // keep the second read of S_bar_in (BGK, stream-only) after the sums
    // above instead of letting it be hoisted (register pressure)
    asm volatile("" ::: "memory");
    // transposed pull: f_i(x) = S_i(x - xi_i)  =>  S_bar_i(x - xi_i) = f_bar_i(x)
    float* const Soutl[kL] = {a.Sbar_out, a.Sbar_out + (size_t)kQ * N, a.Sbar_out + (size_t)2 * kQ * N,
                              a.Sbar_out + (size_t)3 * kQ * N};
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        const uint32_t src = (uint32_t)src_index<PER>(g, xs, ys, zs, q);
#pragma unroll
        for (int l = 0; l < kL; ++l) {
            float fb = Ab[l];
            if (COLL == 0) fb += (1.0f - om) * Sinl[l][(uint32_t)q * N + node];
            else if (COLL == 2) fb += Sinl[l][(uint32_t)q * N + node];
            else fb += (float)xi_x(q) * mb[l][0] + (float)xi_y(q) * mb[l][1] + (float)xi_z(q) * mb[l][2];
            Soutl[l][(uint32_t)q * N + src] = fb;
        }
    }
}

// ------------------------------------------------------------------- R3
template <bool PER>
__global__ void __launch_bounds__(kBX * kBY) adj_faces_kernel(const AdjArgs a) {
    const Grid& g = a.f.g;
    const int i = blockIdx.x * kBX + threadIdx.x;
    const int j = blockIdx.y * kBY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const int64_t o = ((int64_t)k * g.ny + j) * g.nx + i;
    const float* bx = a.bbar[0];
    const float* by = a.bbar[1];
    const float* bz = a.bbar[2];
    const float sx = 0.125f * (rd<PER>(g, bx, i, j, k) + rd<PER>(g, bx, i, j + 1, k) + rd<PER>(g, bx, i, j, k + 1)
                               + rd<PER>(g, bx, i, j + 1, k + 1));
    const float sy = 0.125f * (rd<PER>(g, by, i, j, k) + rd<PER>(g, by, i + 1, j, k) + rd<PER>(g, by, i, j, k + 1)
                               + rd<PER>(g, by, i + 1, j, k + 1));
    const float sz = 0.125f * (rd<PER>(g, bz, i, j, k) + rd<PER>(g, bz, i + 1, j, k) + rd<PER>(g, bz, i, j + 1, k)
                               + rd<PER>(g, bz, i + 1, j + 1, k));
    const float s3[3] = {sx, sy, sz};
    for (int c = 0; c < 3; ++c) {
        if (PER || act_B(g, c, i, j, k)) {
            const float bnt = a.Bnp[c][o] + s3[c];
            a.Bnp[c][o] = bnt;
            a.Bbar[c][o] = bnt + s3[c];
        } else {
            a.Bnp[c][o] = 0.0f;
            a.Bbar[c][o] = 0.0f;
        }
    }
}

// ------------------------------------------------------------------- R4
template <bool PER>
__global__ void __launch_bounds__(kBX * kBY) adj_edges_kernel(const AdjArgs a) {
    const Grid& g = a.f.g;
    const int i = blockIdx.x * kBX + threadIdx.x;
    const int j = blockIdx.y * kBY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const int64_t o = ((int64_t)k * g.ny + j) * g.nx + i;
    const float c = a.f.cdt;
    const float* Bx = a.Bnp[0];
    const float* By = a.Bnp[1];
    const float* Bz = a.Bnp[2];
    const float* ex = a.ebar[0];
    const float* ey = a.ebar[1];
    const float* ez = a.ebar[2];
    if (PER || act_E(g, 0, i, j, k))
        a.Ebar[0][o] = a.Ebar[0][o] + 0.5f * (rd<PER>(g, ex, i, j, k) + rd<PER>(g, ex, i + 1, j, k))
                     + c * (rd<PER>(g, By, i, j, k) - rd<PER>(g, By, i, j, k - 1) - rd<PER>(g, Bz, i, j, k)
                            + rd<PER>(g, Bz, i, j - 1, k));
    else
        a.Ebar[0][o] = 0.0f;
    if (PER || act_E(g, 1, i, j, k))
        a.Ebar[1][o] = a.Ebar[1][o] + 0.5f * (rd<PER>(g, ey, i, j, k) + rd<PER>(g, ey, i, j + 1, k))
                     + c * (-rd<PER>(g, Bx, i, j, k) + rd<PER>(g, Bx, i, j, k - 1) + rd<PER>(g, Bz, i, j, k)
                            - rd<PER>(g, Bz, i - 1, j, k));
    else
        a.Ebar[1][o] = 0.0f;
    if (PER || act_E(g, 2, i, j, k))
        a.Ebar[2][o] = a.Ebar[2][o] + 0.5f * (rd<PER>(g, ez, i, j, k) + rd<PER>(g, ez, i, j, k + 1))
                     + c * (rd<PER>(g, Bx, i, j, k) - rd<PER>(g, Bx, i, j - 1, k) - rd<PER>(g, By, i, j, k)
                            + rd<PER>(g, By, i - 1, j, k));
    else
        a.Ebar[2][o] = 0.0f;
}

// ------------------------------------------------------------- profile
// Initial stored populations S_0,i(y) = w_i n0 prof(r(y + xi_i)) with prof
// piecewise linear in the profile values: accumulate S_bar w_i n0 times the
// interpolation weights into the profile gradient.
constexpr int kMaxProfile = 256;

__global__ void __launch_bounds__(256) adj_profile_kernel(Grid g, const float* Sbar0, float n0, int np,
                                                          double rmax, double dx, double* grad) {
    __shared__ double bins[kMaxProfile];
    for (int t = threadIdx.x; t < np; t += blockDim.x) bins[t] = 0.0;
    __syncthreads();
    const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (node < g.N) {
        const int64_t sxy = (int64_t)g.nx * g.ny;
        const int z = (int)(node / sxy);
        const int64_t r0 = node - (int64_t)z * sxy;
        const int y = (int)(r0 / g.nx);
        const int x = (int)(r0 - (int64_t)y * g.nx);
        (void)z;
        const double xc = 0.5 * (g.nx - 1) * dx, yc = 0.5 * (g.ny - 1) * dx;
        const double h = np > 1 ? rmax / (np - 1) : 1.0;
        for (int q = 0; q < kQ; ++q) {
            const float sb = Sbar0[(int64_t)q * g.N + node];
            if (sb == 0.0f) continue;
            int sx = x + xi_x(q), sy = y + xi_y(q);
            if (g.periodic) { sx = wrapi(sx, g.nx); sy = wrapi(sy, g.ny); }
            else { sx = min(max(sx, 1), g.nx - 2); sy = min(max(sy, 1), g.ny - 2); }
            const double rx = sx * dx - xc, ry = sy * dx - yc;
            const double r = sqrt(rx * rx + ry * ry);
            const double v = (double)sb * wq(q) * n0;
            if (np == 1 || r >= rmax) {
                atomicAdd(&bins[np - 1], v);
            } else {
                const double tt = r / h;
                int jj = (int)floor(tt);
                if (jj >= np - 1) {
                    atomicAdd(&bins[np - 1], v);
                } else {
                    const double fr = tt - jj;
                    atomicAdd(&bins[jj], (1.0 - fr) * v);
                    atomicAdd(&bins[jj + 1], fr * v);
                }
            }
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < np; t += blockDim.x)
        if (bins[t] != 0.0) atomicAdd(grad + t, bins[t]);
}

dim3 grid_of(const Grid& g, int bx, int by) { return dim3((g.nx + bx - 1) / bx, (g.ny + by - 1) / by, g.nz); }

template <int ST, int COLL>
cudaError_t launch_adj_fluid_t(const AdjArgs& a, cudaStream_t s) {
    const int bx = a.f.bx, by = a.f.by;
    const dim3 grid = grid_of(a.f.g, bx, by), block(bx, by, 1);
    if (a.f.g.periodic) {
        adj_fluid_kernel<ST, COLL, true, false><<<grid, block, 0, s>>>(a);
    } else {
        adj_fluid_kernel<ST, COLL, false, true><<<grid, block, 0, s>>>(a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        adj_fluid_kernel<ST, COLL, false, false><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template <int ST>
cudaError_t launch_adj_fluid_s(const AdjArgs& a, int collision, cudaStream_t s) {
    switch (collision) {
        case 0: return launch_adj_fluid_t<ST, 0>(a, s);
        case 1: return launch_adj_fluid_t<ST, 1>(a, s);
        case 2: return launch_adj_fluid_t<ST, 2>(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_adjoint_step(const AdjArgs& a, int storage, int collision, cudaStream_t s) {
    const Grid& g = a.f.g;
    const dim3 grid = grid_of(g, kBX, kBY), block(kBX, kBY, 1);
    const bool per = g.periodic;
    if (a.f.couple) {
        if (per) adj_ampere_kernel<true><<<grid, block, 0, s>>>(a);
        else adj_ampere_kernel<false><<<grid, block, 0, s>>>(a);
    } else {
        // no Maxwell update: B, E pass through; J is not used
        cudaError_t e = cudaMemsetAsync(a.Jbar[0], 0, sizeof(float) * g.N, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(a.Jbar[1], 0, sizeof(float) * g.N, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(a.Jbar[2], 0, sizeof(float) * g.N, s);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    switch (storage) {
        case 0: e = launch_adj_fluid_s<0>(a, collision, s); break;
        case 1: e = launch_adj_fluid_s<1>(a, collision, s); break;
        case 2: e = launch_adj_fluid_s<2>(a, collision, s); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess || !a.f.couple) return e;
    if (per) adj_faces_kernel<true><<<grid, block, 0, s>>>(a);
    else adj_faces_kernel<false><<<grid, block, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (per) adj_edges_kernel<true><<<grid, block, 0, s>>>(a);
    else adj_edges_kernel<false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_profile(const Grid& g, const float* Sbar, float n0, int n_profile, double rmax,
                                   double dx, double* grad_profile, cudaStream_t s) {
    if (n_profile <= 0) return cudaSuccess;
    if (n_profile > kMaxProfile) return cudaErrorInvalidValue;
    const int threads = 256;
    const unsigned blocks = (unsigned)((g.N + threads - 1) / threads);
    adj_profile_kernel<<<blocks, threads, 0, s>>>(g, Sbar, n0, n_profile, rmax, dx, grad_profile);
    return cudaGetLastError();
}

}  // namespace pwfa
