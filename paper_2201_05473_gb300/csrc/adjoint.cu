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

// Read a at (i,j,k): wraps on periodic grids; zero outside an open grid.
template <bool PER>
__device__ __forceinline__ float rd(const Grid& g, const float* a, int i, int j, int k) {
    if (PER) {
        i = wrapi(i, g.nx); j = wrapi(j, g.ny); k = wrapi(k, g.nz);
    } else if (!in_grid(g, i, j, k)) {
        return 0.0f;
    }
    return a[((int64_t)k * g.ny + j) * g.nx + i];
}
// Open-grid neighbours of node o for the field adjoints: the index offsets
// of the +-1 neighbours on each axis (0 where the neighbour lies outside the
// grid, so that every load stays valid and can be issued at once) and the
// matching in-grid flags that mask the loaded values.
struct Nbr {
    int64_t pi, pj, pk, mi, mj, mk;
    bool ip, jp, kp, im, jm, km;
};
__device__ __forceinline__ Nbr nbr_of(const Grid& g, int i, int j, int k) {
    Nbr n;
    n.ip = i + 1 < g.nx; n.jp = j + 1 < g.ny; n.kp = k + 1 < g.nz;
    n.im = i > 0; n.jm = j > 0; n.km = k > 0;
    const int64_t sx = g.nx, sxy = (int64_t)g.nx * g.ny;
    n.pi = n.ip ? 1 : 0; n.pj = n.jp ? sx : 0; n.pk = n.kp ? sxy : 0;
    n.mi = n.im ? 1 : 0; n.mj = n.jm ? sx : 0; n.mk = n.km ? sxy : 0;
    return n;
}
__device__ __forceinline__ float msk(bool ok, float v) { return ok ? v : 0.0f; }

// R3's transposed average of one face component: b_bar at the node and its
// three neighbours across the face (the node B is the mean of two time
// levels, each the mean of four faces: 1/8 per face), each masked by its
// in-grid flag. R4's update of one E_bar component: e the sum of the two
// node-averaged E_bar of the edge, d the transposed Faraday curl of Bn_bar.
// Both the separate and the fused kernels go through these, so they agree
// bit for bit.
__device__ __forceinline__ float r3_sum(float v0, float v1, float v2, float v3, bool m1, bool m2, bool m3) {
    return 0.125f * (v0 + msk(m1, v1) + msk(m2, v2) + msk(m3, v3));
}
__device__ __forceinline__ float r4_arith(float c, float E, float e, float d) { return E + 0.5f * e + c * d; }

// ------------------------------------------------------------------- R1
// Every load of a node is issued before any is used; the driver-gradient
// terms are formed and summed over the warp in FP32 (FP64 arithmetic is slow
// on this part) and each warp adds its three sums to an FP64 slot (no block
// barrier). On open grids E_bar is zero at every inactive component (the
// seed is masked before the sweep, R4 writes zeros there), so a neighbour
// read needs only its grid bound: past the upper walls the clamped index
// lands on an inactive component, below the lower ones the bound masks it.
// The values R1 reads at one node.
struct R1In {
    float ex, ey, ez, ey_k, ez_j, ex_k, ez_i, ex_j, ey_i, ex_m, ey_m, ez_m, b0, b1, b2;
};

template <bool PER>
__device__ __forceinline__ void r1_load(const AdjArgs& a, int i, int j, int k, R1In& v) {
    const Grid& g = a.f.g;
    const int64_t o = ((int64_t)k * g.ny + j) * g.nx + i;
    const float* Ex = a.Ebar[0];
    const float* Ey = a.Ebar[1];
    const float* Ez = a.Ebar[2];
    if (PER) {
        v.ex = rd<true>(g, Ex, i, j, k);
        v.ey = rd<true>(g, Ey, i, j, k);
        v.ez = rd<true>(g, Ez, i, j, k);
        v.ey_k = rd<true>(g, Ey, i, j, k + 1);
        v.ez_j = rd<true>(g, Ez, i, j + 1, k);
        v.ex_k = rd<true>(g, Ex, i, j, k + 1);
        v.ez_i = rd<true>(g, Ez, i + 1, j, k);
        v.ex_j = rd<true>(g, Ex, i, j + 1, k);
        v.ey_i = rd<true>(g, Ey, i + 1, j, k);
        v.ex_m = rd<true>(g, Ex, i - 1, j, k);
        v.ey_m = rd<true>(g, Ey, i, j - 1, k);
        v.ez_m = rd<true>(g, Ez, i, j, k - 1);
    } else {
        const Nbr n = nbr_of(g, i, j, k);
        v.ex = Ex[o];
        v.ey = Ey[o];
        v.ez = Ez[o];
        const float v0 = Ey[o + n.pk], v1 = Ez[o + n.pj], v2 = Ex[o + n.pk], v3 = Ez[o + n.pi], v4 = Ex[o + n.pj],
                    v5 = Ey[o + n.pi], v6 = Ex[o - n.mi], v7 = Ey[o - n.mj], v8 = Ez[o - n.mk];
        v.ey_k = msk(n.kp, v0);
        v.ez_j = msk(n.jp, v1);
        v.ex_k = msk(n.kp, v2);
        v.ez_i = msk(n.ip, v3);
        v.ex_j = msk(n.jp, v4);
        v.ey_i = msk(n.ip, v5);
        v.ex_m = msk(n.im, v6);
        v.ey_m = msk(n.jm, v7);
        v.ez_m = msk(n.km, v8);
    }
    v.b0 = a.Bbar[0][o];
    v.b1 = a.Bbar[1][o];
    v.b2 = a.Bbar[2][o];
}

// R1's arithmetic and stores at one node; the driver-gradient terms are added
// to g3.
template <bool PER>
__device__ __forceinline__ void r1_node(const AdjArgs& a, int i, int j, int k, const R1In& v, float (&g3)[3]) {
    const Grid& g = a.f.g;
    const int64_t o = ((int64_t)k * g.ny + j) * g.nx + i;
    const float c = a.f.cdt, dt = a.f.dt;
    const bool cx = PER || act_B(g, 0, i, j, k);
    const bool cy = PER || act_B(g, 1, i, j, k);
    const bool cz = PER || act_B(g, 2, i, j, k);
    a.Bnp[0][o] = cx ? v.b0 + c * (v.ey - v.ey_k - v.ez + v.ez_j) : 0.0f;
    a.Bnp[1][o] = cy ? v.b1 + c * (-v.ex + v.ex_k + v.ez - v.ez_i) : 0.0f;
    a.Bnp[2][o] = cz ? v.b2 + c * (v.ex - v.ex_j - v.ey + v.ey_i) : 0.0f;
    a.Jbar[0][o] = -0.5f * dt * (v.ex + v.ex_m);
    a.Jbar[1][o] = -0.5f * dt * (v.ey + v.ey_m);
    a.Jbar[2][o] = -0.5f * dt * (v.ez + v.ez_m);
    // driver: E_z += dt alpha gauss  =>  d/d(alpha, sigma_r, sigma_z),
    // the derivative of the forward's FP32 Gaussian evaluated the same way
    if (v.ez != 0.0f) {
        const float xr = ((float)i - 0.5f * (float)(g.nx - 1)) * a.f.dx;
        const float yr = ((float)j - 0.5f * (float)(g.ny - 1)) * a.f.dx;
        const float zeta = ((float)k + 0.5f) * a.f.dx - a.f.zc;
        const float r2 = xr * xr + yr * yr;
        const float er = -r2 * a.f.inv2sr2, ez2 = -zeta * zeta * a.f.inv2sz2;
        // below -104 a factor's exp (< 7e-46) rounds to zero in FP32: the
        // term is dropped
        if (er >= -104.0f && ez2 >= -104.0f) {
            const float ga = expf(er) * expf(ez2);
            const float w = dt * v.ez * ga;
            g3[0] += w;
            g3[1] += w * a.csr * r2;
            g3[2] += w * a.csz * (zeta * zeta);
        }
    }
}

// Each thread takes kR1Planes consecutive planes of its (x, y) column and
// issues all their loads before any store: one node per thread left a
// single memory round in flight per thread (0.63 of the copy bandwidth).
constexpr int kR1Planes = 2;

template <bool PER>
__global__ void __launch_bounds__(kBX * kBY) adj_ampere_kernel(const AdjArgs a) {
    const Grid& g = a.f.g;
    const int i = blockIdx.x * kBX + threadIdx.x;
    const int j = blockIdx.y * kBY + threadIdx.y;
    const int k0 = blockIdx.z * kR1Planes;
    float g3[3] = {0.0f, 0.0f, 0.0f};
    if (i < g.nx && j < g.ny) {
        R1In v[kR1Planes];
#pragma unroll
        for (int p = 0; p < kR1Planes; ++p)
            if (k0 + p < g.nz) r1_load<PER>(a, i, j, k0 + p, v[p]);
#pragma unroll
        for (int p = 0; p < kR1Planes; ++p)
            if (k0 + p < g.nz) r1_node<PER>(a, i, j, k0 + p, v[p], g3);
    }
    // most warps lie where the driver density is zero: no sums to form
    if (!__any_sync(0xffffffffu, g3[0] != 0.0f || g3[1] != 0.0f || g3[2] != 0.0f)) return;
    for (int c3 = 0; c3 < 3; ++c3)
        for (int off = 16; off > 0; off >>= 1) g3[c3] += __shfl_down_sync(0xffffffffu, g3[c3], off);
    const int t = threadIdx.y * kBX + threadIdx.x;
    if ((t & 31) == 0 && (g3[0] != 0.0f || g3[1] != 0.0f || g3[2] != 0.0f)) {
        const uint32_t w = ((blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) * (kBX * kBY / 32) +
                           (uint32_t)(t >> 5);
        double* slot = a.gslots + 3 * (w % kGradSlots);
        for (int c3 = 0; c3 < 3; ++c3) atomicAdd(slot + c3, (double)g3[c3]);
    }
}

__global__ void __launch_bounds__(256) adj_grad_finish_kernel(const double* gslots, double* grad) {
    __shared__ double sh[3][256];
    double s[3] = {0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < kGradSlots; i += blockDim.x)
        for (int c = 0; c < 3; ++c) s[c] += gslots[3 * i + c];
    for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] = s[c];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 3) grad[threadIdx.x] += sh[threadIdx.x][0];
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

// Lattice-split form: a block of four warps takes 32 nodes of one x-row and
// warp l owns lattice l. Each warp issues its lattice's 19 pulled populations
// and 19 stored-population adjoints together (one memory round per node); the
// lattice sums, the per-lattice reductions and the node-level adjoint (done
// once, by warp 0) meet in shared memory.
constexpr int kAdjThreads = 32 * kL;
#ifndef PWFA_ADJ_MIN_BLOCKS
#define PWFA_ADJ_MIN_BLOCKS 8
#endif

// The x = nx - 1 wall node of a row shares its block with the node it clamps
// to (x = nx - 2) unless it opens a new block of 32.
__host__ __device__ __forceinline__ bool xwall_split(int nx) { return (nx & 31) == 1; }

// Boundary nodes whose moment adjoints are produced by the shell pass: the
// two z walls (nx ny each), then per interior plane the rows y = 0 and
// y = ny - 1 (nx each) and, when the x = nx - 1 wall sits alone in its
// block, the column x = nx - 1 of the interior rows (ny - 2). The other
// x-wall nodes of interior rows are handled inside the interior pass, in
// the block of the node they clamp to.
__host__ __device__ __forceinline__ uint32_t shell_count(const Grid& g) {
    const uint32_t ring = 2u * (uint32_t)g.nx + (xwall_split(g.nx) ? (uint32_t)(g.ny - 2) : 0u);
    return 2u * (uint32_t)g.nx * (uint32_t)g.ny + (uint32_t)(g.nz - 2) * ring;
}

__device__ __forceinline__ void shell_node(const Grid& g, uint32_t idx, int& x, int& y, int& z) {
    const uint32_t nx = (uint32_t)g.nx, P = nx * (uint32_t)g.ny;
    if (idx < 2u * P) {
        z = idx < P ? 0 : g.nz - 1;
        const uint32_t r = idx < P ? idx : idx - P;
        y = (int)(r / nx);
        x = (int)(r - (uint32_t)y * nx);
        return;
    }
    idx -= 2u * P;
    const uint32_t M = 2u * nx + (xwall_split(g.nx) ? (uint32_t)(g.ny - 2) : 0u);
    const uint32_t k = idx / M;
    const uint32_t r = idx - k * M;
    z = 1 + (int)k;
    if (r < 2u * nx) {
        y = r < nx ? 0 : g.ny - 1;
        x = (int)(r < nx ? r : r - nx);
    } else {
        x = g.nx - 1;
        y = 1 + (int)(r - 2u * nx);
    }
}

// SHELL: the shell nodes above (open grids), writing their moment adjoints
// A_bar. Otherwise one block per 32 nodes of a row: interior nodes scatter
// their population adjoints, boundary nodes zero the slots they pulled.
template <int ST, int COLL, bool PER, bool SHELL>
__global__ void __launch_bounds__(kAdjThreads, PWFA_ADJ_MIN_BLOCKS) adj_fluid_kernel(const AdjArgs a,
                                                                                    uint32_t nshell) {
    using T = typename Codec<ST>::T;
    __shared__ float sA[kL][32];     // lattice sums A_l
    __shared__ float sG[kL][32];     // sum_i w_i S_bar_l,i
    __shared__ float sU[kL][3][32];  // lattice l's share of u_bar
    __shared__ float sN[4][3][32];   // node E, B sums at t_n and t_{n+1}, J_bar
    __shared__ float sAb[kL][32];    // node-level part of A_bar; then x-wall A_bar
    const StepArgs& s = a.f;
    const Grid& g = s.g;
    const int l = (int)(threadIdx.x >> 5);
    const int lane = (int)(threadIdx.x & 31);
    int x, y, z;
    bool live;
    if (SHELL) {
        const uint32_t item = blockIdx.x * 32u + (uint32_t)lane;
        live = item < nshell;
        x = y = z = 0;
        if (live) shell_node(g, item, x, y, z);
    } else {
        x = (int)blockIdx.x * 32 + lane;
        y = (int)blockIdx.y;
        z = (int)blockIdx.z;
        live = x < g.nx;
    }
    const uint32_t sxy = (uint32_t)g.nx * (uint32_t)g.ny;
    const uint32_t node = ((uint32_t)z * (uint32_t)g.ny + (uint32_t)y) * (uint32_t)g.nx + (uint32_t)x;
    const bool bnd = !PER && (x == 0 || y == 0 || z == 0 || x == g.nx - 1 || y == g.ny - 1 || z == g.nz - 1);
    const bool row_in = y >= 1 && y <= g.ny - 2 && z >= 1 && z <= g.nz - 2;
    const bool xwall = !PER && !SHELL && live && row_in && (x == 0 || (x == g.nx - 1 && lane != 0));
    const int64_t LS = lattice_stride(g);
    const float* __restrict__ mom = s.mom;
    const float* __restrict__ Sin = a.Sbar_in + l * LS;
    float* __restrict__ Sout = a.Sbar_out + l * LS;
    if (!SHELL && live && bnd) {
        // a boundary node's own pull slots are never read by the forward
        // step: their adjoint is zero
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const int sx = x - xi_x(q), sy = y - xi_y(q), sz = z - xi_z(q);
            if (!in_grid(g, sx, sy, sz)) continue;
            const uint32_t so = PWFA_CHECK(
                s.dbg, ((uint32_t)sz * (uint32_t)g.ny + (uint32_t)sy) * (uint32_t)g.nx + (uint32_t)sx, 0, g.Np, 7u);
            Sout[pop_off(q, so)] = 0.0f;
        }
    }
    const bool act = live && (SHELL || !bnd || xwall);
    // pulled node: the clamped interior node on open grids (Eq. 14)
    int xs = x, ys = y, zs = z;
    if (!PER) {
        xs = min(max(x, 1), g.nx - 2);
        ys = min(max(y, 1), g.ny - 2);
        zs = min(max(z, 1), g.nz - 2);
    }
    const uint32_t nodec = ((uint32_t)zs * (uint32_t)g.ny + (uint32_t)ys) * (uint32_t)g.nx + (uint32_t)xs;

    // ---- one memory round: this lattice's pulled populations and S_bar,
    // plus one of the node's field sums (or J_bar) per warp
    float S[kQ];
    float Al = 0.0f;
    const bool forced = (COLL != 2) && s.couple;
    if (act) {
#pragma unroll
        for (int q = 0; q < kQ; ++q) S[q] = __ldg(Sin + pop_off(q, node));
        // the lattice sum of the node's pulled populations, as the forward
        // step formed it (for a boundary node: of its clamped node's)
        Al = __ldg(mom + (int64_t)l * g.N + node);
        float v[3] = {0.0f, 0.0f, 0.0f};
        if (l == 0) { if (forced) node_E<PER>(g, s.E, x, y, z, v, s.dbg); }
        else if (l == 1) { if (forced) node_B_sum<PER>(g, s.Bc, x, y, z, v, s.dbg); }
        else if (l == 2) { if (forced) node_B_sum<PER>(g, s.Bn, x, y, z, v, s.dbg); }
        else { v[0] = a.Jbar[0][node]; v[1] = a.Jbar[1][node]; v[2] = a.Jbar[2][node]; }
#pragma unroll
        for (int c = 0; c < 3; ++c) sN[l][c][lane] = v[c];
    } else {
#pragma unroll
        for (int q = 0; q < kQ; ++q) S[q] = 0.0f;
    }
    sA[l][lane] = Al;
    __syncthreads();

    // ---- forward recompute of the node's velocity (every warp)
    const float A[kL] = {sA[0][lane], sA[1][lane], sA[2][lane], sA[3][lane]};
    const float n = A[0];
    const float nn = n > s.n_floor ? n : s.n_floor;
    const float inn = 1.0f / nn;
    const float p[3] = {A[1] * inn, A[2] * inn, A[3] * inn};
    const float gam = sqrtf(1.0f + p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    const float igam = 1.0f / gam;
    const float beta[3] = {p[0] * igam, p[1] * igam, p[2] * igam};
    const float u[3] = {beta[0] * s.lat, beta[1] * s.lat, beta[2] * s.lat};
    const float om = s.omega;
    const float k3 = 3.0f * (1.0f - om);
    // weight of d fs / d(A phi): omega for interior BGK, 0 for interior
    // stream-only, 1 for the regularized form and for boundary nodes
    const float wA = (COLL == 0 && !bnd) ? om : ((COLL == 2 && !bnd) ? 0.0f : 1.0f);
    const bool proj = COLL == 1 && !bnd;

    // ---- this lattice's reductions over the 19 directions
    // Gb = sum w S, P = sum w S xi, W = sum w S xi (xi.u) and
    // sphi = sum w S phi_i / w_i = base Gb + 3 u.P + 4.5 u.W (since
    // sum w S (xi.u)^2 = u.W): per direction only signed adds into the sums
    // of its weight class (axis 1/18, diagonal 1/36), weighted once at the end.
    float Gb, sphi, P[3], W[3];
    {
        float G1 = 0.0f, G2 = 0.0f, P1[3] = {0.0f, 0.0f, 0.0f}, P2[3] = {0.0f, 0.0f, 0.0f};
        float W1[3] = {0.0f, 0.0f, 0.0f}, W2[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int q = 1; q < kQ; ++q) {
            float xu = 0.0f;
            if (xi_x(q) > 0) xu += u[0]; else if (xi_x(q) < 0) xu -= u[0];
            if (xi_y(q) > 0) xu += u[1]; else if (xi_y(q) < 0) xu -= u[1];
            if (xi_z(q) > 0) xu += u[2]; else if (xi_z(q) < 0) xu -= u[2];
            const float sx = S[q] * xu;
            const bool diag = q > 6;
            float& G = diag ? G2 : G1;
            float* Pc = diag ? P2 : P1;
            float* Wc = diag ? W2 : W1;
            G += S[q];
            if (xi_x(q) > 0) { Pc[0] += S[q]; Wc[0] += sx; } else if (xi_x(q) < 0) { Pc[0] -= S[q]; Wc[0] -= sx; }
            if (xi_y(q) > 0) { Pc[1] += S[q]; Wc[1] += sx; } else if (xi_y(q) < 0) { Pc[1] -= S[q]; Wc[1] -= sx; }
            if (xi_z(q) > 0) { Pc[2] += S[q]; Wc[2] += sx; } else if (xi_z(q) < 0) { Pc[2] -= S[q]; Wc[2] -= sx; }
        }
        const float wa = 1.0f / 18.0f, wd = 1.0f / 36.0f;
        Gb = wq(0) * S[0] + wa * G1 + wd * G2;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            P[c] = wa * P1[c] + wd * P2[c];
            W[c] = wa * W1[c] + wd * W2[c];
        }
        const float base = 1.0f - 1.5f * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        sphi = base * Gb + 3.0f * (u[0] * P[0] + u[1] * P[1] + u[2] * P[2]) +
               4.5f * (u[0] * W[0] + u[1] * W[1] + u[2] * W[2]);
    }
    // u_bar share: d(A_l phi_i)/du through phi_i = w_i (base + 3 xi.u + 4.5 (xi.u)^2),
    // plus the regularized projection's -k3 A_l P_l
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float v = wA * Al * (3.0f * P[c] + 9.0f * W[c] - 3.0f * u[c] * Gb);
        if (proj) v -= k3 * Al * P[c];
        sU[l][c][lane] = v;
    }
    sG[l][lane] = Gb;
    // this lattice's own part of its moment adjoint
    float own = wA * sphi;
    if (proj) own -= k3 * (P[0] * u[0] + P[1] * u[1] + P[2] * u[2]);
    __syncthreads();

    // ---- node-level reverse, once per node (warp 0)
    if (l == 0 && act) {
        float e[3] = {0.0f, 0.0f, 0.0f}, b[3] = {0.0f, 0.0f, 0.0f}, F[3] = {0.0f, 0.0f, 0.0f};
        if (forced) {
            for (int c = 0; c < 3; ++c) {
                e[c] = sN[0][c][lane];
                b[c] = 0.125f * (sN[1][c][lane] + sN[2][c][lane]);
            }
            F[0] = -n * (e[0] + beta[1] * b[2] - beta[2] * b[1]);
            F[1] = -n * (e[1] + beta[2] * b[0] - beta[0] * b[2]);
            F[2] = -n * (e[2] + beta[0] * b[1] - beta[1] * b[0]);
        }
        const float ps[3] = {(A[1] + F[0] * s.dt) * inn, (A[2] + F[1] * s.dt) * inn, (A[3] + F[2] * s.dt) * inn};
        const float gs = sqrtf(1.0f + ps[0] * ps[0] + ps[1] * ps[1] + ps[2] * ps[2]);
        const float igs = 1.0f / gs;
        const float bs[3] = {ps[0] * igs, ps[1] * igs, ps[2] * igs};
        float Am[3], Fb[3];
        float nb, nnb = 0.0f;
        {
            // J = -n beta(p*)
            const float Jb[3] = {sN[3][0][lane], sN[3][1][lane], sN[3][2][lane]};
            nb = -(Jb[0] * bs[0] + Jb[1] * bs[1] + Jb[2] * bs[2]);
            const float v[3] = {-n * Jb[0], -n * Jb[1], -n * Jb[2]};
            const float bv = bs[0] * v[0] + bs[1] * v[1] + bs[2] * v[2];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float psb = (v[c] - bs[c] * bv) * igs;
                Am[c] = psb * inn;
                Fb[c] = psb * s.dt * inn;
                nnb -= psb * ps[c] * inn;
            }
        }
        // source w_i F dt of lattices 1..3
        if (COLL != 2) {
#pragma unroll
            for (int c = 0; c < 3; ++c) Fb[c] += sG[c + 1][lane] * s.dt;
        }
        float betab[3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            betab[c] = s.lat * (sU[0][c][lane] + sU[1][c][lane] + sU[2][c][lane] + sU[3][c][lane]);
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
        {
            // beta = p / gamma
            const float bbv = beta[0] * betab[0] + beta[1] * betab[1] + beta[2] * betab[2];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float pb = (betab[c] - beta[c] * bbv) * igam;
                Am[c] += pb * inn;
                nnb -= pb * p[c] * inn;
            }
        }
        if (n > s.n_floor) nb += nnb;
        sAb[0][lane] = nb;
        sAb[1][lane] = Am[0];
        sAb[2][lane] = Am[1];
        sAb[3][lane] = Am[2];
        for (int c = 0; c < 3; ++c) {
            a.ebar[c][node] = eb[c];
            a.bbar[c][node] = bb[c];
        }
    }
    __syncthreads();

    // ---- this lattice's moment adjoint
    float Ab = sAb[l][lane] + own;
    if (SHELL) {
        if (act) a.Abnd[l][node] = Ab;
        return;
    }
    if (xwall) sAb[l][lane] = Ab;  // handed to the node it clamps to
    __syncthreads();
    if (!act || bnd) return;
    // Boundary nodes that gathered at this node add their A_bar to every
    // population of the corresponding lattice: x-wall nodes of this row from
    // shared memory, the shell nodes from the shell pass.
    if (!PER && (x == 1 || y == 1 || z == 1 || x == g.nx - 2 || y == g.ny - 2 || z == g.nz - 2)) {
        int cx_[3], cy_[3], cz_[3];
        const int mx = wall_candidates(x, g.nx, cx_), my = wall_candidates(y, g.ny, cy_),
                  mz = wall_candidates(z, g.nz, cz_);
        for (int iz = 0; iz < mz; ++iz)
            for (int iy = 0; iy < my; ++iy)
                for (int ix = 0; ix < mx; ++ix) {
                    if (ix == 0 && iy == 0 && iz == 0) continue;
                    const int cx = cx_[ix];
                    if (iy == 0 && iz == 0 && !(cx == g.nx - 1 && xwall_split(g.nx))) {
                        Ab += sAb[l][cx == 0 ? lane - 1 : lane + 1];
                    } else {
                        const uint32_t bo =
                            ((uint32_t)cz_[iz] * (uint32_t)g.ny + (uint32_t)cy_[iy]) * (uint32_t)g.nx + (uint32_t)cx;
                        Ab += a.Abnd[l][bo];
                    }
                }
    }
    // transposed pull: f_i(x) = S_i(x - xi_i)  =>  S_bar_i(x - xi_i) = f_bar_i(x)
    const float mk[3] = {k3 * P[0], k3 * P[1], k3 * P[2]};
    auto fbar = [&](int q) {
        float fb = Ab;
        if (COLL == 0) fb += (1.0f - om) * S[q];
        else if (COLL == 2) fb += S[q];
        else fb += (float)xi_x(q) * mk[0] + (float)xi_y(q) * mk[1] + (float)xi_z(q) * mk[2];
        return fb;
    };
    if (!PER && (g.nx & 31) == 0) {
        // nx a multiple of 32: x - xi_i lies xi_y nx + xi_z nx ny nodes (a
        // whole number of 32-node chunks) from x - xi_x, and x -+ 1 crosses
        // into the neighbouring chunk only at its first / last lane; so each
        // slot is one of three per-node bases plus a per-direction shift
        constexpr uint32_t kC = kQ * 32u;  // elements of one chunk
        const uint32_t cy = (uint32_t)(g.nx >> 5) * kC, cz = (sxy >> 5) * kC;
        const uint32_t l0 = nodec & 31u;
        const uint32_t b0 = (nodec >> 5) * kC + l0;
        const uint32_t bsrc_p = l0 == 31u ? b0 + kC - 31u : b0 + 1u;  // xi_x = -1: the source is x + 1
        const uint32_t bsrc_m = l0 == 0u ? b0 - kC + 31u : b0 - 1u;   // xi_x = +1: the source is x - 1
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const uint32_t base = xi_x(q) > 0 ? bsrc_m : (xi_x(q) < 0 ? bsrc_p : b0);
            uint32_t off = base + (uint32_t)q * 32u;
            if (xi_y(q) > 0) off -= cy; else if (xi_y(q) < 0) off += cy;
            if (xi_z(q) > 0) off -= cz; else if (xi_z(q) < 0) off += cz;
            off = PWFA_CHECK(s.dbg, off, 0, (long long)kQ * g.Np, 7u);
            Sout[off] = fbar(q);
        }
    } else {
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            uint32_t src;
            if (PER) src = (uint32_t)src_index<true>(g, xs, ys, zs, q);
            else src = nodec - (uint32_t)(xi_x(q) + xi_y(q) * g.nx) - (uint32_t)xi_z(q) * sxy;
            src = PWFA_CHECK(s.dbg, src, 0, g.Np, 7u);
            Sout[pop_off(q, src)] = fbar(q);
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
    float sx, sy, sz;
    if (PER) {
        sx = r3_sum(rd<true>(g, bx, i, j, k), rd<true>(g, bx, i, j + 1, k), rd<true>(g, bx, i, j, k + 1),
                    rd<true>(g, bx, i, j + 1, k + 1), true, true, true);
        sy = r3_sum(rd<true>(g, by, i, j, k), rd<true>(g, by, i + 1, j, k), rd<true>(g, by, i, j, k + 1),
                    rd<true>(g, by, i + 1, j, k + 1), true, true, true);
        sz = r3_sum(rd<true>(g, bz, i, j, k), rd<true>(g, bz, i + 1, j, k), rd<true>(g, bz, i, j + 1, k),
                    rd<true>(g, bz, i + 1, j + 1, k), true, true, true);
    } else {
        const Nbr n = nbr_of(g, i, j, k);
        const float x0 = bx[o], x1 = bx[o + n.pj], x2 = bx[o + n.pk], x3 = bx[o + n.pj + n.pk];
        const float y0 = by[o], y1 = by[o + n.pi], y2 = by[o + n.pk], y3 = by[o + n.pi + n.pk];
        const float z0 = bz[o], z1 = bz[o + n.pi], z2 = bz[o + n.pj], z3 = bz[o + n.pi + n.pj];
        sx = r3_sum(x0, x1, x2, x3, n.jp, n.kp, n.jp && n.kp);
        sy = r3_sum(y0, y1, y2, y3, n.ip, n.kp, n.ip && n.kp);
        sz = r3_sum(z0, z1, z2, z3, n.ip, n.jp, n.ip && n.jp);
    }
    const float s3[3] = {sx, sy, sz};
    const float bn[3] = {a.Bnp[0][o], a.Bnp[1][o], a.Bnp[2][o]};
    for (int c = 0; c < 3; ++c) {
        const bool on = PER || act_B(g, c, i, j, k);
        const float bnt = bn[c] + s3[c];
        a.Bnp[c][o] = on ? bnt : 0.0f;
        a.Bbar[c][o] = on ? bnt + s3[c] : 0.0f;
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
    float bx, by, bz, by_k, bz_j, bx_k, bz_i, bx_j, by_i, e0, e1, e2;
    if (PER) {
        bx = rd<true>(g, Bx, i, j, k);
        by = rd<true>(g, By, i, j, k);
        bz = rd<true>(g, Bz, i, j, k);
        by_k = rd<true>(g, By, i, j, k - 1);
        bz_j = rd<true>(g, Bz, i, j - 1, k);
        bx_k = rd<true>(g, Bx, i, j, k - 1);
        bz_i = rd<true>(g, Bz, i - 1, j, k);
        bx_j = rd<true>(g, Bx, i, j - 1, k);
        by_i = rd<true>(g, By, i - 1, j, k);
        e0 = rd<true>(g, ex, i, j, k) + rd<true>(g, ex, i + 1, j, k);
        e1 = rd<true>(g, ey, i, j, k) + rd<true>(g, ey, i, j + 1, k);
        e2 = rd<true>(g, ez, i, j, k) + rd<true>(g, ez, i, j, k + 1);
    } else {
        const Nbr n = nbr_of(g, i, j, k);
        bx = Bx[o];
        by = By[o];
        bz = Bz[o];
        const float v0 = By[o - n.mk], v1 = Bz[o - n.mj], v2 = Bx[o - n.mk], v3 = Bz[o - n.mi], v4 = Bx[o - n.mj],
                    v5 = By[o - n.mi];
        const float x0 = ex[o], x1 = ex[o + n.pi], y0 = ey[o], y1 = ey[o + n.pj], z0 = ez[o], z1 = ez[o + n.pk];
        by_k = msk(n.km, v0);
        bz_j = msk(n.jm, v1);
        bx_k = msk(n.km, v2);
        bz_i = msk(n.im, v3);
        bx_j = msk(n.jm, v4);
        by_i = msk(n.im, v5);
        e0 = x0 + msk(n.ip, x1);
        e1 = y0 + msk(n.jp, y1);
        e2 = z0 + msk(n.kp, z1);
    }
    const float E0 = a.Ebar[0][o], E1 = a.Ebar[1][o], E2 = a.Ebar[2][o];
    const bool a0 = PER || act_E(g, 0, i, j, k);
    const bool a1 = PER || act_E(g, 1, i, j, k);
    const bool a2 = PER || act_E(g, 2, i, j, k);
    a.Ebar[0][o] = a0 ? r4_arith(c, E0, e0, by - by_k - bz + bz_j) : 0.0f;
    a.Ebar[1][o] = a1 ? r4_arith(c, E1, e1, -bx + bx_k + bz - bz_i) : 0.0f;
    a.Ebar[2][o] = a2 ? r4_arith(c, E2, e2, bx - bx_j - by + by_i) : 0.0f;
}

// ------------------------------------------------------------- R3 + R4
// R3 and R4 in one kernel. A block of kRX x kRY threads owns (kRX - 1) x
// (kRY - 1) columns and marches up kRZ planes, starting one plane below its
// slab. Each thread forms R3 at its column (lane 0 and row 0 are the -x / -y
// neighbour columns of the tile, evaluated again by their owners), so the
// new Bn_bar stays on chip: R4 takes the -x neighbour's by a shuffle, the
// -y neighbour's from shared memory (one barrier per plane, two buffers) and
// the -z one from the thread's registers. Nothing reads Bn_bar after R4, so
// it is not written back: 72 B per node against the separate kernels' 96.
// The plane above's b_bar_x, b_bar_y and e_bar_z that a plane reads are the
// next plane's own values (kept in registers), and each iteration issues the
// next plane's loads before it works on its own.
constexpr int kRX = 32, kRY = 8, kRZ = 16;
#ifndef PWFA_ADJ_FE_MIN_BLOCKS
#define PWFA_ADJ_FE_MIN_BLOCKS 4
#endif

// The loads of one plane of a column (o its index; pi, pj, pk its +1
// neighbour offsets): R3's b_bar_x, b_bar_y one plane up, b_bar_z and Bn_bar
// of the plane; R4's node-averaged E_bar (e_bar_z one plane up) and E_bar,
// for an owned node of the slab (e_bar_z one plane up for any owned node: the
// next plane takes it as its own).
struct AdjFEPlane {
    float x2, x3, y2, y3, z0, z1, z2, z3, bn0, bn1, bn2, ex0, ex1, ey0, ey1, ez1, E0, E1, E2;
};

__device__ __forceinline__ void adj_fe_load(const AdjArgs& a, int o, int pi, int pj, int pk, bool own, bool slab,
                                            AdjFEPlane& v) {
#ifdef PWFA_DEBUG
    o = (int)PWFA_CHECK(a.f.dbg, o, 0, a.f.g.N, 7u);
    pk = (int)PWFA_CHECK(a.f.dbg, o + pi + pj + pk, 0, a.f.g.N, 7u) - o - pi - pj;
#endif
    const float *bx = a.bbar[0], *by = a.bbar[1], *bz = a.bbar[2];
    v.x2 = __ldg(bx + o + pk);
    v.x3 = __ldg(bx + o + pj + pk);
    v.y2 = __ldg(by + o + pk);
    v.y3 = __ldg(by + o + pi + pk);
    v.z0 = __ldg(bz + o);
    v.z1 = __ldg(bz + o + pi);
    v.z2 = __ldg(bz + o + pj);
    v.z3 = __ldg(bz + o + pi + pj);
    v.bn0 = __ldg(a.Bnp[0] + o);
    v.bn1 = __ldg(a.Bnp[1] + o);
    v.bn2 = __ldg(a.Bnp[2] + o);
    v.ez1 = own ? __ldg(a.ebar[2] + o + pk) : 0.0f;
    if (slab) {
        v.ex0 = __ldg(a.ebar[0] + o);
        v.ex1 = __ldg(a.ebar[0] + o + pi);
        v.ey0 = __ldg(a.ebar[1] + o);
        v.ey1 = __ldg(a.ebar[1] + o + pj);
        v.E0 = a.Ebar[0][o];
        v.E1 = a.Ebar[1][o];
        v.E2 = a.Ebar[2][o];
    } else {
        v.ex0 = v.ex1 = v.ey0 = v.ey1 = v.E0 = v.E1 = v.E2 = 0.0f;
    }
}

template <bool PER>
__global__ void __launch_bounds__(kRX * kRY, PWFA_ADJ_FE_MIN_BLOCKS) adj_faces_edges_kernel(const AdjArgs a) {
    const Grid& g = a.f.g;
    const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny;
    __shared__ float sBx[2][kRY][kRX], sBz[2][kRY][kRX];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x = (int)blockIdx.x * (kRX - 1) + tx - 1, y = (int)blockIdx.y * (kRY - 1) + ty - 1;
    const bool own = tx > 0 && ty > 0 && x < nx && y < ny;
    // the evaluated column: wrapped (periodic) or clamped into the grid (an
    // open grid's clamped -1 column is masked by R4's bound below)
    const int xe = PER ? (x < 0 ? x + nx : x % nx) : min(max(x, 0), nx - 1);
    const int ye = PER ? (y < 0 ? y + ny : y % ny) : min(max(y, 0), ny - 1);
    // +1 neighbours (R3, R4's node averages) and -1 bounds (R4's curl)
    const bool ip = PER || xe + 1 < nx, jp = PER || ye + 1 < ny;
    const bool im = PER || x > 0, jm = PER || y > 0;
    const int pi = xe + 1 < nx ? 1 : (PER ? 1 - nx : 0);
    const int pj = ye + 1 < ny ? nx : (PER ? nx - nxy : 0);
    const float c = a.f.cdt;
    // the +z offset of plane kk (wrapped on a periodic grid, clamped on an
    // open one)
    auto zoff = [&](int kk) { return kk + 1 < nz ? nxy : (PER ? nxy - nz * nxy : 0); };

    const int kz0 = (int)blockIdx.z * kRZ, kend = min(kz0 + kRZ, nz);
    const int kfirst = PER || kz0 > 0 ? kz0 - 1 : kz0;
    int kk = kfirst < 0 ? kfirst + nz : kfirst;
    int o = (kk * ny + ye) * nx + xe;
    int pk = zoff(kk);
    // the first plane: b_bar_x, b_bar_y at the plane and e_bar_z (its
    // neighbours one plane up come with the plane's loads)
    float x0, x1, y0, y1, ez0;
    {
        int oc = o;
#ifdef PWFA_DEBUG
        oc = (int)PWFA_CHECK(a.f.dbg, oc + pi + pj, 0, g.N, 7u) - pi - pj;
#endif
        x0 = __ldg(a.bbar[0] + oc);
        x1 = __ldg(a.bbar[0] + oc + pj);
        y0 = __ldg(a.bbar[1] + oc);
        y1 = __ldg(a.bbar[1] + oc + pi);
        ez0 = own && kfirst >= kz0 ? __ldg(a.ebar[2] + oc) : 0.0f;
    }
    AdjFEPlane nxt;
    adj_fe_load(a, o, pi, pj, pk, own, own && kfirst >= kz0, nxt);
    float pbx = 0.0f, pby = 0.0f;  // new Bn_bar (x, y) of the plane below
    for (int k = kfirst; k < kend; ++k) {
        const int buf = (k - kfirst) & 1;
        const AdjFEPlane v = nxt;
        const bool slab = own && k >= kz0;
        const bool kp = PER || kk + 1 < nz, km = PER || kk > 0;
        // the next plane's loads, in flight while this one is worked on
        const int kn = PER && kk + 1 >= nz ? kk + 1 - nz : kk + 1;
        const int on = o + (kn > kk ? nxy : -kk * nxy);
        const int pkn = zoff(kn);
        if (k + 1 < kend) adj_fe_load(a, on, pi, pj, pkn, own, own && k + 1 >= kz0, nxt);
        // R3 at (xe, ye, kk)
        const float s3[3] = {r3_sum(x0, x1, v.x2, v.x3, jp, kp, jp && kp),
                             r3_sum(y0, y1, v.y2, v.y3, ip, kp, ip && kp),
                             r3_sum(v.z0, v.z1, v.z2, v.z3, ip, jp, ip && jp)};
        const float bn[3] = {v.bn0, v.bn1, v.bn2};
        float bnew[3];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            const bool on_c = PER || act_B(g, cc, xe, ye, kk);
            const float bnt = bn[cc] + s3[cc];
            bnew[cc] = on_c ? bnt : 0.0f;
            if (slab) a.Bbar[cc][o] = on_c ? bnt + s3[cc] : 0.0f;
        }
        // R4 at (x, y, kk): the -x neighbour's Bn_bar from lane - 1, the -y
        // neighbour's from row - 1, the -z one from the plane below
        const float bz_i = __shfl_up_sync(0xffffffffu, bnew[2], 1);
        const float by_i = __shfl_up_sync(0xffffffffu, bnew[1], 1);
        sBx[buf][ty][tx] = bnew[0];
        sBz[buf][ty][tx] = bnew[2];
        __syncthreads();
        if (slab) {
            const float bx_j = msk(jm, sBx[buf][ty - 1][tx]), bz_j = msk(jm, sBz[buf][ty - 1][tx]);
            const float bx_k = msk(km, pbx), by_k = msk(km, pby);
            const float bz_im = msk(im, bz_i), by_im = msk(im, by_i);
            const float e0 = v.ex0 + msk(ip, v.ex1), e1 = v.ey0 + msk(jp, v.ey1), e2 = ez0 + msk(kp, v.ez1);
            const float bxn = bnew[0], byn = bnew[1], bzn = bnew[2];
            const bool a0 = PER || act_E(g, 0, x, y, kk);
            const bool a1 = PER || act_E(g, 1, x, y, kk);
            const bool a2 = PER || act_E(g, 2, x, y, kk);
            a.Ebar[0][o] = a0 ? r4_arith(c, v.E0, e0, byn - by_k - bzn + bz_j) : 0.0f;
            a.Ebar[1][o] = a1 ? r4_arith(c, v.E1, e1, -bxn + bx_k + bzn - bz_im) : 0.0f;
            a.Ebar[2][o] = a2 ? r4_arith(c, v.E2, e2, bxn - bx_j - byn + by_im) : 0.0f;
        }
        pbx = bnew[0];
        pby = bnew[1];
        // this plane's values one plane up are the next plane's own
        x0 = v.x2;
        x1 = v.x3;
        y0 = v.y2;
        y1 = v.y3;
        ez0 = v.ez1;
        kk = kn;
        o = on;
        pk = pkn;
    }
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
            const float sb = Sbar0[pop_off(q, (uint32_t)node)];
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
    const Grid& g = a.f.g;
    const dim3 rows((unsigned)(g.nx + 31) / 32, (unsigned)g.ny, (unsigned)g.nz);
    if (g.periodic) {
        adj_fluid_kernel<ST, COLL, true, false><<<rows, kAdjThreads, 0, s>>>(a, 0u);
    } else {
        const uint32_t nb = shell_count(g);
        adj_fluid_kernel<ST, COLL, false, true><<<(nb + 31) / 32, kAdjThreads, 0, s>>>(a, nb);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        adj_fluid_kernel<ST, COLL, false, false><<<rows, kAdjThreads, 0, s>>>(a, 0u);
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

cudaError_t launch_adjoint_grad_finish(const double* gslots, double* grad, cudaStream_t s) {
    adj_grad_finish_kernel<<<1, 256, 0, s>>>(gslots, grad);
    return cudaGetLastError();
}

static AdjArgs with_driver_factors(const AdjArgs& a0) {
    AdjArgs a = a0;
    a.csr = a.f.alpha / (a.sr * a.sr * a.sr);
    a.csz = a.f.alpha / (a.sz * a.sz * a.sz);
    return a;
}

cudaError_t launch_adjoint_ampere(const AdjArgs& a0, cudaStream_t s) {
    const AdjArgs a = with_driver_factors(a0);
    const Grid& g = a.f.g;
    const dim3 block(kBX, kBY, 1);
    const dim3 grid((g.nx + kBX - 1) / kBX, (g.ny + kBY - 1) / kBY, (g.nz + kR1Planes - 1) / kR1Planes);
    if (a.f.couple) {
        if (g.periodic) adj_ampere_kernel<true><<<grid, block, 0, s>>>(a);
        else adj_ampere_kernel<false><<<grid, block, 0, s>>>(a);
    } else {
        // no Maxwell update: B, E pass through; J is not used
        cudaError_t e = cudaMemsetAsync(a.Jbar[0], 0, sizeof(float) * g.N, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(a.Jbar[1], 0, sizeof(float) * g.N, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(a.Jbar[2], 0, sizeof(float) * g.N, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t launch_adjoint_fluid(const AdjArgs& a0, int storage, int collision, cudaStream_t s) {
    const AdjArgs a = with_driver_factors(a0);
    switch (storage) {
        case 0: return launch_adj_fluid_s<0>(a, collision, s);
        case 1: return launch_adj_fluid_s<1>(a, collision, s);
        case 2: return launch_adj_fluid_s<2>(a, collision, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_adjoint_fields(const AdjArgs& a0, bool fused, cudaStream_t s) {
    const AdjArgs a = with_driver_factors(a0);
    if (!a.f.couple) return cudaSuccess;
    const Grid& g = a.f.g;
    const bool per = g.periodic;
    if (fused) {
        const dim3 tiles((unsigned)(g.nx + kRX - 2) / (kRX - 1), (unsigned)(g.ny + kRY - 2) / (kRY - 1),
                         (unsigned)(g.nz + kRZ - 1) / kRZ);
        const dim3 block(kRX, kRY, 1);
        if (per) adj_faces_edges_kernel<true><<<tiles, block, 0, s>>>(a);
        else adj_faces_edges_kernel<false><<<tiles, block, 0, s>>>(a);
        return cudaGetLastError();
    }
    const dim3 grid = grid_of(g, kBX, kBY), block(kBX, kBY, 1);
    if (per) adj_faces_kernel<true><<<grid, block, 0, s>>>(a);
    else adj_faces_kernel<false><<<grid, block, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (per) adj_edges_kernel<true><<<grid, block, 0, s>>>(a);
    else adj_edges_kernel<false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_step(const AdjArgs& a, int storage, int collision, cudaStream_t s) {
    cudaError_t e = launch_adjoint_ampere(a, s);
    if (e == cudaSuccess) e = launch_adjoint_fluid(a, storage, collision, s);
    if (e == cudaSuccess) e = launch_adjoint_fields(a, true, s);
    return e;
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
