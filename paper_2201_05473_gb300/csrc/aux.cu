// Set-up, state exchange and diagnostics kernels (not on the per-step path).
#include "lbm_kernels.h"
#include "lbm_node.cuh"

namespace pwfa {

namespace {

constexpr int kBX = 32;
constexpr int kBY = 4;

__device__ __forceinline__ void node_xyz(const Grid& g, int64_t node, int& x, int& y, int& z) {
    const int64_t sxy = (int64_t)g.nx * g.ny;
    z = (int)(node / sxy);
    const int64_t r = node - (int64_t)z * sxy;
    y = (int)(r / g.nx);
    x = (int)(r - (int64_t)y * g.nx);
}

// Radial multiplier: linear between r_j = j rmax/(np-1), last value beyond.
__device__ double profile_at(const double* prof, int np, double rmax, double r) {
    if (np <= 0) return 1.0;
    if (np == 1 || r >= rmax) return prof[np - 1];
    const double h = rmax / (np - 1);
    const double t = r / h;
    int j = (int)floor(t);
    if (j >= np - 1) return prof[np - 1];
    const double fr = t - j;
    return (1.0 - fr) * prof[j] + fr * prof[j + 1];
}

// Stored array S with S_i(y) = f^0_i(y + xi_i): pulling it yields the plasma
// at rest f^0 = w_i n0 prof(r) (lattice 0) and 0 (momentum lattices). Open
// grids clamp y + xi_i to the interior (such entries are only pulled by
// interior nodes, for which the clamp is the identity). Every population
// node up to Np is written: the plane above the box (present with a moving
// window) keeps this fresh plasma for good.
template <int ST>
__global__ void init_kernel(Grid g, typename Codec<ST>::T* f, float n0, const double* prof, int np,
                            double rmax, double dx) {
    const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= g.Np) return;
    int x, y, z;
    node_xyz(g, node, x, y, z);
    const double xc = 0.5 * (g.nx - 1) * dx, yc = 0.5 * (g.ny - 1) * dx;
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        float n = n0;
        if (np > 0) {  // FP64 only where a profile is given
            int sx = x + xi_x(q), sy = y + xi_y(q);
            if (g.periodic) { sx = wrapi(sx, g.nx); sy = wrapi(sy, g.ny); }
            else { sx = min(max(sx, 1), g.nx - 2); sy = min(max(sy, 1), g.ny - 2); }
            const double rx = sx * dx - xc, ry = sy * dx - yc;
            n = (float)((double)n0 * profile_at(prof, np, rmax, sqrt(rx * rx + ry * ry)));
        }
        const uint32_t off = pop_off(q, (uint32_t)node);
        const int64_t LS = lattice_stride(g);
        Codec<ST>::store(f + pop_elem<ST>(0, off, LS), wq(q) * n, 0, q, n0);
#pragma unroll
        for (int l = 1; l < kL; ++l) Codec<ST>::store(f + pop_elem<ST>(l, off, LS), 0.0f, l, q, n0);
    }
}

// f^n at every node (boundary nodes: f^eq of the clamped interior node).
template <int ST, bool PER>
__global__ void __launch_bounds__(kBX * kBY) export_f_kernel(const StepArgs a, float* out) {
    using T = typename Codec<ST>::T;
    const Grid& g = a.g;
    const int x = blockIdx.x * kBX + threadIdx.x;
    const int y = blockIdx.y * kBY + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const int64_t node = ((int64_t)z * g.ny + y) * g.nx + x;
    float f[kL][kQ];
    bool bnd;
    gather<ST, PER>(g, static_cast<const T*>(a.fin), a.n0, x, y, z, f, bnd, 0u, a.dbg);
    if (!PER && bnd) {
        float A[kL], inn, beta[3], phi[kQ];
        node_moments(f, a.n_floor, A, inn, beta);
        const float u[3] = {beta[0] * a.lat, beta[1] * a.lat, beta[2] * a.lat};
        eq_factors(u, phi);
        for (int l = 0; l < kL; ++l)
            for (int q = 0; q < kQ; ++q) f[l][q] = A[l] * phi[q];
    }
#pragma unroll
    for (int l = 0; l < kL; ++l)
#pragma unroll
        for (int q = 0; q < kQ; ++q) out[(int64_t)(l * kQ + q) * g.N + node] = f[l][q];
}

// Inverse of the pull: S_i(y) = f^n_i(y + xi_i).
template <int ST>
__global__ void import_f_kernel(Grid g, const float* in, typename Codec<ST>::T* f, float n0) {
    const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= g.N) return;
    int x, y, z;
    node_xyz(g, node, x, y, z);
#pragma unroll 1
    for (int q = 0; q < kQ; ++q) {
        int sx = x + xi_x(q), sy = y + xi_y(q), sz = z + xi_z(q);
        if (g.periodic) { sx = wrapi(sx, g.nx); sy = wrapi(sy, g.ny); sz = wrapi(sz, g.nz); }
        else { sx = min(max(sx, 0), g.nx - 1); sy = min(max(sy, 0), g.ny - 1); sz = min(max(sz, 0), g.nz - 1); }
        const int64_t src = ((int64_t)sz * g.ny + sy) * g.nx + sx;
        for (int l = 0; l < kL; ++l)
            Codec<ST>::store(f + pop_elem<ST>(l, pop_off(q, (uint32_t)node), lattice_stride(g)),
                             in[(int64_t)(l * kQ + q) * g.N + src], l, q, n0);
    }
}

template <int ST, bool PER>
__global__ void __launch_bounds__(kBX * kBY) export_fields_kernel(const StepArgs a, unsigned mask, float* out) {
    using T = typename Codec<ST>::T;
    const Grid& g = a.g;
    const int x = blockIdx.x * kBX + threadIdx.x;
    const int y = blockIdx.y * kBY + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const int64_t node = ((int64_t)z * g.ny + y) * g.nx + x;
    float vals[16];
    if (mask & 0xE00Fu) {
        float f[kL][kQ];
        bool bnd;
        gather<ST, PER>(g, static_cast<const T*>(a.fin), a.n0, x, y, z, f, bnd, 0u, a.dbg);
        float A[kL], inn, beta[3];
        node_moments(f, a.n_floor, A, inn, beta);
        vals[0] = A[0];
        vals[1] = beta[0]; vals[2] = beta[1]; vals[3] = beta[2];
        vals[13] = A[1]; vals[14] = A[2]; vals[15] = A[3];
    }
    const bool raw = (mask >> 31) & 1u;
    if (mask & 0x70u) {
        if (raw) { for (int c = 0; c < 3; ++c) vals[4 + c] = a.E[c][node]; }
        else { float e[3]; node_E<PER>(g, a.E, x, y, z, e, a.dbg); for (int c = 0; c < 3; ++c) vals[4 + c] = e[c]; }
    }
    if (mask & 0x380u) {
        if (raw) { for (int c = 0; c < 3; ++c) vals[7 + c] = a.Bc[c][node]; }
        else { float b[3]; node_B_sum<PER>(g, a.Bc, x, y, z, b, a.dbg); for (int c = 0; c < 3; ++c) vals[7 + c] = 0.25f * b[c]; }
    }
    if (mask & 0x1C00u) { for (int c = 0; c < 3; ++c) vals[10 + c] = a.J[c][node]; }
    int slot = 0;
    for (int bit = 0; bit < 16; ++bit)
        if (mask & (1u << bit)) out[(int64_t)(slot++) * g.N + node] = vals[bit];
}

// ---------------------------------------------------------------- line cuts
// Values along z at transverse offset r (c/omega_p) from the axis in +x,
// bilinear between the four nodes around (x_c + r, y_c): slot 0 density n,
// slot 1 node-averaged E_z (each thread one z).
template <int ST, bool PER>
__global__ void linecut_kernel(const StepArgs a, double xr, float* out) {
    using T = typename Codec<ST>::T;
    const Grid& g = a.g;
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= g.nz) return;
    const double xs = xr / a.dx + 0.5 * (g.nx - 1), ys = 0.5 * (g.ny - 1);
    int x0 = (int)floor(xs), y0 = (int)floor(ys);
    x0 = min(max(x0, 0), g.nx - 2);
    y0 = min(max(y0, 0), g.ny - 2);
    const float fx = (float)(xs - x0), fy = (float)(ys - y0);
    float nsum = 0.0f, esum = 0.0f;
    for (int c = 0; c < 4; ++c) {
        const int x = x0 + (c & 1), y = y0 + (c >> 1);
        const float wgt = ((c & 1) ? fx : 1.0f - fx) * ((c >> 1) ? fy : 1.0f - fy);
        float f[kL][kQ];
        bool bnd;
        gather<ST, PER>(g, static_cast<const T*>(a.fin), a.n0, x, y, z, f, bnd, 0u, a.dbg);
        float A[kL], inn, beta[3];
        node_moments(f, a.n_floor, A, inn, beta);
        float e[3];
        node_E<PER>(g, a.E, x, y, z, e, a.dbg);
        nsum += wgt * A[0];
        esum += wgt * e[2];
    }
    out[z] = nsum;
    out[g.nz + z] = esum;
}

// ---------------------------------------------------------------- diagnostics
struct Diag {
    double sn, s1, s2, s3, en, mn, mb, bad;
};

__device__ __forceinline__ void diag_combine(Diag& a, const Diag& b) {
    a.sn += b.sn; a.s1 += b.s1; a.s2 += b.s2; a.s3 += b.s3; a.en += b.en;
    a.mn = fmin(a.mn, b.mn); a.mb = fmax(a.mb, b.mb); a.bad += b.bad;
}

__device__ __forceinline__ Diag diag_shfl(const Diag& d, int off) {
    Diag r;
    r.sn = __shfl_down_sync(0xffffffffu, d.sn, off);
    r.s1 = __shfl_down_sync(0xffffffffu, d.s1, off);
    r.s2 = __shfl_down_sync(0xffffffffu, d.s2, off);
    r.s3 = __shfl_down_sync(0xffffffffu, d.s3, off);
    r.en = __shfl_down_sync(0xffffffffu, d.en, off);
    r.mn = __shfl_down_sync(0xffffffffu, d.mn, off);
    r.mb = __shfl_down_sync(0xffffffffu, d.mb, off);
    r.bad = __shfl_down_sync(0xffffffffu, d.bad, off);
    return r;
}

// Block reduction (warp shuffles, then one warp over the warp results).
__device__ void diag_block_reduce(Diag d, double* dst) {
    __shared__ Diag sh[kDiagThreads / 32];
    for (int off = 16; off > 0; off >>= 1) diag_combine(d, diag_shfl(d, off));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = d;
    __syncthreads();
    if (warp == 0) {
        d = lane < kDiagThreads / 32 ? sh[lane] : Diag{0, 0, 0, 0, 0, 1e300, 0, 0};
        for (int off = 16; off > 0; off >>= 1) diag_combine(d, diag_shfl(d, off));
        if (lane == 0) {
            dst[0] = d.sn; dst[1] = d.s1; dst[2] = d.s2; dst[3] = d.s3;
            dst[4] = d.en; dst[5] = d.mn; dst[6] = d.mb; dst[7] = d.bad;
        }
    }
}

// Grid-stride over nodes; one partial record of 8 doubles per block.
template <int ST, bool PER>
__global__ void __launch_bounds__(kDiagThreads) diag_kernel(const StepArgs a, double dxcube, double* partials) {
    using T = typename Codec<ST>::T;
    const Grid& g = a.g;
    Diag d{0, 0, 0, 0, 0, 1e300, 0, 0};
    for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < g.N;
         node += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz(g, node, x, y, z);
        float f[kL][kQ];
        bool bnd;
        gather<ST, PER>(g, static_cast<const T*>(a.fin), a.n0, x, y, z, f, bnd, 0u, a.dbg);
        float A[kL], inn, beta[3];
        node_moments(f, a.n_floor, A, inn, beta);
        const bool fin = isfinite(A[0]) && isfinite(A[1]) && isfinite(A[2]) && isfinite(A[3]);
        d.bad += fin ? 0.0 : 1.0;
        d.sn += A[0]; d.s1 += A[1]; d.s2 += A[2]; d.s3 += A[3];
        d.mn = fmin(d.mn, (double)A[0]);
        d.mb = fmax(d.mb, sqrt((double)beta[0] * beta[0] + (double)beta[1] * beta[1] + (double)beta[2] * beta[2]));
        double e2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            const double ev = a.E[c][node], bv = a.Bc[c][node];
            e2 += ev * ev + bv * bv;
        }
        d.en += 0.5 * e2 * dxcube;
    }
    diag_block_reduce(d, partials + 8 * (int64_t)blockIdx.x);
}

__global__ void __launch_bounds__(kDiagThreads) diag_finish_kernel(const double* partials, int64_t nparts, double* out) {
    Diag d{0, 0, 0, 0, 0, 1e300, 0, 0};
    for (int64_t b = threadIdx.x; b < nparts; b += blockDim.x) {
        const double* p = partials + 8 * b;
        diag_combine(d, Diag{p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7]});
    }
    diag_block_reduce(d, out);
}

// Block b combines FP32 fluid records [b per, (b + 1) per) and energy
// records [b per_e, (b + 1) per_e) in FP64 into scratch[b]. A fluid record's
// slot 6 holds min(-|beta|^2) (3e38 when the warp had no node).
__global__ void __launch_bounds__(kDiagThreads) diag_chunk_kernel(const float* rec, int64_t nrec, int64_t per,
                                                                  const float* en, int64_t nen, int64_t per_e,
                                                                  double dxcube, double* scratch) {
    Diag d{0, 0, 0, 0, 0, 1e300, 0, 0};
    const int64_t b0 = (int64_t)blockIdx.x * per;
    const int64_t b1 = b0 + per < nrec ? b0 + per : nrec;
    for (int64_t b = b0 + threadIdx.x; b < b1; b += blockDim.x) {
        const float4 p = reinterpret_cast<const float4*>(rec)[2 * b];
        const float4 q = reinterpret_cast<const float4*>(rec)[2 * b + 1];
        diag_combine(d, Diag{p.x, p.y, p.z, p.w, q.x, q.y >= 3.0e38f ? 1e300 : (double)q.y,
                             sqrt(fmax(0.0, -(double)q.z)), q.w});
    }
    const int64_t e0 = (int64_t)blockIdx.x * per_e;
    const int64_t e1 = e0 + per_e < nen ? e0 + per_e : nen;
    for (int64_t b = e0 + threadIdx.x; b < e1; b += blockDim.x) d.en += en[b];
    d.en *= dxcube;
    diag_block_reduce(d, scratch + 8 * (int64_t)blockIdx.x);
}

dim3 node_grid(const Grid& g) { return dim3((g.nx + kBX - 1) / kBX, (g.ny + kBY - 1) / kBY, g.nz); }

// Witness slab: the x range [rows[2 j], rows[2 j + 1]) of each row j in plane
// k. One block sums E_z over it in FP64 (the slab holds at most a few
// thousand edges).
constexpr int kWitnessThreads = 256;
__global__ void __launch_bounds__(kWitnessThreads) witness_sum_kernel(Grid g, const float* Ez, int k,
                                                                      const int* rows, double* out) {
    double s = 0.0;
    const int64_t plane = (int64_t)k * g.nx * g.ny;
    for (int j = 0; j < g.ny; ++j) {
        const int lo = rows[2 * j], hi = rows[2 * j + 1];
        for (int i = lo + (int)threadIdx.x; i < hi; i += kWitnessThreads) s += Ez[plane + (int64_t)j * g.nx + i];
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    __shared__ double sh[kWitnessThreads / 32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kWitnessThreads / 32; ++w) t += sh[w];
        *out = t;
    }
}

// Ez_bar := value on the witness slab (the rest of the array is untouched).
__global__ void witness_seed_kernel(Grid g, float* Ezbar, int k, const int* rows, float value) {
    const int j = blockIdx.x;
    const int lo = rows[2 * j], hi = rows[2 * j + 1];
    const int64_t row = ((int64_t)k * g.ny + j) * g.nx;
    for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) Ezbar[row + i] = value;
}

}  // namespace

cudaError_t launch_witness_sum(const Grid& g, const float* Ez, int k, const int* rows, double* out, cudaStream_t s) {
    witness_sum_kernel<<<1, kWitnessThreads, 0, s>>>(g, Ez, k, rows, out);
    return cudaGetLastError();
}

cudaError_t launch_witness_seed(const Grid& g, float* Ezbar, int k, const int* rows, float value, cudaStream_t s) {
    witness_seed_kernel<<<g.ny, 128, 0, s>>>(g, Ezbar, k, rows, value);
    return cudaGetLastError();
}

cudaError_t launch_diag_finish_step(const DiagOut& d, int64_t nrec, cudaStream_t s) {
    int64_t chunks = (nrec + 1023) / 1024;
    if (chunks < 1) chunks = 1;
    if (chunks > kDiagBlocks) chunks = kDiagBlocks;
    const int64_t per = (nrec + chunks - 1) / chunks;
    const int64_t per_e = (d.nenergy + chunks - 1) / chunks;
    diag_chunk_kernel<<<(unsigned)chunks, kDiagThreads, 0, s>>>(d.records, nrec, per, d.energy, d.nenergy, per_e,
                                                                d.dxcube, d.scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_finish_kernel<<<1, kDiagThreads, 0, s>>>(d.scratch, chunks, d.out);
    return cudaGetLastError();
}

cudaError_t launch_init(const Grid& g, void* f, int storage, float n0, const double* d_profile, int n_profile,
                        double profile_rmax, double dx, cudaStream_t s) {
    const int threads = 256;
    const unsigned blocks = (unsigned)((g.Np + threads - 1) / threads);
    switch (storage) {
        case 0: init_kernel<0><<<blocks, threads, 0, s>>>(g, (float*)f, n0, d_profile, n_profile, profile_rmax, dx); break;
        case 1: init_kernel<1><<<blocks, threads, 0, s>>>(g, (__nv_bfloat16*)f, n0, d_profile, n_profile, profile_rmax, dx); break;
        case 2: init_kernel<2><<<blocks, threads, 0, s>>>(g, (__half*)f, n0, d_profile, n_profile, profile_rmax, dx); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_export_f(const StepArgs& a, int storage, float* out, cudaStream_t s) {
    const dim3 grid = node_grid(a.g), block(kBX, kBY, 1);
    const bool per = a.g.periodic;
    switch (storage) {
        case 0: if (per) export_f_kernel<0, true><<<grid, block, 0, s>>>(a, out); else export_f_kernel<0, false><<<grid, block, 0, s>>>(a, out); break;
        case 1: if (per) export_f_kernel<1, true><<<grid, block, 0, s>>>(a, out); else export_f_kernel<1, false><<<grid, block, 0, s>>>(a, out); break;
        case 2: if (per) export_f_kernel<2, true><<<grid, block, 0, s>>>(a, out); else export_f_kernel<2, false><<<grid, block, 0, s>>>(a, out); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_import_f(const Grid& g, const float* in, void* f, int storage, float n0, cudaStream_t s) {
    const int threads = 256;
    const unsigned blocks = (unsigned)((g.N + threads - 1) / threads);
    switch (storage) {
        case 0: import_f_kernel<0><<<blocks, threads, 0, s>>>(g, in, (float*)f, n0); break;
        case 1: import_f_kernel<1><<<blocks, threads, 0, s>>>(g, in, (__nv_bfloat16*)f, n0); break;
        case 2: import_f_kernel<2><<<blocks, threads, 0, s>>>(g, in, (__half*)f, n0); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_export_fields(const StepArgs& a, int storage, unsigned mask, float* out, cudaStream_t s) {
    const dim3 grid = node_grid(a.g), block(kBX, kBY, 1);
    const bool per = a.g.periodic;
    switch (storage) {
        case 0: if (per) export_fields_kernel<0, true><<<grid, block, 0, s>>>(a, mask, out); else export_fields_kernel<0, false><<<grid, block, 0, s>>>(a, mask, out); break;
        case 1: if (per) export_fields_kernel<1, true><<<grid, block, 0, s>>>(a, mask, out); else export_fields_kernel<1, false><<<grid, block, 0, s>>>(a, mask, out); break;
        case 2: if (per) export_fields_kernel<2, true><<<grid, block, 0, s>>>(a, mask, out); else export_fields_kernel<2, false><<<grid, block, 0, s>>>(a, mask, out); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_linecut(const StepArgs& a, int storage, double r, float* out, cudaStream_t s) {
    const int threads = 128;
    const unsigned blocks = (unsigned)((a.g.nz + threads - 1) / threads);
    const bool per = a.g.periodic;
    switch (storage) {
        case 0: if (per) linecut_kernel<0, true><<<blocks, threads, 0, s>>>(a, r, out); else linecut_kernel<0, false><<<blocks, threads, 0, s>>>(a, r, out); break;
        case 1: if (per) linecut_kernel<1, true><<<blocks, threads, 0, s>>>(a, r, out); else linecut_kernel<1, false><<<blocks, threads, 0, s>>>(a, r, out); break;
        case 2: if (per) linecut_kernel<2, true><<<blocks, threads, 0, s>>>(a, r, out); else linecut_kernel<2, false><<<blocks, threads, 0, s>>>(a, r, out); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_diag(const StepArgs& a, int storage, double dxcube, double* partials, double* out, cudaStream_t s) {
    const int64_t need = (a.g.N + kDiagThreads - 1) / kDiagThreads;
    const int blocks = (int)(need < kDiagBlocks ? need : kDiagBlocks);
    const bool per = a.g.periodic;
    switch (storage) {
        case 0: if (per) diag_kernel<0, true><<<blocks, kDiagThreads, 0, s>>>(a, dxcube, partials); else diag_kernel<0, false><<<blocks, kDiagThreads, 0, s>>>(a, dxcube, partials); break;
        case 1: if (per) diag_kernel<1, true><<<blocks, kDiagThreads, 0, s>>>(a, dxcube, partials); else diag_kernel<1, false><<<blocks, kDiagThreads, 0, s>>>(a, dxcube, partials); break;
        case 2: if (per) diag_kernel<2, true><<<blocks, kDiagThreads, 0, s>>>(a, dxcube, partials); else diag_kernel<2, false><<<blocks, kDiagThreads, 0, s>>>(a, dxcube, partials); break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_finish_kernel<<<1, kDiagThreads, 0, s>>>(partials, blocks, out);
    return cudaGetLastError();
}

}  // namespace pwfa
