// Fused fluid kernel of one time step: the hot path of the method (the
// per-node body is in fluid_node.cuh).
//
// Memory traffic per node: 76 population reads + 76 writes (FP32: 608 B),
// E (one edge per component) + two B time levels (36 B) read, J (12 B)
// written; neighbouring edge/face reads hit L1/L2.
#include <algorithm>

#include "lbm_kernels.h"
#include "fluid_node.cuh"

namespace pwfa {

namespace {

template <int ST, int COLL, bool PER>
__global__ void __launch_bounds__(PWFA_FLUID_MAX_THREADS, FluidOcc<ST, COLL>::blocks) fluid_kernel(const StepArgs a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.g.nx || y >= a.g.ny) return;
    fluid_node<ST, COLL, PER>(a, x, y, blockIdx.z);
}

// The same step with the diagnostics of the entering state fused in: each
// warp writes one FP32 record of 8 slots (sum n, sum n p_x, p_y, p_z, field
// energy / dx^3 when fields is set, min n, min of -|beta|^2, non-finite
// count) to records[warp]; launch_diag_finish_step combines the records in
// FP64. A warp's sums run over 32 nodes, so FP32 costs them ~1e-7 relative;
// FP64 arithmetic, slow on this part, and block barriers stay out of this
// kernel.
__device__ __forceinline__ float diag_comb(int slot, float a, float b) {
    return (slot == 5 || slot == 6) ? fminf(a, b) : a + b;
}

// Warp reduction of 8 values per lane by recursive halving: at offsets 16, 8
// and 4 a lane keeps the half of its slots chosen by that lane bit and
// combines it with the partner's copy (4 + 2 + 1 shuffles), which leaves lane
// L with slot (L >> 2) & 7 reduced over 8 lanes; offsets 2 and 1 finish it.
// Nine shuffles instead of the forty of eight separate tree reductions.
__device__ __forceinline__ float diag8_warp(const float (&v)[8], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float keep = b4 ? v[k + 4] : v[k];
        const float send = b4 ? v[k] : v[k + 4];
        w[k] = diag_comb(b4 ? k + 4 : k, keep, __shfl_xor_sync(0xffffffffu, send, 16));
    }
    float u[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float keep = b3 ? w[j + 2] : w[j];
        const float send = b3 ? w[j] : w[j + 2];
        u[j] = diag_comb((b4 ? 4 : 0) + (b3 ? 2 : 0) + j, keep, __shfl_xor_sync(0xffffffffu, send, 8));
    }
    const int slot = (lane >> 2) & 7;
    float s = diag_comb(slot, b2 ? u[1] : u[0], __shfl_xor_sync(0xffffffffu, b2 ? u[0] : u[1], 4));
    s = diag_comb(slot, s, __shfl_xor_sync(0xffffffffu, s, 2));
    return diag_comb(slot, s, __shfl_xor_sync(0xffffffffu, s, 1));
}

template <int ST, int COLL, bool PER>
__global__ void __launch_bounds__(PWFA_FLUID_MAX_THREADS, FluidOcc<ST, COLL>::blocks)
    fluid_diag_kernel(const StepArgs a, int fields, float* records) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    float v[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 3.0e38f, 3.0e38f, 0.0f};
    if (x < a.g.nx && y < a.g.ny) {
        NodeDiag nd;
        fluid_node<ST, COLL, PER, true>(a, x, y, z, &nd);
        if (fields) {
            const int64_t o = ((int64_t)z * a.g.ny + y) * a.g.nx + x;
            float e2 = 0.0f;
            for (int c = 0; c < 3; ++c) {
                const float ev = __ldg(a.E[c] + o), bv = __ldg(a.Bc[c] + o);
                e2 += ev * ev + bv * bv;
            }
            v[4] = 0.5f * e2;
        }
        const bool fin = isfinite(nd.n) && isfinite(nd.a1) && isfinite(nd.a2) && isfinite(nd.a3);
        v[0] = nd.n; v[1] = nd.a1; v[2] = nd.a2; v[3] = nd.a3;
        v[5] = nd.n;
        v[6] = -nd.beta2;
        v[7] = fin ? 0.0f : 1.0f;
    }
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31;
    const float s = diag8_warp(v, lane);
    if ((lane & 3) == 0) {
        const int64_t b = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        const int64_t w = b * ((blockDim.x * blockDim.y) >> 5) + (tid >> 5);
        records[8 * w + (lane >> 2)] = s;
    }
}

// ---------------------------------------------------------------- staged
// Software-pipelined variant: persistent CTAs of 128 threads walk the node
// tiles; while a thread computes its node of tile k from registers, the
// pulled populations of its node of tile k+1 are already in flight into its
// own column of shared memory through 4-byte cp.async copies (76 values in
// FP32, 38 words of lattice pairs in the 16-bit forms). A thread reads back
// only the words it copied itself, so the only wait is cp.async.wait_group
// on its own copies (no barrier, no spin).
constexpr int kStageThreads = 128;
template <int ST>
constexpr int stage_words() { return ST == 0 ? kPop : kPop / 2; }

__device__ __forceinline__ void cp_async4(uint32_t smem, const void* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

struct TileNode {
    int x, y, z;
    bool valid;
};

__device__ __forceinline__ TileNode tile_node(const StepArgs& a, int64_t tile, int tiles_x, int tiles_y) {
    const int64_t per_plane = (int64_t)tiles_x * tiles_y;
    const int z = (int)(tile / per_plane);
    const int r = (int)(tile - (int64_t)z * per_plane);
    const int ty = r / tiles_x;
    const int tx = r - ty * tiles_x;
    TileNode n;
    n.x = tx * a.bx + (int)threadIdx.x % a.bx;
    n.y = ty * (kStageThreads / a.bx) + (int)threadIdx.x / a.bx;
    n.z = z;
    n.valid = n.x < a.g.nx && n.y < a.g.ny;
    return n;
}

// Word (l, q) of a thread's column: FP32 word l * 19 + q is f_l,q; 16-bit
// word p * 19 + q holds lattices 2p and 2p + 1 of direction q.
template <int ST, bool PER>
__device__ __forceinline__ void stage_copies(const StepArgs& a, const TileNode& n, uint32_t col) {
    const Grid& g = a.g;
    int xs = n.x, ys = n.y, zs = n.z;
    if (!PER) {
        xs = min(max(n.x, 1), g.nx - 2);
        ys = min(max(n.y, 1), g.ny - 2);
        zs = min(max(n.z, 1), g.nz - 2);
    }
    using T = typename Codec<ST>::T;
    const T* fin = static_cast<const T*>(a.fin);
    const int64_t LS = lattice_stride(g);
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        const uint32_t off = pop_off(q, (uint32_t)src_index<PER>(g, xs, ys, zs, q));
        if constexpr (ST == 0) {
#pragma unroll
            for (int l = 0; l < kL; ++l)
                cp_async4(col + 4u * (uint32_t)((l * kQ + q) * kStageThreads), fin + l * LS + off);
        } else {
#pragma unroll
            for (int p = 0; p < 2; ++p)
                cp_async4(col + 4u * (uint32_t)((p * kQ + q) * kStageThreads), fin + 2 * p * LS + 2 * off);
        }
    }
}

template <int ST, int COLL, bool PER>
__global__ void __launch_bounds__(kStageThreads, 4) fluid_staged_kernel(const StepArgs a, int tiles_x, int tiles_y,
                                                                         int64_t ntiles) {
    extern __shared__ uint32_t stage[];  // [stage_words<ST>()][kStageThreads]
    const uint32_t col = (uint32_t)__cvta_generic_to_shared(stage + threadIdx.x);
    int64_t tile = blockIdx.x;
    TileNode cur = tile_node(a, tile, tiles_x, tiles_y);
    if (tile < ntiles && cur.valid) stage_copies<ST, PER>(a, cur, col);
    cp_async_commit();
    while (tile < ntiles) {
        cp_async_wait_all();
        float f[kL][kQ];
        if constexpr (ST == 0) {
#pragma unroll
            for (int l = 0; l < kL; ++l)
#pragma unroll
                for (int q = 0; q < kQ; ++q)
                    f[l][q] = __uint_as_float(stage[(l * kQ + q) * kStageThreads + threadIdx.x]);
        } else {
#pragma unroll
            for (int p = 0; p < 2; ++p)
#pragma unroll
                for (int q = 0; q < kQ; ++q)
                    Codec<ST>::from_word(stage[(p * kQ + q) * kStageThreads + threadIdx.x], 2 * p, q, a.n0,
                                         f[2 * p][q], f[2 * p + 1][q]);
        }
        const int64_t nxt = tile + gridDim.x;
        const TileNode nn = tile_node(a, nxt, tiles_x, tiles_y);
        if (nxt < ntiles && nn.valid) stage_copies<ST, PER>(a, nn, col);
        cp_async_commit();
        if (cur.valid) {
            bool bnd = false;
            if (!PER)
                bnd = cur.x == 0 || cur.y == 0 || cur.z == 0 || cur.x == a.g.nx - 1 || cur.y == a.g.ny - 1 ||
                      cur.z == a.g.nz - 1;
            fluid_compute<ST, COLL, PER>(a, cur.x, cur.y, cur.z, f, bnd);
        }
        tile = nxt;
        cur = nn;
    }
}

template <int ST, int COLL>
cudaError_t launch_staged_t(const StepArgs& a, cudaStream_t s) {
    const int bx = a.bx;
    if (bx <= 0 || kStageThreads % bx) return cudaErrorInvalidConfiguration;
    const int by = kStageThreads / bx;
    const int tiles_x = (a.g.nx + bx - 1) / bx, tiles_y = (a.g.ny + by - 1) / by;
    const int64_t ntiles = (int64_t)tiles_x * tiles_y * a.g.nz;
    static int grid_cache[2] = {0, 0};
    int& grid = grid_cache[a.g.periodic ? 1 : 0];
    const size_t smem = sizeof(uint32_t) * stage_words<ST>() * kStageThreads;
    if (grid == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaError_t e = a.g.periodic
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fluid_staged_kernel<ST, COLL, true>, kStageThreads,
                                                            smem)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fluid_staged_kernel<ST, COLL, false>, kStageThreads,
                                                            smem);
        if (e != cudaSuccess) return e;
        grid = sms * (per_sm > 0 ? per_sm : 1);
    }
    const int blocks = (int)std::min<int64_t>(grid, ntiles);
    if (a.g.periodic)
        fluid_staged_kernel<ST, COLL, true><<<blocks, kStageThreads, smem, s>>>(a, tiles_x, tiles_y, ntiles);
    else
        fluid_staged_kernel<ST, COLL, false><<<blocks, kStageThreads, smem, s>>>(a, tiles_x, tiles_y, ntiles);
    return cudaGetLastError();
}

template <int ST, int COLL>
cudaError_t launch_fluid_t(const StepArgs& a, cudaStream_t s, const DiagOut* d) {
    // (a window-moving step pulls one plane up: direct kernel)
    if (a.staged && !d && a.src_shift == 0) return launch_staged_t<ST, COLL>(a, s);
    const int bx = a.bx, by = a.by;
    if (bx * by > PWFA_FLUID_MAX_THREADS || bx <= 0 || by <= 0 || (bx * by) % 32) return cudaErrorInvalidConfiguration;
    dim3 block(bx, by, 1);
    dim3 grid((a.g.nx + bx - 1) / bx, (a.g.ny + by - 1) / by, a.g.nz);
    if (d) {
        const int64_t nrec = (int64_t)grid.x * grid.y * grid.z * (bx * by / 32);
        if (nrec > d->capacity) return cudaErrorInvalidValue;
        const int fields = d->nenergy > 0 ? 0 : 1;
        if (a.g.periodic) fluid_diag_kernel<ST, COLL, true><<<grid, block, 0, s>>>(a, fields, d->records);
        else fluid_diag_kernel<ST, COLL, false><<<grid, block, 0, s>>>(a, fields, d->records);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return launch_diag_finish_step(*d, nrec, s);
    }
    if (a.g.periodic) fluid_kernel<ST, COLL, true><<<grid, block, 0, s>>>(a);
    else fluid_kernel<ST, COLL, false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

template <int ST>
cudaError_t launch_fluid_s(const StepArgs& a, int collision, cudaStream_t s, const DiagOut* d) {
    switch (collision) {
        case 0: return launch_fluid_t<ST, 0>(a, s, d);
        case 1: return launch_fluid_t<ST, 1>(a, s, d);
        case 2: return launch_fluid_t<ST, 2>(a, s, d);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_fluid(const StepArgs& a, int storage, int collision, cudaStream_t s, const DiagOut* d) {
    switch (storage) {
        case 0: return launch_fluid_s<0>(a, collision, s, d);
        case 1: return launch_fluid_s<1>(a, collision, s, d);
        case 2: return launch_fluid_s<2>(a, collision, s, d);
    }
    return cudaErrorInvalidValue;
}

}  // namespace pwfa
