// Yee FDTD field kernels of one step (bodies in fields_node.cuh): Faraday,
// Ampere (with the PIC deposit box), Ampere fused with the next step's
// Faraday, the moving window's field move and the wall-zeroing helper used
// after a state import.
#include "lbm_kernels.h"
#include "fields_fused.cuh"

namespace pwfa {

namespace {

// Block shape of the field kernels: 64 x 2 (128 threads) measured 2.5 %
// faster than 32 x 8 for Faraday and Ampere on the 512x256x256 grid
// (0.207 / 0.291 against 0.213 / 0.298 ms).
#ifndef PWFA_FIELD_BX
#define PWFA_FIELD_BX 64
#endif
#ifndef PWFA_FIELD_BY
#define PWFA_FIELD_BY 2
#endif
constexpr int kBX = PWFA_FIELD_BX;
constexpr int kBY = PWFA_FIELD_BY;

template <bool PER>
__global__ void __launch_bounds__(kBX * kBY) faraday_kernel(const StepArgs a) {
    const int i = blockIdx.x * kBX + threadIdx.x;
    const int j = blockIdx.y * kBY + threadIdx.y;
    if (i >= a.g.nx || j >= a.g.ny) return;
    faraday_node<PER>(a, i, j, blockIdx.z);
}

// Faraday with the field energy of its nodes: (|E|^2 + |Bc|^2)/2 at each
// node's index (the six staggered components stored there), summed in FP32
// over each warp (32 nodes) into energy[warp].
template <bool PER>
__global__ void __launch_bounds__(kBX * kBY) faraday_energy_kernel(const StepArgs a, float* energy) {
    const int i = blockIdx.x * kBX + threadIdx.x;
    const int j = blockIdx.y * kBY + threadIdx.y;
    float e2 = 0.0f;
    if (i < a.g.nx && j < a.g.ny) {
        faraday_node<PER>(a, i, j, blockIdx.z);
        const int64_t o = ((int64_t)blockIdx.z * a.g.ny + j) * a.g.nx + i;
        for (int c = 0; c < 3; ++c) {
            const float ev = __ldg(a.E[c] + o), bv = __ldg(a.Bc[c] + o);
            e2 += ev * ev + bv * bv;
        }
        e2 *= 0.5f;
    }
    for (int off = 16; off > 0; off >>= 1) e2 += __shfl_down_sync(0xffffffffu, e2, off);
    const int tid = threadIdx.y * kBX + threadIdx.x;
    if ((tid & 31) == 0) {
        const int64_t b = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        energy[b * (kBX * kBY / 32) + (tid >> 5)] = e2;
    }
}

template <bool PER>
__global__ void __launch_bounds__(kBX * kBY) ampere_kernel(const StepArgs a) {
    const int i = blockIdx.x * kBX + threadIdx.x;
    const int j = blockIdx.y * kBY + threadIdx.y;
    if (a.jbox_next && i == 0 && j == 0 && blockIdx.z == 0) {
        // the next step's deposit box starts empty
        a.jbox_next[0] = a.jbox_next[1] = a.jbox_next[2] = 0x7fffffff;
        a.jbox_next[3] = a.jbox_next[4] = a.jbox_next[5] = -1;
    }
    if (i >= a.g.nx || j >= a.g.ny) return;
    ampere_node<PER>(a, i, j, blockIdx.z, a.zc);
}

template <bool PER>
__global__ void __launch_bounds__(kAFX * kAFY, PWFA_AF_MIN_BLOCKS)
    ampere_faraday_kernel(const StepArgs a, const FieldPair out) {
    ampere_faraday_tile<PER>(a, out, blockIdx.x, blockIdx.y, blockIdx.z, a.zc);
}

__global__ void __launch_bounds__(kBX * kBY) zero_walls_kernel(const StepArgs a) {
    const Grid& g = a.g;
    const int i = blockIdx.x * kBX + threadIdx.x;
    const int j = blockIdx.y * kBY + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.nx || j >= g.ny) return;
    const int64_t o = ((int64_t)k * g.ny + j) * g.nx + i;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    if (!(i <= nx - 2 && j >= 1 && j <= ny - 2 && k >= 1 && k <= nz - 2)) a.Eout[0][o] = 0.0f;
    if (!(i >= 1 && i <= nx - 2 && j <= ny - 2 && k >= 1 && k <= nz - 2)) a.Eout[1][o] = 0.0f;
    if (!(i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2 && k <= nz - 2)) a.Eout[2][o] = 0.0f;
    float* Bc0 = const_cast<float*>(a.Bc[0]);
    float* Bc1 = const_cast<float*>(a.Bc[1]);
    float* Bc2 = const_cast<float*>(a.Bc[2]);
    if (!(i >= 1 && i <= nx - 2 && j <= ny - 2 && k <= nz - 2)) Bc0[o] = 0.0f;
    if (!(i <= nx - 2 && j >= 1 && j <= ny - 2 && k <= nz - 2)) Bc1[o] = 0.0f;
    if (!(i <= nx - 2 && j <= ny - 2 && k >= 1 && k <= nz - 2)) Bc2[o] = 0.0f;
}

// The moving window's field move: each thread moves kMovePlanes planes of its
// (x, y) column, with all 6 kMovePlanes loads issued before any store (one
// plane per thread left it latency-bound at 0.57 of the copy bandwidth).
// Every output element is written (moved value, or zero outside the
// conducting box).
constexpr int kMovePlanes = 4;

__global__ void __launch_bounds__(kBX * kBY) window_move_kernel(const WindowMove w) {
    const Grid& g = w.g;
    const int i = blockIdx.x * kBX + threadIdx.x;
    const int j = blockIdx.y * kBY + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const bool ix = i >= 1 && i <= nx - 2, jy = j >= 1 && j <= ny - 2;
    const bool xi = i <= nx - 2, yj = j <= ny - 2;
    float v[kMovePlanes][6];
#pragma unroll
    for (int p = 0; p < kMovePlanes; ++p) {
        const int k = blockIdx.z * kMovePlanes + p;
        const int64_t up = ((int64_t)(k + 1) * ny + j) * nx + i;
        const bool in = k + 1 < nz;
        const bool kz = k >= 1 && k <= nz - 2, zk = k <= nz - 2;
        const bool m[6] = {in && xi && jy && kz, in && ix && yj && kz, in && ix && jy && zk,
                           in && ix && yj && zk, in && xi && jy && zk, in && xi && yj && kz};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            v[p][c] = m[c] ? w.E[c][up] : 0.0f;
            v[p][3 + c] = m[3 + c] ? w.B[c][up] : 0.0f;
        }
    }
#pragma unroll
    for (int p = 0; p < kMovePlanes; ++p) {
        const int k = blockIdx.z * kMovePlanes + p;
        if (k >= nz) break;
        const int64_t o = ((int64_t)k * ny + j) * nx + i;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            w.Eo[c][o] = v[p][c];
            w.Bo[c][o] = v[p][3 + c];
        }
    }
}

}  // namespace

cudaError_t launch_window_move(const WindowMove& w, cudaStream_t s) {
    dim3 block(kBX, kBY, 1);
    dim3 grid((w.g.nx + kBX - 1) / kBX, (w.g.ny + kBY - 1) / kBY, (w.g.nz + kMovePlanes - 1) / kMovePlanes);
    window_move_kernel<<<grid, block, 0, s>>>(w);
    return cudaGetLastError();
}

cudaError_t launch_zero_walls(const StepArgs& a, cudaStream_t s) {
    dim3 block(kBX, kBY, 1);
    dim3 grid((a.g.nx + kBX - 1) / kBX, (a.g.ny + kBY - 1) / kBY, a.g.nz);
    zero_walls_kernel<<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

int64_t faraday_energy_records(const Grid& g) {
    return (int64_t)((g.nx + kBX - 1) / kBX) * ((g.ny + kBY - 1) / kBY) * g.nz * (kBX * kBY / 32);
}

cudaError_t launch_faraday(const StepArgs& a, cudaStream_t s, float* energy) {
    dim3 block(kBX, kBY, 1);
    dim3 grid((a.g.nx + kBX - 1) / kBX, (a.g.ny + kBY - 1) / kBY, a.g.nz);
    if (energy) {
        if (a.g.periodic) faraday_energy_kernel<true><<<grid, block, 0, s>>>(a, energy);
        else faraday_energy_kernel<false><<<grid, block, 0, s>>>(a, energy);
    } else if (a.g.periodic) faraday_kernel<true><<<grid, block, 0, s>>>(a);
    else faraday_kernel<false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

void fused_field_tiles(const Grid& g, int* tx, int* ty, int* tz) {
    *tx = (g.nx + kAFX - 2) / (kAFX - 1);
    *ty = (g.ny + kAFY - 2) / (kAFY - 1);
    *tz = (g.nz + kAFZ - 1) / kAFZ;
}

cudaError_t launch_ampere_faraday(const StepArgs& a, const FieldPair& out, cudaStream_t s) {
    if (a.Jb[0]) return cudaErrorInvalidValue;  // the PIC deposit is cleared by the plain Ampere kernel
    dim3 block(kAFX, kAFY, 1);
    dim3 grid((a.g.nx + kAFX - 2) / (kAFX - 1), (a.g.ny + kAFY - 2) / (kAFY - 1), (a.g.nz + kAFZ - 1) / kAFZ);
    if (a.g.periodic) ampere_faraday_kernel<true><<<grid, block, 0, s>>>(a, out);
    else ampere_faraday_kernel<false><<<grid, block, 0, s>>>(a, out);
    return cudaGetLastError();
}

cudaError_t launch_ampere(const StepArgs& a, cudaStream_t s) {
    dim3 block(kBX, kBY, 1);
    dim3 grid((a.g.nx + kBX - 1) / kBX, (a.g.ny + kBY - 1) / kBY, a.g.nz);
    if (a.g.periodic) ampere_kernel<true><<<grid, block, 0, s>>>(a);
    else ampere_kernel<false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pwfa
