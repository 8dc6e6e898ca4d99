// FP64 diagnostics of a caller-held state with no device allocation.
//
// Some callers cannot let a library call cudaMalloc: an in-situ analysis hook
// that runs between the time steps of another code, or a host application
// that owns a fixed device-memory budget through its own pool. For them
// cudaMalloc/cudaFree break the memory accounting and cudaFree synchronises
// the whole device, stalling their other streams. This entry point reduces a
// state that the caller already holds in device memory and writes the result
// to caller memory; its only scratch is the file-scope array below, which
// every GPU that loads the library keeps until the process exits.
#include <mutex>
#include <string>

#include "../../include/pwfa_lbm.h"
#include "lbm_device.cuh"

namespace pwfa {
int set_error(int code, const std::string& msg);  // api.cu
}

namespace {

constexpr int kThreads = 256;
constexpr int kNodesPerThread = 16;
constexpr int64_t kNodesPerBlock = (int64_t)kThreads * kNodesPerThread;  // 4096
constexpr int kMaxBlocks = 16384;                                         // 1 MiB of scratch
constexpr int kMaxDevices = 64;

// One record of 8 doubles per block; every call overwrites the records it
// uses, so nothing has to be cleared between calls.
static __device__ __align__(256) double g_diag_scratch[kMaxBlocks * 8];

struct Red {
    double sn, s1, s2, s3, en, mn, mb, bad;
};

__device__ __forceinline__ void red_combine(Red& a, const Red& b) {
    a.sn += b.sn; a.s1 += b.s1; a.s2 += b.s2; a.s3 += b.s3; a.en += b.en;
    a.mn = fmin(a.mn, b.mn); a.mb = fmax(a.mb, b.mb); a.bad += b.bad;
}

__device__ __forceinline__ Red red_shfl(const Red& d, int off) {
    Red r;
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

__device__ void red_block(Red d, double* dst) {
    __shared__ Red sh[kThreads / 32];
    for (int off = 16; off > 0; off >>= 1) red_combine(d, red_shfl(d, off));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = d;
    __syncthreads();
    if (warp == 0) {
        d = lane < kThreads / 32 ? sh[lane] : Red{0, 0, 0, 0, 0, 1e300, 0, 0};
        for (int off = 16; off > 0; off >>= 1) red_combine(d, red_shfl(d, off));
        if (lane == 0) {
            dst[0] = d.sn; dst[1] = d.s1; dst[2] = d.s2; dst[3] = d.s3;
            dst[4] = d.en; dst[5] = d.mn; dst[6] = d.mb; dst[7] = d.bad;
        }
    }
}

// Block b reduces nodes [b*4096, (b+1)*4096) of a state given as
// pre-collision populations f^n [4][19][N] and raw Yee E, B [3][N].
__global__ void __launch_bounds__(kThreads) diag_noalloc_kernel(int64_t N, double dxcube, float n_floor,
                                                                const float* __restrict__ f,
                                                                const float* __restrict__ E,
                                                                const float* __restrict__ B,
                                                                double* scratch) {
    Red d{0, 0, 0, 0, 0, 1e300, 0, 0};
    const int64_t base = (int64_t)blockIdx.x * kNodesPerBlock;
    for (int k = 0; k < kNodesPerThread; ++k) {
        const int64_t node = base + (int64_t)k * kThreads + threadIdx.x;
        if (node >= N) break;
        float A[pwfa::kL];
        for (int l = 0; l < pwfa::kL; ++l) {
            float s = 0.0f;
            for (int q = 0; q < pwfa::kQ; ++q) s += __ldg(f + (int64_t)(l * pwfa::kQ + q) * N + node);
            A[l] = s;
        }
        const float nn = A[0] > n_floor ? A[0] : n_floor;
        const float p0 = A[1] / nn, p1 = A[2] / nn, p2 = A[3] / nn;
        const float gam = sqrtf(1.0f + p0 * p0 + p1 * p1 + p2 * p2);
        const double b0 = p0 / gam, b1 = p1 / gam, b2 = p2 / gam;
        const bool fin = isfinite(A[0]) && isfinite(A[1]) && isfinite(A[2]) && isfinite(A[3]);
        d.bad += fin ? 0.0 : 1.0;
        d.sn += A[0]; d.s1 += A[1]; d.s2 += A[2]; d.s3 += A[3];
        d.mn = fmin(d.mn, (double)A[0]);
        d.mb = fmax(d.mb, sqrt(b0 * b0 + b1 * b1 + b2 * b2));
        double e2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            const double ev = __ldg(E + (int64_t)c * N + node), bv = __ldg(B + (int64_t)c * N + node);
            e2 += ev * ev + bv * bv;
        }
        d.en += 0.5 * e2 * dxcube;
    }
    red_block(d, scratch + 8 * (int64_t)blockIdx.x);
}

__global__ void __launch_bounds__(kThreads) diag_noalloc_finish(const double* scratch, int nblocks, double* out) {
    Red d{0, 0, 0, 0, 0, 1e300, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += kThreads) {
        const double* p = scratch + 8 * (int64_t)b;
        red_combine(d, Red{p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7]});
    }
    red_block(d, out);
}

// Device address of the scratch array, looked up once per device with that
// device current (the array's name is only a host-side stand-in).
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

int scratch_for_current_device(double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return pwfa::set_error(PWFA_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return pwfa::set_error(PWFA_ERR_CUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_diag_scratch);
        if (e != cudaSuccess)
            return pwfa::set_error(PWFA_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return PWFA_OK;
}

}  // namespace

extern "C" int pwfa_lbm_diag_noalloc(int32_t nx, int32_t ny, int32_t nz, double dx, double n_floor,
                                     const float* dev_f, const float* dev_E, const float* dev_B,
                                     double* dev_out, void* cuda_stream) {
    if (nx < 1 || ny < 1 || nz < 1) return pwfa::set_error(PWFA_ERR_PARAM, "nx, ny, nz must be >= 1");
    const int64_t N = (int64_t)nx * ny * nz;
    if (N > (int64_t)kMaxBlocks * kNodesPerBlock)
        return pwfa::set_error(PWFA_ERR_PARAM, "grid of " + std::to_string(N) + " nodes exceeds the "
                               "allocation-free diagnostics limit of " +
                               std::to_string((int64_t)kMaxBlocks * kNodesPerBlock) + " nodes");
    if (!dev_f || !dev_E || !dev_B || !dev_out) return pwfa::set_error(PWFA_ERR_PARAM, "null pointer argument");
    if (!(dx > 0)) return pwfa::set_error(PWFA_ERR_PARAM, "dx must be > 0");
    // as pwfa_lbm_create: 0 selects the default floor, a negative or NaN one is an error
    if (!(n_floor >= 0)) return pwfa::set_error(PWFA_ERR_PARAM, "n_floor must be >= 0");
    double* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int nblocks = (int)((N + kNodesPerBlock - 1) / kNodesPerBlock);
    const float floor_f = (float)(n_floor == 0 ? 1e-6 : n_floor);
    diag_noalloc_kernel<<<nblocks, kThreads, 0, s>>>(N, dx * dx * dx, floor_f, dev_f, dev_E, dev_B, scratch);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        diag_noalloc_finish<<<1, kThreads, 0, s>>>(scratch, nblocks, dev_out);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return pwfa::set_error(PWFA_ERR_CUDA, std::string("diag_noalloc: ") + cudaGetErrorString(e));
    return PWFA_OK;
}
