// Host runtime of the 2D-axisymmetric form (pwfa_axi_* in
// include/pwfa_lbm.h): validation, one device arena, the per-step launch
// sequence (fused Faraday + fluid -> Ampere), state exchange and per-kernel
// timing.
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/pwfa_lbm.h"
#include "axi.h"

namespace pwfa {
int set_error(int code, const std::string& msg);  // api.cu
cudaError_t dev_alloc(void** p, size_t bytes);    // api.cu
int alloc_fail(const std::string& what);           // api.cu
}

using pwfa::set_error;

struct pwfa_axi {
    pwfa_axi_params p{};
    cudaStream_t stream = nullptr;
    int64_t N = 0, Np = 0;
    void* arena = nullptr;
    float* f[2] = {nullptr, nullptr};
    int fcur = 0;
    float* Am = nullptr;
    float* Ez = nullptr;
    float* Er = nullptr;
    float* Bt[2] = {nullptr, nullptr};
    int bcur = 0;
    float* Jz = nullptr;
    float* Jr = nullptr;
    float* staging = nullptr;  // 6 N floats for exports
    int64_t steps = 0;
    bool profiling = false;
    std::vector<cudaEvent_t> ev;   // pairs per kernel kind, per step (reused)
    std::vector<int> pending;      // kinds of the recorded pairs
    double ms[4] = {0, 0, 0, 0};
    int64_t launches[4] = {0, 0, 0, 0};
};

namespace {

#define AXI_CUDA(call, where)                                                                          \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return set_error(PWFA_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e_)); \
    } while (0)

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
constexpr int kPairs = 1024;

int validate(const pwfa_axi_params& p) {
    auto bad = [](const char* what) { return set_error(PWFA_ERR_PARAM, std::string("axisymmetric: ") + what); };
    if (p.nz < 3 || p.nr < 3) return bad("nz, nr must be >= 3");
    if ((int64_t)p.nz * p.nr * 27 >= ((int64_t)1 << 40)) return bad("grid too large");
    if (!(p.dx > 0) || !std::isfinite(p.dx)) return bad("dx must be > 0");
    if (!(p.dt >= 0) || !std::isfinite(p.dt)) return bad("dt must be >= 0 (0 = default)");
    const double dt = p.dt > 0 ? p.dt : 0.17628 * p.dx;
    if (p.couple && !(dt < p.dx / std::sqrt(2.0))) return bad("dt violates the 2D Yee Courant limit dx/sqrt(2)");
    if (!(p.tau > 0.5) || !std::isfinite(p.tau)) return bad("tau must be > 0.5");
    if (p.collision != PWFA_BGK && p.collision != PWFA_STREAM_ONLY) return bad("collision must be BGK or stream-only");
    if (p.couple < 0 || p.couple > 1) return bad("couple must be 0 or 1");
    if (!(p.n0 >= 0) || !std::isfinite(p.n0)) return bad("n0 must be >= 0");
    if (!(p.alpha >= 0) || !std::isfinite(p.alpha)) return bad("alpha must be >= 0");
    if (!(p.sigma_r > 0) || !(p.sigma_z > 0)) return bad("sigma_r and sigma_z must be > 0");
    if (!std::isfinite(p.z0)) return bad("z0 must be finite");
    if (!(p.n_floor >= 0)) return bad("n_floor must be >= 0");
    return PWFA_OK;
}

pwfa::axi::Args make_args(const pwfa_axi* h) {
    pwfa::axi::Args a{};
    const auto& p = h->p;
    a.nz = p.nz;
    a.nr = p.nr;
    a.N = h->N;
    a.Np = h->Np;
    a.fin = h->f[h->fcur];
    a.fout = h->f[1 - h->fcur];
    a.Am = h->Am;
    a.Ez = h->Ez;
    a.Er = h->Er;
    a.EzO = h->Ez;
    a.ErO = h->Er;
    a.Bt = h->Bt[h->bcur];
    a.Btn = h->Bt[1 - h->bcur];
    a.Jz = h->Jz;
    a.Jr = h->Jr;
    a.omega = (float)(1.0 / p.tau);
    a.lat = (float)(p.dt / p.dx);
    a.dt = (float)p.dt;
    a.cdt = (float)(p.dt / p.dx);
    a.dx = (float)p.dx;
    a.D = (float)((p.tau - 0.5) / 3.0 * p.dx * p.dx / p.dt);
    a.n_floor = (float)p.n_floor;
    a.n0 = (float)p.n0;
    a.couple = p.couple;
    a.collision = p.collision;
    a.alpha = (float)p.alpha;
    a.inv2sr2 = (float)(1.0 / (2.0 * p.sigma_r * p.sigma_r));
    a.inv2sz2 = (float)(1.0 / (2.0 * p.sigma_z * p.sigma_z));
    a.zc = (float)(p.z0 + (double)(h->steps + 1) * p.dt);
    return a;
}

template <class F>
int timed(pwfa_axi* h, int kind, const char* what, F&& launch) {
    if (h->profiling) {
        if ((int)h->pending.size() == kPairs) {
            AXI_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
            for (size_t i = 0; i < h->pending.size(); ++i) {
                float t = 0.0f;
                AXI_CUDA(cudaEventElapsedTime(&t, h->ev[2 * i], h->ev[2 * i + 1]), "cudaEventElapsedTime");
                h->ms[h->pending[i]] += t;
            }
            h->pending.clear();
        }
        const size_t i = h->pending.size();
        AXI_CUDA(cudaEventRecord(h->ev[2 * i], h->stream), "cudaEventRecord");
        AXI_CUDA(launch(), what);
        AXI_CUDA(cudaEventRecord(h->ev[2 * i + 1], h->stream), "cudaEventRecord");
        h->pending.push_back(kind);
    } else {
        AXI_CUDA(launch(), what);
    }
    ++h->launches[kind];
    return PWFA_OK;
}

// copies between a caller's [3][9][N] array (host or device) and the
// [3][9][Np] population planes, one plane at a time
int planes_to_user(pwfa_axi* h, const float* planes, float* user) {
    for (int lq = 0; lq < 27; ++lq)
        AXI_CUDA(cudaMemcpyAsync(user + (int64_t)lq * h->N, planes + (int64_t)lq * h->Np, sizeof(float) * h->N,
                                 cudaMemcpyDefault, h->stream), "cudaMemcpyAsync");
    return PWFA_OK;
}
int user_to_planes(pwfa_axi* h, const float* user, float* planes) {
    for (int lq = 0; lq < 27; ++lq)
        AXI_CUDA(cudaMemcpyAsync(planes + (int64_t)lq * h->Np, user + (int64_t)lq * h->N, sizeof(float) * h->N,
                                 cudaMemcpyDefault, h->stream), "cudaMemcpyAsync");
    return PWFA_OK;
}

}  // namespace

extern "C" {

int pwfa_axi_create(const pwfa_axi_params* params, void* cuda_stream, pwfa_axi_t** out) {
    if (!out) return set_error(PWFA_ERR_PARAM, "out is NULL");
    *out = nullptr;
    if (!params) return set_error(PWFA_ERR_PARAM, "params is NULL");
    int rc = validate(*params);
    if (rc) return rc;
    pwfa_axi* h = new (std::nothrow) pwfa_axi();
    if (!h) return set_error(PWFA_ERR_ALLOC, "host allocation failed");
    h->p = *params;
    if (h->p.dt == 0) h->p.dt = 0.17628 * h->p.dx;
    if (h->p.n_floor == 0) h->p.n_floor = 1e-6;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->N = (int64_t)h->p.nz * h->p.nr;
    h->Np = (h->N + 31) / 32 * 32;
    const size_t fbytes = align_up(sizeof(float) * 27 * (size_t)h->Np);
    const size_t vb = align_up(sizeof(float) * (size_t)h->N);
    const size_t total = 2 * fbytes + 3 * vb + 6 * vb + 6 * vb;  // f x2, moments, E 2 + B 2 + J 2, staging
    if (pwfa::dev_alloc((void**)&h->arena, total) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return pwfa::alloc_fail("cudaMalloc of the axisymmetric state failed");
    }
    char* b = static_cast<char*>(h->arena);
    h->f[0] = (float*)b; b += fbytes;
    h->f[1] = (float*)b; b += fbytes;
    h->Am = (float*)b; b += 3 * vb;
    char* fields = b;
    h->Ez = (float*)b; b += vb;
    h->Er = (float*)b; b += vb;
    h->Bt[0] = (float*)b; b += vb;
    h->Bt[1] = (float*)b; b += vb;
    h->Jz = (float*)b; b += vb;
    h->Jr = (float*)b; b += vb;
    h->staging = (float*)b;
    auto bail = [&](int code) {
        cudaFree(h->arena);
        delete h;
        return code;
    };
    if (cudaMemsetAsync(fields, 0, 6 * vb, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->f[1], 0, fbytes, h->stream) != cudaSuccess) {
        cudaGetLastError();
        return bail(set_error(PWFA_ERR_CUDA, "cudaMemsetAsync failed"));
    }
    pwfa::axi::Args a = make_args(h);
    cudaError_t e = pwfa::axi::launch_init(a, h->f[0], h->stream);
    if (e != cudaSuccess) return bail(set_error(PWFA_ERR_CUDA, std::string("init: ") + cudaGetErrorString(e)));
    h->ev.resize(2 * kPairs);
    for (auto& x : h->ev)
        if (cudaEventCreate(&x) != cudaSuccess) {
            cudaGetLastError();
            x = nullptr;
        }
    *out = h;
    return PWFA_OK;
}

int pwfa_axi_step(pwfa_axi_t* h, int32_t nsteps) {
    if (!h) return set_error(PWFA_ERR_PARAM, "null handle");
    if (nsteps < 0) return set_error(PWFA_ERR_PARAM, "nsteps must be >= 0");
    for (int32_t n = 0; n < nsteps; ++n) {
        pwfa::axi::Args a = make_args(h);
        int rc = PWFA_OK;
        // (Faraday's law runs inside the fluid kernel)
        rc = timed(h, 2, "axi fluid", [&] { return pwfa::axi::launch_fluid(a, h->stream); });
        if (rc == PWFA_OK && h->p.couple)
            rc = timed(h, 3, "axi ampere", [&] { return pwfa::axi::launch_ampere(a, h->stream); });
        if (rc) return rc;
        h->fcur = 1 - h->fcur;
        h->bcur = 1 - h->bcur;
        ++h->steps;
    }
    return PWFA_OK;
}

int pwfa_axi_fields(pwfa_axi_t* h, float* out) {
    if (!h || !out) return set_error(PWFA_ERR_PARAM, "null argument");
    pwfa::axi::Args a = make_args(h);
    const int64_t N = h->N;
    // moments of the current state, then n, beta_z, beta_r
    cudaError_t e = pwfa::axi::launch_moments(a, h->stream);
    if (e == cudaSuccess) e = pwfa::axi::launch_export_moments(a, h->staging, h->stream);
    if (e != cudaSuccess) return set_error(PWFA_ERR_CUDA, std::string("fields: ") + cudaGetErrorString(e));
    AXI_CUDA(cudaMemcpyAsync(h->staging + 3 * N, h->Ez, sizeof(float) * N, cudaMemcpyDeviceToDevice, h->stream), "copy");
    AXI_CUDA(cudaMemcpyAsync(h->staging + 4 * N, h->Er, sizeof(float) * N, cudaMemcpyDeviceToDevice, h->stream), "copy");
    AXI_CUDA(cudaMemcpyAsync(h->staging + 5 * N, h->Bt[h->bcur], sizeof(float) * N, cudaMemcpyDeviceToDevice, h->stream),
             "copy");
    AXI_CUDA(cudaMemcpyAsync(out, h->staging, sizeof(float) * 6 * N, cudaMemcpyDefault, h->stream), "copy");
    AXI_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return PWFA_OK;
}

int pwfa_axi_get_source(pwfa_axi_t* h, float* fs) {
    if (!h || !fs) return set_error(PWFA_ERR_PARAM, "null argument");
    int rc = planes_to_user(h, h->f[h->fcur], fs);
    if (rc) return rc;
    AXI_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return PWFA_OK;
}

int pwfa_axi_set_source(pwfa_axi_t* h, const float* fs) {
    if (!h || !fs) return set_error(PWFA_ERR_PARAM, "null argument");
    int rc = user_to_planes(h, fs, h->f[h->fcur]);
    if (rc) return rc;
    AXI_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return PWFA_OK;
}

int64_t pwfa_axi_steps_done(pwfa_axi_t* h) {
    if (!h) return set_error(PWFA_ERR_PARAM, "null handle");
    return h->steps;
}

int pwfa_axi_profile(pwfa_axi_t* h, int32_t enable) {
    if (!h) return set_error(PWFA_ERR_PARAM, "null handle");
    for (auto x : h->ev)
        if (!x) return set_error(PWFA_ERR_CUDA, "profiling events unavailable");
    h->profiling = enable != 0;
    return PWFA_OK;
}

int pwfa_axi_kernel_times(pwfa_axi_t* h, double* ms, int64_t* launches) {
    if (!h) return set_error(PWFA_ERR_PARAM, "null handle");
    AXI_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    for (size_t i = 0; i < h->pending.size(); ++i) {
        float t = 0.0f;
        AXI_CUDA(cudaEventElapsedTime(&t, h->ev[2 * i], h->ev[2 * i + 1]), "cudaEventElapsedTime");
        h->ms[h->pending[i]] += t;
    }
    h->pending.clear();
    for (int k = 0; k < 4; ++k) {
        if (ms) ms[k] = h->ms[k];
        if (launches) launches[k] = h->launches[k];
        h->ms[k] = 0.0;
        h->launches[k] = 0;
    }
    return PWFA_OK;
}

int pwfa_axi_destroy(pwfa_axi_t* h) {
    if (!h) return PWFA_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    for (auto x : h->ev)
        if (x) cudaEventDestroy(x);
    if (h->arena) cudaFree(h->arena);
    delete h;
    return PWFA_OK;
}

}  // extern "C"
