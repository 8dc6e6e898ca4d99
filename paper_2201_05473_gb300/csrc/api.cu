// Host runtime of the C ABI declared in include/pwfa_lbm.h: parameter
// validation, one device arena per instance, the per-step launch sequence
// (Faraday -> fused fluid -> Ampere), state exchange and diagnostics.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <atomic>
#include <cstdlib>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pwfa_lbm.h"
#include "lbm_adjoint.h"
#include "lbm_batch.h"
#include "lbm_kernels.h"

using namespace pwfa;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    return fail(PWFA_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// NVTX range over a public call (named in profiler timelines).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

#define PWFA_CUDA(call, where)                          \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

size_t storage_bytes(int st) { return st == PWFA_F32 ? 4 : 2; }


constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Instance {
    pwfa_lbm_params p{};
    std::vector<double> profile;
    Grid g{};
    void* arena = nullptr;
    void* f[2] = {nullptr, nullptr};
    int fcur = 0;
    float* E[3] = {nullptr, nullptr, nullptr};
    float* Ealt[3] = {nullptr, nullptr, nullptr};  // second E buffer: moving window, fused field step
    // B of the next step already computed (by the fused Ampere-Faraday kernel)
    // in the other B buffer: the next step skips its Faraday launch
    bool lookahead = false;
    float* Jb[3] = {nullptr, nullptr, nullptr};    // PIC driver: deposited current
    float* particles = nullptr;                    // PIC driver: [6][np]
    int* jbox = nullptr;                           // PIC driver: deposit boxes of the two step parities
    int64_t np = 0;
    double pweight = 0.0;
    float* B[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    int bcur = 0;
    float* J[3] = {nullptr, nullptr, nullptr};
    double* d_profile = nullptr;
    int* d_wrows = nullptr;     // witness slab: x range of each row (2 ny ints)
    double* d_wout = nullptr;   // witness slab: FP64 sum of E_z
    unsigned* d_dbg = nullptr;  // debug builds: index-error word (site, index, count)
    int64_t steps = 0;
    int bx = 64, by = 2;  // fluid kernel block shape (pwfa_lbm_autotune refines it)
    int variant = PWFA_FLUID_DIRECT;  // fluid kernel variant
    // recording for the adjoint: checkpoints every K steps (+ the final
    // state), one segment of per-step states, adjoint scratch
    struct Recording {
        int64_t T = 0;
        int K = 0, ncp = 0;
        bool valid = false;
        void* cp = nullptr;
        size_t cp_stride = 0;
        void* seg = nullptr;
        size_t seg_stride = 0;
        void* adj = nullptr;
        int filled = -1;  // segment whose per-step slots already hold its steps
    } rec;
};

}  // namespace

namespace pwfa {
// Record the calling thread's error message for pwfa_lbm_last_error (used by
// entry points defined in other translation units).
int set_error(int code, const std::string& msg) { return fail(code, msg); }

// Every device allocation of the library goes through here. Fault injection
// for tests: with PWFA_FAIL_ALLOC_AT=n in the environment, the n-th
// allocation of the process (counting from 1) fails as an out-of-memory
// cudaMalloc would, so that each failure path can be exercised without
// exhausting the device.
namespace {
std::atomic<long> g_alloc_count{0};
}
namespace {
thread_local cudaError_t t_alloc_error = cudaSuccess;  // of the calling thread's last dev_alloc
}
cudaError_t dev_alloc(void** p, size_t bytes) {
    const long k = ++g_alloc_count;
    if (const char* v = std::getenv("PWFA_FAIL_ALLOC_AT")) {
        if (std::atol(v) == k) {
            *p = nullptr;
            return t_alloc_error = cudaErrorMemoryAllocation;
        }
    }
    return t_alloc_error = cudaMalloc(p, bytes);
}
// The status of a failed dev_alloc: PWFA_ERR_ALLOC when the device had no
// room, PWFA_ERR_CUDA when the runtime refused the call for another reason
// (for instance while the caller captures the stream into a graph); the
// message names the CUDA error. Clears the runtime's last error.
int alloc_fail(const std::string& what) {
    const cudaError_t e = t_alloc_error;
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? PWFA_ERR_ALLOC : PWFA_ERR_CUDA,
                what + " (" + cudaGetErrorString(e) + ")");
}
}  // namespace pwfa

struct pwfa_lbm {
    std::vector<Instance> inst;
    cudaStream_t stream = nullptr;
    double* d_partials = nullptr;  // kDiagBlocks x 8 doubles
    double* d_diag = nullptr;      // 8 doubles
    void* staging = nullptr;       // device buffer for host-side exchanges
    size_t staging_bytes = 0;
    // per-kernel timing
    bool profiling = false;
    std::vector<cudaEvent_t> events;          // pool, used in start/stop pairs
    std::vector<int> pending_kind;            // kind of each recorded pair
    double ms[PWFA_KERNEL_KINDS] = {};
    int64_t launches[PWFA_KERNEL_KINDS] = {};
    // Ampere fused with the next step's Faraday (rigid driver, no window):
    // PWFA_FUSION_OFF / _AUTO (grids of kFuseMinNodes and more) / _ON
    int field_fusion = PWFA_FUSION_AUTO;
    // batched path (several homogeneous instances, one launch per phase)
    bool batching = true;
    bool batch_valid = false;
    bool batch_fused = false;          // the table was built for the fused field step
    BatchEntry* d_entries = nullptr;   // instance table (capacity: entries_cap)
    int64_t* d_steps = nullptr;        // two driver step counters per instance
    int entries_cap = 0;
    uint16_t* d_tile_inst = nullptr;   // instance of each fluid tile, then of each fused-field tile
    int64_t tile_inst_cap = 0;
    BatchLaunch blaunch{};
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph2 = nullptr;  // two steps (both parities)
    // fused per-step diagnostics: per-block records and per-instance results
    float* d_step_records = nullptr;  // fused-diagnostics records (fluid blocks, then Faraday blocks)
    int64_t step_records_cap = 0;
    int64_t step_energy_cap = 0;
    double* d_step_scratch = nullptr;  // kDiagBlocks FP64 records of the two-level reduction
    double* d_step_diag = nullptr;
};

namespace {

// Planes the moving window has advanced after n steps: the window starts
// when the driver centre z0 + t passes window_z and then keeps it there.
int64_t window_planes_at(const pwfa_lbm_params& p, int64_t n) {
    if (!p.moving_window) return 0;
    const double v = std::floor((p.z0 + (double)n * p.dt - p.window_z) / p.dx);
    return v > 0.0 ? (int64_t)v : 0;
}

int validate(const pwfa_lbm_params& p, int idx) {
    char buf[256];
    auto bad = [&](const char* what) {
        std::snprintf(buf, sizeof buf, "instance %d: %s", idx, what);
        return fail(PWFA_ERR_PARAM, buf);
    };
    if (p.nx < 3 || p.ny < 3 || p.nz < 3) return bad("nx, ny, nz must be >= 3");
    if ((int64_t)p.nx * p.ny > (int64_t)1 << 30 || p.nz > 65535) return bad("grid too large");
    // one lattice's 19 planes (plus the window's fresh plane) are addressed
    // with 32-bit element offsets
    if (((int64_t)p.nx * p.ny * (p.nz + 1) + 31) / 32 * 32 * 19 >= ((int64_t)1 << 32))
        return bad("grid too large (nodes * 19 >= 2^32)");
    if (!(p.dx > 0) || !std::isfinite(p.dx)) return bad("dx must be > 0");
    if (!(p.dt >= 0) || !std::isfinite(p.dt)) return bad("dt must be >= 0 (0 = default)");
    const double dt = p.dt > 0 ? p.dt : 0.17628 * p.dx;
    if (p.couple && !(dt < p.dx / std::sqrt(3.0))) return bad("dt violates the Yee Courant limit dx/sqrt(3)");
    if (!(p.tau > 0.5) || !std::isfinite(p.tau)) return bad("tau must be > 0.5");
    if (p.collision < 0 || p.collision > 2) return bad("unknown collision operator");
    if (p.storage < 0 || p.storage > 2) return bad("unknown storage format");
    if (p.boundary < 0 || p.boundary > 1) return bad("unknown boundary mode");
    if (p.couple < 0 || p.couple > 1) return bad("couple must be 0 or 1");
    if (!(p.n0 >= 0) || !std::isfinite(p.n0)) return bad("n0 must be >= 0");
    if (p.n_profile < 0) return bad("n_profile must be >= 0");
    if (p.n_profile > 0 && !p.profile) return bad("profile is NULL but n_profile > 0");
    if (p.n_profile >= 2 && !(p.profile_rmax > 0)) return bad("profile_rmax must be > 0");
    for (int i = 0; i < p.n_profile; ++i)
        if (!(p.profile[i] >= 0) || !std::isfinite(p.profile[i])) return bad("profile values must be finite and >= 0");
    if (!(p.alpha >= 0) || !std::isfinite(p.alpha)) return bad("alpha must be >= 0");
    if (!(p.sigma_r > 0) || !(p.sigma_z > 0)) return bad("sigma_r and sigma_z must be > 0");
    if (!std::isfinite(p.z0)) return bad("z0 must be finite");
    if (!(p.n_floor >= 0)) return bad("n_floor must be >= 0");
    if (p.moving_window < 0 || p.moving_window > 1) return bad("moving_window must be 0 or 1");
    if (p.moving_window && p.boundary != PWFA_OPEN) return bad("the moving window needs the open boundary");
    if (p.moving_window && !std::isfinite(p.window_z)) return bad("window_z must be finite");
    if (p.driver != PWFA_DRIVER_RIGID && p.driver != PWFA_DRIVER_PIC) return bad("unknown driver");
    if (p.driver == PWFA_DRIVER_PIC && p.moving_window) return bad("the PIC driver does not support the moving window");
    return PWFA_OK;
}

int check_instance(pwfa_lbm* h, int32_t i) {
    if (!h) return fail(PWFA_ERR_PARAM, "null handle");
    if (i < 0 || i >= (int32_t)h->inst.size()) return fail(PWFA_ERR_PARAM, "instance index out of range");
    return PWFA_OK;
}

StepArgs make_args(const Instance& in) {
    StepArgs a{};
    a.g = in.g;
    a.fin = in.f[in.fcur];
    a.fout = in.f[1 - in.fcur];
    const int bc = in.bcur, bn = 1 - in.bcur;
    for (int c = 0; c < 3; ++c) {
        a.E[c] = in.E[c];
        a.Eout[c] = in.E[c];
        a.Bc[c] = in.B[bc][c];
        a.Bn[c] = in.B[bn][c];
        a.J[c] = in.J[c];
    }
    const pwfa_lbm_params& p = in.p;
    a.omega = (float)(1.0 / p.tau);
    a.lat = (float)(p.dt / p.dx);
    a.dt = (float)p.dt;
    a.cdt = (float)(p.dt / p.dx);
    a.n_floor = (float)p.n_floor;
    a.n0 = (float)p.n0;
    a.couple = p.couple;
    a.alpha = (float)p.alpha;
    a.inv2sr2 = (float)(1.0 / (2.0 * p.sigma_r * p.sigma_r));
    a.inv2sz2 = (float)(1.0 / (2.0 * p.sigma_z * p.sigma_z));
    // driver centre at t_{n+1}, in box coordinates
    const int64_t w1 = window_planes_at(p, in.steps + 1);
    a.zc = (float)(p.z0 + (double)(in.steps + 1) * p.dt - (double)w1 * p.dx);
    a.src_shift = w1 > window_planes_at(p, in.steps) ? (uint32_t)(in.g.nx * in.g.ny) : 0u;
    a.dx = (float)p.dx;
    a.bx = in.bx;
    a.by = in.by;
    a.staged = in.variant == PWFA_FLUID_STAGED && in.bx * in.by == 128;
    a.dbg = in.d_dbg;
    for (int c = 0; c < 3; ++c) a.Jb[c] = in.Jb[c];
    a.jbox = in.jbox ? in.jbox + 6 * (in.steps & 1) : nullptr;
    a.jbox_next = in.jbox ? in.jbox + 6 * ((in.steps + 1) & 1) : nullptr;
    return a;
}

bool is_device_ptr(const void* ptr) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

int ensure_staging(pwfa_lbm* h, size_t bytes) {
    if (h->staging_bytes >= bytes) return PWFA_OK;
    if (h->staging) cudaFree(h->staging);
    h->staging = nullptr;
    h->staging_bytes = 0;
    if (dev_alloc((void**)&h->staging, bytes) != cudaSuccess) {
        cudaGetLastError();
        return alloc_fail("cudaMalloc of the staging buffer failed");
    }
    h->staging_bytes = bytes;
    return PWFA_OK;
}

void free_recording(Instance& in) {
    if (in.rec.cp) cudaFree(in.rec.cp);
    if (in.rec.seg) cudaFree(in.rec.seg);
    if (in.rec.adj) cudaFree(in.rec.adj);
    in.rec = Instance::Recording{};
}

void free_instance(Instance& in) {
    free_recording(in);
    if (in.particles) cudaFree(in.particles);
    in.particles = nullptr;
    if (in.jbox) cudaFree(in.jbox);
    in.jbox = nullptr;
    if (in.arena) cudaFree(in.arena);
    in.arena = nullptr;
}

// Instances whose Ampere launch can take the next step's Faraday along: the
// rigid driver (the PIC deposit is cleared by the plain Ampere kernel) and
// a fixed box (a window move rewrites the B buffer the fused kernel fills).
bool fusable(const pwfa_lbm_params& p) {
    return p.couple && p.driver == PWFA_DRIVER_RIGID && !p.moving_window;
}

// The fused kernel marches 16 planes per block, so small grids give it too
// few blocks: on the GB300 it was slower up to 192x96x96 (1.8 M nodes: 225
// against 223 us per step; 64x32x32: 27 against 18 us) and faster from
// 256x128x128 (4.2 M nodes: 485 against 488 us; 512x256x256: 1.2 %).
constexpr int64_t kFuseMinNodes = (int64_t)4 << 20;

// Zero guard in front of every Yee/current array a step kernel reads: on an
// open grid the node averages read the -1 neighbours in x, y and z without
// bounds checks (one x-y plane, one row and one element before index 0 at
// the lowest node), and every component on or outside the conducting walls
// is kept at zero, so those reads see zeros and stay inside the array's own
// allocation.
size_t guard_bytes(const Grid& g) {
    return align_up(((size_t)g.nx * g.ny + g.nx + 1) * sizeof(float));
}

int alloc_instance(Instance& in, cudaStream_t s) {
    const int64_t N = in.g.N;
    const size_t fbytes = align_up((size_t)in.g.Np * kPop * storage_bytes(in.p.storage));
    const size_t pad = guard_bytes(in.g);
    const size_t vbytes = pad + align_up((size_t)N * sizeof(float));
    const size_t pbytes = align_up(sizeof(double) * (in.profile.empty() ? 1 : in.profile.size()));
    const size_t wbytes = align_up(sizeof(int) * 2 * (size_t)in.g.ny) + align_up(sizeof(double)) + kAlign;
    // E 3, B 2x3, J 3 (+ a second E for the window move or the fused field
    // step, + the PIC driver's current)
    const bool ealt = in.p.moving_window || fusable(in.p);
    const int nvec = 12 + (ealt ? 3 : 0) + (in.p.driver == PWFA_DRIVER_PIC ? 3 : 0);
    const size_t total = 2 * fbytes + nvec * vbytes + pbytes + wbytes;
    if (dev_alloc((void**)&in.arena, total) != cudaSuccess) {
        cudaGetLastError();
        in.arena = nullptr;
        char buf[160];
        std::snprintf(buf, sizeof buf, "cudaMalloc of %.3f GB for one instance failed", total / 1e9);
        return alloc_fail(buf);
    }
    char* base = static_cast<char*>(in.arena);
    in.f[0] = base; base += fbytes;
    in.f[1] = base; base += fbytes;
    char* fields = base;
    for (int c = 0; c < 3; ++c) { in.E[c] = (float*)(base + pad); base += vbytes; }
    for (int t = 0; t < 2; ++t)
        for (int c = 0; c < 3; ++c) { in.B[t][c] = (float*)(base + pad); base += vbytes; }
    for (int c = 0; c < 3; ++c) { in.J[c] = (float*)(base + pad); base += vbytes; }
    if (ealt)
        for (int c = 0; c < 3; ++c) { in.Ealt[c] = (float*)(base + pad); base += vbytes; }
    if (in.p.driver == PWFA_DRIVER_PIC)
        for (int c = 0; c < 3; ++c) { in.Jb[c] = (float*)(base + pad); base += vbytes; }
    in.d_profile = (double*)base;
    base += pbytes;
    in.d_wrows = (int*)base;
    in.d_wout = (double*)(base + align_up(sizeof(int) * 2 * (size_t)in.g.ny));
    in.d_dbg = (unsigned*)(base + align_up(sizeof(int) * 2 * (size_t)in.g.ny) + align_up(sizeof(double)));
    if (in.p.driver == PWFA_DRIVER_PIC) {
        // deposit boxes of both step parities, empty
        const int empty[12] = {0x7fffffff, 0x7fffffff, 0x7fffffff, -1, -1, -1,
                               0x7fffffff, 0x7fffffff, 0x7fffffff, -1, -1, -1};
        if (dev_alloc((void**)&in.jbox, sizeof empty) != cudaSuccess) {
            cudaGetLastError();
            return alloc_fail("cudaMalloc of the deposit boxes failed");
        }
        PWFA_CUDA(cudaMemcpy(in.jbox, empty, sizeof empty, cudaMemcpyHostToDevice), "cudaMemcpy");
    }
    // Fields, currents, their guards and the second population buffer
    // start at zero.
    PWFA_CUDA(cudaMemsetAsync(in.f[1], 0, fbytes, s), "cudaMemsetAsync");
    PWFA_CUDA(cudaMemsetAsync(fields, 0, nvec * vbytes, s), "cudaMemsetAsync");
    PWFA_CUDA(cudaMemsetAsync(in.d_dbg, 0, kAlign, s), "cudaMemsetAsync");
    if (!in.profile.empty())
        PWFA_CUDA(cudaMemcpyAsync(in.d_profile, in.profile.data(), sizeof(double) * in.profile.size(),
                                  cudaMemcpyHostToDevice, s),
                  "cudaMemcpyAsync profile");
    // both ping-pong buffers carry the fresh-plasma plane above the box that
    // a moving window pulls from
    for (int b = 0; b < (in.p.moving_window ? 2 : 1); ++b)
        PWFA_CUDA(launch_init(in.g, in.f[b], in.p.storage, (float)in.p.n0, in.d_profile, (int)in.profile.size(),
                              in.p.profile_rmax, in.p.dx, s),
                  "init kernel");
    return PWFA_OK;
}

constexpr size_t kEventPairs = 2048;

// Fold the recorded event pairs into the per-kind accumulators.
int fold_events(pwfa_lbm* h) {
    if (h->pending_kind.empty()) return PWFA_OK;
    PWFA_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    for (size_t k = 0; k < h->pending_kind.size(); ++k) {
        float t = 0.0f;
        PWFA_CUDA(cudaEventElapsedTime(&t, h->events[2 * k], h->events[2 * k + 1]), "cudaEventElapsedTime");
        h->ms[h->pending_kind[k]] += t;
    }
    h->pending_kind.clear();
    return PWFA_OK;
}

// Launch one kernel, bracketed by an event pair when profiling.
template <class F>
int timed_launch(pwfa_lbm* h, int kind, const char* what, F&& launch) {
    if (h->profiling) {
        if (h->pending_kind.size() == kEventPairs) {
            int rc = fold_events(h);
            if (rc) return rc;
        }
        const size_t k = h->pending_kind.size();
        PWFA_CUDA(cudaEventRecord(h->events[2 * k], h->stream), "cudaEventRecord");
        PWFA_CUDA(launch(), what);
        PWFA_CUDA(cudaEventRecord(h->events[2 * k + 1], h->stream), "cudaEventRecord");
        h->pending_kind.push_back(kind);
    } else {
        PWFA_CUDA(launch(), what);
    }
    ++h->launches[kind];
    return PWFA_OK;
}

// Back to the initial condition (t = 0): populations of the plasma at
// rest, zero fields and currents.
int reset_instance(Instance& in, cudaStream_t s) {
    const int64_t N = in.g.N;
    for (int c = 0; c < 3; ++c) {
        PWFA_CUDA(cudaMemsetAsync(in.E[c], 0, sizeof(float) * N, s), "cudaMemsetAsync");
        PWFA_CUDA(cudaMemsetAsync(in.J[c], 0, sizeof(float) * N, s), "cudaMemsetAsync");
        for (int t = 0; t < 2; ++t) PWFA_CUDA(cudaMemsetAsync(in.B[t][c], 0, sizeof(float) * N, s), "cudaMemsetAsync");
    }
    in.fcur = 0;
    in.bcur = 0;
    in.steps = 0;
    in.lookahead = false;
    PWFA_CUDA(launch_init(in.g, in.f[0], in.p.storage, (float)in.p.n0, in.d_profile, (int)in.profile.size(),
                          in.p.profile_rmax, in.p.dx, s),
              "init kernel");
    return PWFA_OK;
}

// ---------------------------------------------------------------- batched
bool batch_eligible(const pwfa_lbm* h) {
    if (!h->batching || h->inst.size() < 2 || h->inst.size() > (size_t)kMaxBatch) return false;
    const auto& p0 = h->inst[0].p;
    for (const auto& in : h->inst)
        if (in.p.storage != p0.storage || in.p.collision != p0.collision || in.p.boundary != p0.boundary ||
            in.p.couple != p0.couple || in.p.moving_window || in.p.driver != PWFA_DRIVER_RIGID)
            return false;
    return true;
}

void batch_release(pwfa_lbm* h) {
    if (h->graph2) cudaGraphExecDestroy(h->graph2);
    h->graph2 = nullptr;
    h->batch_valid = false;
}

int batch_launch_all(pwfa_lbm* h, int parity, cudaStream_t s, bool timed);

// Build the device instance table for the current ping-pong state and
// capture a two-step graph (parity 0 then 1). With the fused field step the
// instances first get B(t_{n+1}) where it is not already computed.
int batch_build(pwfa_lbm* h) {
    batch_release(h);
    const int n = (int)h->inst.size();
    const auto& p0 = h->inst[0].p;
    const bool fused = p0.couple && h->field_fusion != PWFA_FUSION_OFF;
    if (fused) {
        for (auto& in : h->inst) {
            if (in.lookahead) continue;
            StepArgs a = make_args(in);
            int rc = timed_launch(h, PWFA_KERNEL_FARADAY, "faraday kernel", [&] { return launch_faraday(a, h->stream); });
            if (rc) return rc;
            in.lookahead = true;
        }
    }
    std::vector<BatchEntry> ent(n);
    std::vector<int64_t> steps(2 * (size_t)n);
    int64_t ntiles = 0, nftiles = 0;
    for (int i = 0; i < n; ++i) {
        Instance& in = h->inst[i];
        BatchEntry& e = ent[i];
        for (int par = 0; par < 2; ++par) {
            e.args[par] = make_args(in);
            for (int c = 0; c < 3; ++c) {
                e.out[par].E[c] = in.Ealt[c];
                e.out[par].B[c] = in.B[in.bcur][c];
            }
            // the pointers of the next step
            in.fcur = 1 - in.fcur;
            if (in.p.couple) in.bcur = 1 - in.bcur;
            if (fused) for (int c = 0; c < 3; ++c) std::swap(in.E[c], in.Ealt[c]);
        }
        e.ntiles = (in.g.N + kBatchTile - 1) / kBatchTile;
        e.tile_begin = ntiles;
        ntiles += (e.ntiles + kBatchGroup - 1) / kBatchGroup;
        int fz = 0;
        fused_field_tiles(in.g, &e.ftiles_x, &e.ftiles_y, &fz);
        e.ftile_begin = nftiles;
        nftiles += (int64_t)e.ftiles_x * e.ftiles_y * fz;
        e.z0 = in.p.z0;
        e.dt = in.p.dt;
        e.step = h->d_steps;  // set below, once the counters exist
        steps[2 * i] = in.steps;
        steps[2 * i + 1] = in.steps + 1;
    }
    if (ntiles > INT32_MAX || nftiles > INT32_MAX) return fail(PWFA_ERR_PARAM, "batched grid longer than 2^31 tiles");
    if (n > h->entries_cap) {
        if (h->d_entries) cudaFree(h->d_entries);
        if (h->d_steps) cudaFree(h->d_steps);
        h->d_entries = nullptr;
        h->d_steps = nullptr;
        h->entries_cap = 0;
        if (dev_alloc((void**)&h->d_entries, sizeof(BatchEntry) * n) != cudaSuccess ||
            dev_alloc((void**)&h->d_steps, sizeof(int64_t) * 2 * n) != cudaSuccess) {
            cudaGetLastError();
            return alloc_fail("cudaMalloc of the batch table failed");
        }
        h->entries_cap = n;
    }
    if (ntiles + nftiles > h->tile_inst_cap) {
        if (h->d_tile_inst) cudaFree(h->d_tile_inst);
        h->d_tile_inst = nullptr;
        h->tile_inst_cap = 0;
        if (dev_alloc((void**)&h->d_tile_inst, sizeof(uint16_t) * (ntiles + nftiles)) != cudaSuccess) {
            cudaGetLastError();
            return alloc_fail("cudaMalloc of the batch tile map failed");
        }
        h->tile_inst_cap = ntiles + nftiles;
    }
    std::vector<uint16_t> map((size_t)(ntiles + nftiles));
    for (int i = 0; i < n; ++i) {
        const int64_t t1 = i + 1 < n ? ent[i + 1].tile_begin : ntiles;
        const int64_t f1 = i + 1 < n ? ent[i + 1].ftile_begin : nftiles;
        std::fill(map.begin() + ent[i].tile_begin, map.begin() + t1, (uint16_t)i);
        std::fill(map.begin() + ntiles + ent[i].ftile_begin, map.begin() + ntiles + f1, (uint16_t)i);
        ent[i].step = h->d_steps + 2 * i;
    }
    PWFA_CUDA(cudaMemcpyAsync(h->d_entries, ent.data(), sizeof(BatchEntry) * n, cudaMemcpyHostToDevice, h->stream),
              "batch table copy");
    PWFA_CUDA(cudaMemcpyAsync(h->d_steps, steps.data(), sizeof(int64_t) * 2 * n, cudaMemcpyHostToDevice, h->stream),
              "batch counters copy");
    PWFA_CUDA(cudaMemcpyAsync(h->d_tile_inst, map.data(), sizeof(uint16_t) * map.size(), cudaMemcpyHostToDevice,
                              h->stream),
              "batch tile map copy");
    PWFA_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    h->blaunch.entries = h->d_entries;
    h->blaunch.tile_inst = h->d_tile_inst;
    h->blaunch.ftile_inst = h->d_tile_inst + ntiles;
    h->blaunch.ninst = n;
    h->blaunch.ntiles = ntiles;
    h->blaunch.nftiles = nftiles;
    h->batch_fused = fused;
    if (!h->capture_stream) PWFA_CUDA(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking), "cudaStreamCreate");
    cudaGraph_t graph = nullptr;
    PWFA_CUDA(cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    int rc = batch_launch_all(h, 0, h->capture_stream, false);
    if (rc == PWFA_OK) rc = batch_launch_all(h, 1, h->capture_stream, false);
    cudaError_t e = cudaStreamEndCapture(h->capture_stream, &graph);
    if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&h->graph2, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    h->batch_valid = true;
    return PWFA_OK;
}

int step_instance(pwfa_lbm* h, Instance& in, const DiagOut* diag = nullptr);

// The launches of one batched step of every instance with the given parity:
// fluid + fused field step, or Faraday + fluid + Ampere, or the fluid alone
// (uncoupled).
int batch_phases(const pwfa_lbm* h, int* phases) {
    if (!h->inst[0].p.couple) { phases[0] = 1; return 1; }
    if (h->batch_fused) { phases[0] = 1; phases[1] = 3; return 2; }
    phases[0] = 0; phases[1] = 1; phases[2] = 2;
    return 3;
}

int batch_launch_all(pwfa_lbm* h, int parity, cudaStream_t s, bool timed) {
    const auto& p0 = h->inst[0].p;
    const bool per = p0.boundary == PWFA_PERIODIC;
    const int kinds[4] = {PWFA_KERNEL_FARADAY, PWFA_KERNEL_FLUID, PWFA_KERNEL_AMPERE, PWFA_KERNEL_AMPERE};
    int phases[3];
    const int np = batch_phases(h, phases);
    for (int k = 0; k < np; ++k) {
        const int phase = phases[k];
        if (timed) {
            cudaStream_t keep = h->stream;
            h->stream = s;
            int rc = timed_launch(h, kinds[phase], "batch kernel", [&] {
                return launch_batch_phase(h->blaunch, phase, parity, p0.storage, p0.collision, per, s);
            });
            h->stream = keep;
            if (rc) return rc;
        } else {
            PWFA_CUDA(launch_batch_phase(h->blaunch, phase, parity, p0.storage, p0.collision, per, s), "batch kernel");
        }
    }
    return PWFA_OK;
}

int batch_steps(pwfa_lbm* h, int32_t nsteps) {
    const int32_t pairs = nsteps / 2;
    if (pairs > 0) {
        if (!h->batch_valid) {
            int rc = batch_build(h);
            if (rc) return rc;
        }
        const int kinds[4] = {PWFA_KERNEL_FARADAY, PWFA_KERNEL_FLUID, PWFA_KERNEL_AMPERE, PWFA_KERNEL_AMPERE};
        int phases[3];
        const int np = batch_phases(h, phases);
        for (int32_t k = 0; k < pairs; ++k) {
            if (h->profiling) {
                int rc = batch_launch_all(h, 0, h->stream, true);
                if (rc == PWFA_OK) rc = batch_launch_all(h, 1, h->stream, true);
                if (rc) return rc;
            } else {
                PWFA_CUDA(cudaGraphLaunch(h->graph2, h->stream), "cudaGraphLaunch");
                for (int q = 0; q < np; ++q) h->launches[kinds[phases[q]]] += 2;  // launches inside the graph
            }
        }
        for (auto& in : h->inst) {
            in.steps += 2 * (int64_t)pairs;
            in.lookahead = h->batch_fused;
        }
    }
    if (nsteps % 2) {
        for (auto& in : h->inst) {
            int rc = step_instance(h, in);
            if (rc) return rc;
        }
        h->batch_valid = false;  // ping-pong parity changed
    }
    return PWFA_OK;
}

int step_instance(pwfa_lbm* h, Instance& in, const DiagOut* diag) {
    cudaStream_t s = h->stream;
    if (window_planes_at(in.p, in.steps + 1) > window_planes_at(in.p, in.steps)) {
        // move the box one plane: E and the current B level here, the
        // populations inside the fluid kernel (src_shift)
        WindowMove w{};
        w.g = in.g;
        for (int c = 0; c < 3; ++c) {
            w.E[c] = in.E[c];
            w.B[c] = in.B[in.bcur][c];
            w.Eo[c] = in.Ealt[c];
            w.Bo[c] = in.B[1 - in.bcur][c];
        }
        int rc = timed_launch(h, PWFA_KERNEL_AUX, "window move kernel", [&] { return launch_window_move(w, s); });
        if (rc) return rc;
        for (int c = 0; c < 3; ++c) std::swap(in.E[c], in.Ealt[c]);
        in.bcur = 1 - in.bcur;
    }
    StepArgs a = make_args(in);
    int rc;
    DiagOut dg{};
    if (diag) dg = *diag;
    if (in.p.couple && !in.lookahead) {
        // with diagnostics the Faraday launch also takes the field energy of
        // the entering state (it reads E and B(t_n) anyway)
        float* energy = nullptr;
        if (diag && faraday_energy_records(in.g) <= dg.energy_capacity) {
            energy = dg.energy;
            dg.nenergy = faraday_energy_records(in.g);
        }
        rc = timed_launch(h, PWFA_KERNEL_FARADAY, "faraday kernel", [&] { return launch_faraday(a, s, energy); });
        if (rc) return rc;
    }
    rc = timed_launch(h, PWFA_KERNEL_FLUID, "fluid kernel",
                      [&] { return launch_fluid(a, in.p.storage, in.p.collision, s, diag ? &dg : nullptr); });
    if (rc) return rc;
    if (in.p.driver == PWFA_DRIVER_PIC) {
        rc = timed_launch(h, PWFA_KERNEL_AUX, "particle kernel",
                          [&] { return launch_push_deposit(a, in.particles, in.np, in.pweight, in.Jb, s); });
        if (rc) return rc;
    }
    in.lookahead = false;
    const bool fuse = h->field_fusion == PWFA_FUSION_ON ||
                      (h->field_fusion == PWFA_FUSION_AUTO && in.g.N >= kFuseMinNodes);
    if (in.p.couple && fuse && fusable(in.p) && in.Ealt[0]) {
        // Ampere with the next step's Faraday: E into the other E buffer, the
        // next B into the buffer of B(t_n)
        FieldPair out{};
        for (int c = 0; c < 3; ++c) {
            out.E[c] = in.Ealt[c];
            out.B[c] = in.B[in.bcur][c];
        }
        rc = timed_launch(h, PWFA_KERNEL_AMPERE, "ampere-faraday kernel",
                          [&] { return launch_ampere_faraday(a, out, s); });
        if (rc) return rc;
        for (int c = 0; c < 3; ++c) std::swap(in.E[c], in.Ealt[c]);
        in.lookahead = true;
        h->batch_valid = false;  // the batch table holds the E pointers
    } else if (in.p.couple) {
        rc = timed_launch(h, PWFA_KERNEL_AMPERE, "ampere kernel", [&] { return launch_ampere(a, s); });
        if (rc) return rc;
    }
    in.fcur = 1 - in.fcur;
    if (in.p.couple) in.bcur = 1 - in.bcur;
    ++in.steps;
    return PWFA_OK;
}

// ---------------------------------------------------------------- adjoint
// One segment of a recording: the two population buffers the recomputed
// forward steps ping-pong between, then E of each of its K states and B of
// its K + 1 states (each field array behind a zero guard), and the lattice
// sums A_l ([4][N]) that each recomputed step stores for the reverse step.
struct SegLayout {
    size_t fb, vb, gvb, gb;
    int64_t K;
    size_t pop(int b) const { return fb * (size_t)b; }
    size_t E(int64_t j, int c) const { return 2 * fb + gvb * (size_t)(3 * j + c) + gb; }
    size_t B(int64_t j, int c) const { return 2 * fb + gvb * (size_t)(3 * K + 3 * j + c) + gb; }
    size_t mom(int64_t j) const { return 2 * fb + gvb * (size_t)(6 * K + 3) + 4 * vb * (size_t)j; }
    size_t bytes() const { return mom(K); }
};

size_t fbytes_of(const Instance& in) { return align_up((size_t)in.g.Np * kPop * storage_bytes(in.p.storage)); }
size_t vbytes_of(const Instance& in) { return align_up((size_t)in.g.N * sizeof(float)); }
// one field array with its zero guard in front (the recorded segment states
// that the recomputed forward steps read)
size_t gvbytes_of(const Instance& in) { return guard_bytes(in.g) + vbytes_of(in); }

SegLayout seg_layout(const Instance& in, int K) {
    SegLayout L;
    L.fb = fbytes_of(in);
    L.vb = vbytes_of(in);
    L.gvb = gvbytes_of(in);
    L.gb = guard_bytes(in.g);
    L.K = K;
    return L;
}


struct StateRef {  // one stored state inside a recording buffer
    void* f;
    float* E[3];
    float* B[3];
    float* Bn[3];
};

StateRef state_at(const Instance& in, void* base, bool with_bn) {
    const size_t fb = fbytes_of(in), vb = vbytes_of(in);
    char* p = static_cast<char*>(base);
    StateRef r{};
    r.f = p; p += fb;
    for (int c = 0; c < 3; ++c) { r.E[c] = (float*)p; p += vb; }
    for (int c = 0; c < 3; ++c) { r.B[c] = (float*)p; p += vb; }
    if (with_bn) for (int c = 0; c < 3; ++c) { r.Bn[c] = (float*)p; p += vb; }
    return r;
}

int copy_state(const Instance& in, const StateRef& dst, bool to_rec, cudaStream_t s) {
    const size_t fb = (size_t)in.g.Np * kPop * storage_bytes(in.p.storage);
    const size_t vb = sizeof(float) * (size_t)in.g.N;
    if (to_rec) {
        PWFA_CUDA(cudaMemcpyAsync(dst.f, in.f[in.fcur], fb, cudaMemcpyDeviceToDevice, s), "checkpoint copy");
        for (int c = 0; c < 3; ++c) {
            PWFA_CUDA(cudaMemcpyAsync(dst.E[c], in.E[c], vb, cudaMemcpyDeviceToDevice, s), "checkpoint copy");
            PWFA_CUDA(cudaMemcpyAsync(dst.B[c], in.B[in.bcur][c], vb, cudaMemcpyDeviceToDevice, s), "checkpoint copy");
        }
    } else {
        PWFA_CUDA(cudaMemcpyAsync(in.f[in.fcur], dst.f, fb, cudaMemcpyDeviceToDevice, s), "restore copy");
        for (int c = 0; c < 3; ++c) {
            PWFA_CUDA(cudaMemcpyAsync(in.E[c], dst.E[c], vb, cudaMemcpyDeviceToDevice, s), "restore copy");
            PWFA_CUDA(cudaMemcpyAsync(in.B[in.bcur][c], dst.B[c], vb, cudaMemcpyDeviceToDevice, s), "restore copy");
        }
    }
    return PWFA_OK;
}

// The built-in objective of the gradient calls (the witness loss): L =
// -mean(E_z) over the witness slab after T steps. The slab is the layer of
// E_z edges (z = (k + 1/2) dx) nearest z_w = z0 + T dt - 3 pi, i.e. 1.5
// plasma wavelengths 2 pi c / omega_p behind the driver centre (in box
// coordinates when the window has moved), over the transverse nodes that are
// not on the walls and lie within r <= 1 c/omega_p of the axis; k is kept in
// 1..nz-2. The mask depends on the grid alone, not on the driver parameters.
// rows receives the x range [lo, hi) of each row j; returns the edge count.
int64_t witness_slab(const Instance& in, int64_t T, int* k_out, std::vector<int>& rows) {
    const pwfa_lbm_params& p = in.p;
    const double zw = p.z0 + (double)T * p.dt - 3.0 * M_PI - (double)window_planes_at(p, T) * p.dx;
    int k = (int)std::nearbyint(zw / p.dx - 0.5);  // half-way cases to even
    k = std::min(std::max(k, 1), in.g.nz - 2);
    *k_out = k;
    rows.assign(2 * (size_t)in.g.ny, 0);
    int64_t count = 0;
    const double r2max = 1.0;
    for (int j = 1; j < in.g.ny - 1; ++j) {
        // squares kept in memory apart from the sum: no fused multiply-add
        volatile double yy = ((double)j - 0.5 * (in.g.ny - 1)) * p.dx;
        volatile double y2 = yy * yy;
        int lo = -1, hi = -1;
        for (int i = 1; i < in.g.nx - 1; ++i) {
            volatile double xx = ((double)i - 0.5 * (in.g.nx - 1)) * p.dx;
            volatile double x2 = xx * xx;
            volatile double r2 = x2 + y2;
            if (r2 <= r2max) {
                if (lo < 0) lo = i;
                hi = i + 1;
            }
        }
        if (lo >= 0) {
            rows[2 * j] = lo;
            rows[2 * j + 1] = hi;
            count += hi - lo;
        }
    }
    return count;
}

// The slots of one segment of a recording (SegLayout): the population
// buffers its steps ping-pong between, E and B of each state, the lattice
// sums of each step.
struct SegSlots {
    SegLayout L;
    char* p;
    void* pop(int64_t j) const { return p + L.pop((int)(j & 1)); }
    float* E(int64_t j, int c) const { return (float*)(p + L.E(j, c)); }
    float* B(int64_t j, int c) const { return (float*)(p + L.B(j, c)); }
    float* mom(int64_t j) const { return (float*)(p + L.mom(j)); }
};
SegSlots seg_slots(const Instance& in) { return SegSlots{seg_layout(in, in.rec.K), static_cast<char*>(in.rec.seg)}; }

// Run segment seg of the recording (steps s0 = seg K .. s1) from its
// checkpoint into the segment slots. Its last step leaves the populations
// at s1 in in.f[1 - in.fcur], E(t_s1) in in.E and B(t_s1) in slot B(s1 - s0);
// J in in.J.
int fill_segment(pwfa_lbm* h, Instance& in, int seg) {
    cudaStream_t s = h->stream;
    const auto& r = in.rec;
    const int64_t N = in.g.N;
    const int64_t s0 = (int64_t)seg * r.K, s1 = std::min<int64_t>(r.T, s0 + r.K);
    const SegSlots S = seg_slots(in);
    // restore the checkpoint into state 0 of the segment
    {
        StateRef cp = state_at(in, (char*)r.cp + r.cp_stride * seg, false);
        const size_t fb = (size_t)in.g.Np * kPop * storage_bytes(in.p.storage);
        PWFA_CUDA(cudaMemcpyAsync(S.pop(0), cp.f, fb, cudaMemcpyDeviceToDevice, s), "restore copy");
        for (int c = 0; c < 3; ++c) {
            PWFA_CUDA(cudaMemcpyAsync(S.E(0, c), cp.E[c], sizeof(float) * N, cudaMemcpyDeviceToDevice, s),
                      "restore copy");
            PWFA_CUDA(cudaMemcpyAsync(S.B(0, c), cp.B[c], sizeof(float) * N, cudaMemcpyDeviceToDevice, s),
                      "restore copy");
        }
    }
    // recompute the segment's steps: populations ping-pong, E and B of
    // each state and the lattice sums of each step into their slots; Ampere
    // of step j runs fused with Faraday of step j + 1 where that B slot
    // exists
    const int64_t len = s1 - s0;
    bool b_ahead = false;
    for (int64_t j = 0; j < len; ++j) {
        const int64_t keep_steps = in.steps;
        in.steps = s0 + j;
        StepArgs f = make_args(in);
        in.steps = keep_steps;
        const bool last = j + 1 == len;
        f.fin = S.pop(j);
        f.fout = last ? in.f[1 - in.fcur] : S.pop(j + 1);
        f.mom = S.mom(j);
        for (int c = 0; c < 3; ++c) {
            f.E[c] = S.E(j, c);
            f.Bc[c] = S.B(j, c);
            f.Bn[c] = S.B(j + 1, c);
            f.Eout[c] = last ? in.E[c] : S.E(j + 1, c);  // Ampere out of place writes every component
        }
        if (in.p.couple) {
            if (!b_ahead) {
                int rc = timed_launch(h, PWFA_KERNEL_FARADAY, "faraday kernel", [&] { return launch_faraday(f, s); });
                if (rc) return rc;
            }
        } else {
            // no Maxwell update: E and B pass through
            for (int c = 0; c < 3; ++c) {
                PWFA_CUDA(cudaMemcpyAsync(f.Bn[c], f.Bc[c], sizeof(float) * N, cudaMemcpyDeviceToDevice, s),
                          "B copy");
                PWFA_CUDA(cudaMemcpyAsync(f.Eout[c], f.E[c], sizeof(float) * N, cudaMemcpyDeviceToDevice, s),
                          "E copy");
            }
        }
        int rc = timed_launch(h, PWFA_KERNEL_FLUID, "fluid kernel",
                              [&] { return launch_fluid_mom(f, in.p.storage, in.p.collision, s); });
        if (rc) return rc;
        b_ahead = false;
        if (in.p.couple && !last && fusable(in.p)) {
            // B(t_{n+2}) of the next recomputed step into its slot
            FieldPair out{};
            for (int c = 0; c < 3; ++c) {
                out.E[c] = f.Eout[c];
                out.B[c] = S.B(j + 2, c);
            }
            rc = timed_launch(h, PWFA_KERNEL_AMPERE, "ampere-faraday kernel",
                              [&] { return launch_ampere_faraday(f, out, s); });
            if (rc) return rc;
            b_ahead = true;
        } else if (in.p.couple) {
            rc = timed_launch(h, PWFA_KERNEL_AMPERE, "ampere kernel", [&] { return launch_ampere(f, s); });
            if (rc) return rc;
        }
    }
    return PWFA_OK;
}

int record_instance(pwfa_lbm* h, Instance& in, int32_t nsteps, int32_t ckpt_every) {
    cudaStream_t s = h->stream;
    if (in.p.moving_window) return fail(PWFA_ERR_PARAM, "the adjoint does not support the moving window");
    if (in.p.driver != PWFA_DRIVER_RIGID) return fail(PWFA_ERR_PARAM, "the adjoint needs the rigid driver");
    free_recording(in);
    auto& r = in.rec;
    r.T = nsteps;
    r.K = ckpt_every > 0 ? ckpt_every : (int)std::ceil(std::sqrt((double)nsteps));
    if (r.K > nsteps) r.K = nsteps;
    r.ncp = (int)((nsteps + r.K - 1) / r.K);
    const size_t fb = fbytes_of(in), vb = vbytes_of(in);
    r.cp_stride = fb + 6 * vb;
    const size_t seg_bytes = seg_layout(in, r.K).bytes();
    const size_t adj_bytes = 2 * align_up((size_t)in.g.Np * kPop * sizeof(float)) + 22 * vb +
                             align_up(sizeof(double) * (260 + 3 * kGradSlots));
    if (dev_alloc((void**)&r.cp, r.cp_stride * (r.ncp + 1)) != cudaSuccess ||
        dev_alloc((void**)&r.seg, seg_bytes) != cudaSuccess ||
        dev_alloc((void**)&r.adj, adj_bytes) != cudaSuccess) {
        cudaGetLastError();
        char buf[200];
        std::snprintf(buf, sizeof buf, "recording needs %.2f GB (%d checkpoints + a segment of %d steps)",
                      (r.cp_stride * (r.ncp + 1) + seg_bytes + adj_bytes) / 1e9, r.ncp + 1, r.K);
        free_recording(in);
        return alloc_fail(buf);
    }
    // the guards in front of the segment's field slots stay zero
    PWFA_CUDA(cudaMemsetAsync(r.seg, 0, seg_bytes, s), "cudaMemsetAsync");
    int rc = reset_instance(in, s);
    if (rc) return rc;
    // the segments before the last one: ordinary steps with a checkpoint at
    // the start of each
    const int64_t s_last = (int64_t)(r.ncp - 1) * r.K;
    for (int64_t n = 0; n < s_last; ++n) {
        if (n % r.K == 0) {
            rc = copy_state(in, state_at(in, (char*)r.cp + r.cp_stride * (n / r.K), false), true, s);
            if (rc) return rc;
        }
        rc = step_instance(h, in);
        if (rc) return rc;
    }
    rc = copy_state(in, state_at(in, (char*)r.cp + r.cp_stride * (r.ncp - 1), false), true, s);
    if (rc) return rc;
    // the last segment runs as the reverse sweep would recompute it, into
    // the segment slots, which the sweep then reverses first without a
    // recomputation (with one segment, ckpt_every >= nsteps, nothing is
    // recomputed at all)
    rc = fill_segment(h, in, r.ncp - 1);
    if (rc) return rc;
    // the state at T: populations and E where the last step left them, B
    // from the segment's last slot
    in.fcur = 1 - in.fcur;
    {
        const SegSlots S = seg_slots(in);
        for (int c = 0; c < 3; ++c)
            PWFA_CUDA(cudaMemcpyAsync(in.B[in.bcur][c], S.B(r.T - s_last, c), sizeof(float) * (size_t)in.g.N,
                                      cudaMemcpyDeviceToDevice, s),
                      "B copy");
    }
    in.lookahead = false;
    in.steps = r.T;
    h->batch_valid = false;  // the batch table holds the population pointers
    rc = copy_state(in, state_at(in, (char*)r.cp + r.cp_stride * r.ncp, false), true, s);
    if (rc) return rc;
    r.filled = r.ncp - 1;
    r.valid = true;
    return PWFA_OK;
}

int adjoint_instance(pwfa_lbm* h, Instance& in, const float* seed_E, int32_t nsteps, int32_t ckpt_every,
                     double* host_grad, int32_t n_grad) {
    cudaStream_t s = h->stream;
    auto& r = in.rec;
    if (nsteps > 0 && (!r.valid || r.T != nsteps || (ckpt_every > 0 && r.K != std::min(ckpt_every, nsteps)))) {
        // no recording of this run yet: record it now
        int rc = record_instance(h, in, nsteps, ckpt_every);
        if (rc) return rc;
    }
    if (!r.valid) return fail(PWFA_ERR_STATE, "no recording: pass nsteps >= 1 or call pwfa_lbm_record first");
    const int np = (int)in.profile.size();
    if (n_grad < 3 + np) return fail(PWFA_ERR_PARAM, "n_grad must be >= 3 + n_profile");
    if (np > 256) return fail(PWFA_ERR_PARAM, "the adjoint supports at most 256 profile points");
    const int64_t N = in.g.N;
    const size_t vb = vbytes_of(in);
    const size_t sb = align_up((size_t)in.g.Np * kPop * sizeof(float));
    char* p = static_cast<char*>(r.adj);
    float* Sbar[2] = {(float*)p, (float*)(p + sb)};
    p += 2 * sb;
    AdjArgs a{};
    float* Ebar[3];
    float* Bbar[3];
    for (int c = 0; c < 3; ++c) { Ebar[c] = (float*)p; p += vb; }
    for (int c = 0; c < 3; ++c) { Bbar[c] = (float*)p; p += vb; }
    for (int c = 0; c < 3; ++c) { a.Bnp[c] = (float*)p; p += vb; }
    for (int c = 0; c < 3; ++c) { a.Jbar[c] = (float*)p; p += vb; }
    for (int c = 0; c < 3; ++c) { a.ebar[c] = (float*)p; p += vb; }
    for (int c = 0; c < 3; ++c) { a.bbar[c] = (float*)p; p += vb; }
    for (int l = 0; l < 4; ++l) { a.Abnd[l] = (float*)p; p += vb; }
    double* grad = (double*)p;
    for (int c = 0; c < 3; ++c) { a.Ebar[c] = Ebar[c]; a.Bbar[c] = Bbar[c]; }
    a.grad = grad;
    a.gslots = grad + 260;
    a.sr = (float)in.p.sigma_r;
    a.sz = (float)in.p.sigma_z;
    PWFA_CUDA(cudaMemsetAsync(r.adj, 0, (size_t)(p - (char*)r.adj) + sizeof(double) * (260 + 3 * kGradSlots), s),
              "cudaMemsetAsync");
    if (seed_E) {
        for (int c = 0; c < 3; ++c)
            PWFA_CUDA(cudaMemcpyAsync(Ebar[c], seed_E + c * N, sizeof(float) * N, cudaMemcpyDefault, s), "seed copy");
    } else {
        // the witness loss: dL/dE_z = -1/count on the slab, zero elsewhere
        int k = 0;
        std::vector<int> rows;
        const int64_t count = witness_slab(in, r.T, &k, rows);
        if (count == 0) return fail(PWFA_ERR_PARAM, "the witness slab holds no edge (grid narrower than r <= 1)");
        PWFA_CUDA(cudaMemcpyAsync(in.d_wrows, rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice, s),
                  "witness rows copy");
        PWFA_CUDA(launch_witness_seed(in.g, Ebar[2], k, in.d_wrows, (float)(-1.0 / (double)count), s),
                  "witness seed kernel");
        // the rows are read by the kernel before this call returns
        PWFA_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    }
    if (!in.g.periodic) {
        // the adjoint keeps E_bar zero at the components the conducting walls
        // hold at zero; the seed's values there never enter the forward
        StepArgs z = make_args(in);
        for (int c = 0; c < 3; ++c) {
            z.Eout[c] = Ebar[c];
            z.Bc[c] = Bbar[c];
        }
        PWFA_CUDA(launch_zero_walls(z, s), "seed mask");
    }
    int cur = 0;
    for (int seg = r.ncp - 1; seg >= 0; --seg) {
        const int64_t s0 = (int64_t)seg * r.K, s1 = std::min<int64_t>(r.T, s0 + r.K);
        const SegSlots S = seg_slots(in);
        // the recording leaves its last segment's steps in the slots; every
        // other segment is recomputed from its checkpoint (which overwrites
        // them)
        const bool have = r.filled == seg;
        r.filled = -1;
        if (!have) {
            int rc = fill_segment(h, in, seg);
            if (rc) return rc;
        }
        for (int64_t n = s1 - 1; n >= s0; --n) {
            const int64_t j = n - s0;
            const int64_t keep_steps = in.steps;  // forward arguments of step n
            in.steps = n;
            StepArgs f = make_args(in);
            in.steps = keep_steps;
            f.fin = nullptr;  // the reverse step reads the lattice sums instead
            f.fout = nullptr;
            f.mom = S.mom(j);
            for (int c = 0; c < 3; ++c) {
                f.E[c] = S.E(j, c);
                f.Bc[c] = S.B(j, c);
                f.Bn[c] = S.B(j + 1, c);
                f.Eout[c] = nullptr;
                f.J[c] = nullptr;
            }
            a.f = f;
            a.Sbar_in = Sbar[cur];
            a.Sbar_out = Sbar[1 - cur];
            int rc = timed_launch(h, PWFA_KERNEL_ADJ_FIELD, "adjoint ampere kernel",
                                  [&] { return launch_adjoint_ampere(a, s); });
            if (rc) return rc;
            rc = timed_launch(h, PWFA_KERNEL_ADJ_FLUID, "adjoint fluid kernel",
                              [&] { return launch_adjoint_fluid(a, in.p.storage, in.p.collision, s); });
            if (rc) return rc;
            rc = timed_launch(h, PWFA_KERNEL_ADJ_FIELD, "adjoint field kernels", [&] {
                return launch_adjoint_fields(a, h->field_fusion != PWFA_FUSION_OFF, s);
            });
            if (rc) return rc;
            cur = 1 - cur;
        }
    }
    PWFA_CUDA(launch_adjoint_grad_finish(a.gslots, grad, s), "driver gradient");
    PWFA_CUDA(launch_adjoint_profile(in.g, Sbar[cur], (float)in.p.n0, np, in.p.profile_rmax, in.p.dx, grad + 3, s),
              "profile gradient");
    PWFA_CUDA(cudaMemcpyAsync(host_grad, grad, sizeof(double) * (3 + np), cudaMemcpyDeviceToHost, s), "grad copy");
    int rc = copy_state(in, state_at(in, (char*)r.cp + r.cp_stride * r.ncp, false), false, s);
    if (rc) return rc;
    in.lookahead = false;
    in.steps = r.T;
    PWFA_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    return PWFA_OK;
}



int ensure_step_diag(pwfa_lbm* h) {
    int64_t need = 1, need_e = 1;
    for (const auto& in : h->inst) {
        const int64_t b = (int64_t)((in.g.nx + in.bx - 1) / in.bx) * ((in.g.ny + in.by - 1) / in.by) * in.g.nz;
        need = std::max(need, b * (in.bx * in.by / 32));  // one record per warp
        need_e = std::max(need_e, faraday_energy_records(in.g));
    }
    if (!h->d_step_diag) {
        if (dev_alloc((void**)&h->d_step_diag, sizeof(double) * 8 * h->inst.size()) != cudaSuccess ||
            dev_alloc((void**)&h->d_step_scratch, sizeof(double) * 8 * kDiagBlocks) != cudaSuccess) {
            cudaGetLastError();
            return alloc_fail("cudaMalloc of the diagnostics results failed");
        }
    }
    if (need > h->step_records_cap || need_e > h->step_energy_cap) {
        if (h->d_step_records) cudaFree(h->d_step_records);
        h->d_step_records = nullptr;
        h->step_records_cap = h->step_energy_cap = 0;
        if (dev_alloc((void**)&h->d_step_records, sizeof(float) * (8 * need + need_e)) != cudaSuccess) {
            cudaGetLastError();
            return alloc_fail("cudaMalloc of the diagnostics records failed");
        }
        h->step_records_cap = need;
        h->step_energy_cap = need_e;
    }
    return PWFA_OK;
}

// Debug builds: after a call that ran kernels, fail it with PWFA_ERR_STATE
// if a kernel recorded an index outside its array (the word stays set).
// Release builds return rc unchanged without touching the device.
int debug_after(pwfa_lbm* h, int rc) {
#ifdef PWFA_DEBUG
    if (!h) return rc;
    for (size_t i = 0; i < h->inst.size(); ++i) {
        unsigned w[3] = {0, 0, 0};
        if (cudaMemcpyAsync(w, h->inst[i].d_dbg, sizeof w, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "debug word copy");
        if (w[0]) {
            char buf[200];
            std::snprintf(buf, sizeof buf,
                          "debug build: instance %d, index %d out of range at site %u (%u accesses)", (int)i,
                          (int)w[1], w[0], w[2]);
            return fail(PWFA_ERR_STATE, buf);
        }
    }
#else
    (void)h;
#endif
    return rc;
}

}  // namespace

extern "C" {

const char* pwfa_lbm_last_error(void) { return g_err.c_str(); }

static int step_diag_impl(pwfa_lbm_t* h, int32_t nsteps, double* host_diag) {
    NvtxRange nvtx_("pwfa_lbm_step_diag");
    if (!h) return fail(PWFA_ERR_PARAM, "null handle");
    if (nsteps < 1 || !host_diag) return fail(PWFA_ERR_PARAM, "nsteps must be >= 1 and host_diag not NULL");
    int rc = pwfa_lbm_step(h, nsteps - 1);
    if (rc) return rc;
    rc = ensure_step_diag(h);
    if (rc) return rc;
    for (size_t i = 0; i < h->inst.size(); ++i) {
        Instance& in = h->inst[i];
        DiagOut d{};
        d.records = h->d_step_records;
        d.capacity = h->step_records_cap;
        d.energy = h->d_step_records + 8 * h->step_records_cap;
        d.energy_capacity = h->step_energy_cap;
        d.scratch = h->d_step_scratch;
        d.out = h->d_step_diag + 8 * i;
        d.dxcube = in.p.dx * in.p.dx * in.p.dx;
        rc = step_instance(h, in, &d);
        if (rc) return rc;
    }
    h->batch_valid = false;  // the last step ran per instance
    PWFA_CUDA(cudaMemcpyAsync(host_diag, h->d_step_diag, sizeof(double) * 8 * h->inst.size(),
                              cudaMemcpyDeviceToHost, h->stream),
              "cudaMemcpyAsync");
    PWFA_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    for (size_t i = 0; i < h->inst.size(); ++i) {
        const double* d = host_diag + 8 * i;
        if (d[7] > 0 || d[5] < 0) {
            char buf[160];
            std::snprintf(buf, sizeof buf, "instance %d unstable: %g non-finite nodes, min n = %g", (int)i, d[7], d[5]);
            return fail(PWFA_ERR_UNSTABLE, buf);
        }
    }
    return PWFA_OK;
}

int pwfa_lbm_step_diag(pwfa_lbm_t* h, int32_t nsteps, double* host_diag) {
    return debug_after(h, step_diag_impl(h, nsteps, host_diag));
}

static int record_impl(pwfa_lbm_t* h, int32_t instance, int32_t nsteps, int32_t ckpt_every) {
    NvtxRange nvtx_("pwfa_lbm_record");
    int rc = check_instance(h, instance);
    if (rc) return rc;
    if (nsteps < 1 || ckpt_every < 0) return fail(PWFA_ERR_PARAM, "nsteps must be >= 1 and ckpt_every >= 0");
    h->batch_valid = false;
    return record_instance(h, h->inst[instance], nsteps, ckpt_every);
}

int pwfa_lbm_record(pwfa_lbm_t* h, int32_t instance, int32_t nsteps, int32_t ckpt_every) {
    return debug_after(h, record_impl(h, instance, nsteps, ckpt_every));
}

static int adjoint_impl(pwfa_lbm_t* h, int32_t instance, const float* seed_E, int32_t nsteps, int32_t ckpt_every,
                        double* host_grad, int32_t n_grad) {
    NvtxRange nvtx_("pwfa_lbm_adjoint_step");
    int rc = check_instance(h, instance);
    if (rc) return rc;
    if (!host_grad) return fail(PWFA_ERR_PARAM, "host_grad must not be NULL");
    if (nsteps < 0 || ckpt_every < 0) return fail(PWFA_ERR_PARAM, "nsteps and ckpt_every must be >= 0");
    h->batch_valid = false;
    return adjoint_instance(h, h->inst[instance], seed_E, nsteps, ckpt_every, host_grad, n_grad);
}

int pwfa_lbm_adjoint_step(pwfa_lbm_t* h, int32_t instance, const float* seed_E, int32_t nsteps, int32_t ckpt_every,
                          double* host_grad, int32_t n_grad) {
    return debug_after(h, adjoint_impl(h, instance, seed_E, nsteps, ckpt_every, host_grad, n_grad));
}

int pwfa_lbm_witness_loss(pwfa_lbm_t* h, int32_t instance, double* host_loss) {
    int rc = check_instance(h, instance);
    if (rc) return rc;
    if (!host_loss) return fail(PWFA_ERR_PARAM, "host_loss must not be NULL");
    Instance& in = h->inst[instance];
    int k = 0;
    std::vector<int> rows;
    const int64_t count = witness_slab(in, in.steps, &k, rows);
    if (count == 0) return fail(PWFA_ERR_PARAM, "the witness slab holds no edge (grid narrower than r <= 1)");
    PWFA_CUDA(cudaMemcpyAsync(in.d_wrows, rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice, h->stream),
              "witness rows copy");
    PWFA_CUDA(launch_witness_sum(in.g, in.E[2], k, in.d_wrows, in.d_wout, h->stream), "witness sum kernel");
    double sum = 0.0;
    PWFA_CUDA(cudaMemcpyAsync(&sum, in.d_wout, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "cudaMemcpyAsync");
    PWFA_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    *host_loss = -sum / (double)count;
    return PWFA_OK;
}

int pwfa_lbm_create(const pwfa_lbm_params* params, int32_t n_instances, void* cuda_stream, pwfa_lbm_t** out) {
    NvtxRange nvtx_("pwfa_lbm_create");
    if (!out) return fail(PWFA_ERR_PARAM, "out is NULL");
    *out = nullptr;
    if (!params || n_instances < 1) return fail(PWFA_ERR_PARAM, "params is NULL or n_instances < 1");
    for (int i = 0; i < n_instances; ++i) {
        int rc = validate(params[i], i);
        if (rc) return rc;
    }
    pwfa_lbm* h = new (std::nothrow) pwfa_lbm();
    if (!h) return fail(PWFA_ERR_ALLOC, "host allocation failed");
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    h->inst.resize(n_instances);
    int rc = PWFA_OK;
    for (int i = 0; i < n_instances && rc == PWFA_OK; ++i) {
        Instance& in = h->inst[i];
        in.p = params[i];
        if (in.p.dt == 0) in.p.dt = 0.17628 * in.p.dx;
        if (in.p.n_floor == 0) in.p.n_floor = 1e-6;
        if (in.p.n_profile > 0) in.profile.assign(in.p.profile, in.p.profile + in.p.n_profile);
        in.p.profile = nullptr;
        in.g.nx = in.p.nx; in.g.ny = in.p.ny; in.g.nz = in.p.nz;
        in.g.N = (int64_t)in.p.nx * in.p.ny * in.p.nz;
        // with a moving window one more plane (fresh plasma above the box)
        in.g.Np = (in.g.N + (in.p.moving_window ? (int64_t)in.p.nx * in.p.ny : 0) + 31) / 32 * 32;
        in.g.periodic = in.p.boundary == PWFA_PERIODIC;
        rc = alloc_instance(in, h->stream);
    }
    if (rc == PWFA_OK) {
        if (dev_alloc((void**)&h->d_partials, sizeof(double) * 8 * (kDiagBlocks + 1)) != cudaSuccess) {
            cudaGetLastError();
            rc = alloc_fail("cudaMalloc of the diagnostics buffer failed");
        } else {
            h->d_diag = h->d_partials + 8 * kDiagBlocks;
        }
    }
    if (rc == PWFA_OK) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "create");
    }
    if (rc != PWFA_OK) {
        std::string msg = g_err;
        pwfa_lbm_destroy(h);
        g_err = msg;
        return rc;
    }
    *out = h;
    return PWFA_OK;
}

static int step_impl(pwfa_lbm_t* h, int32_t nsteps) {
    NvtxRange nvtx_("pwfa_lbm_step");
    if (!h) return fail(PWFA_ERR_PARAM, "null handle");
    if (nsteps < 0) return fail(PWFA_ERR_PARAM, "nsteps must be >= 0");
    if (batch_eligible(h)) return batch_steps(h, nsteps);
    for (int32_t s = 0; s < nsteps; ++s)
        for (auto& in : h->inst) {
            int rc = step_instance(h, in);
            if (rc) return rc;
        }
    return PWFA_OK;
}

int pwfa_lbm_step(pwfa_lbm_t* h, int32_t nsteps) { return debug_after(h, step_impl(h, nsteps)); }

static int fields_impl(pwfa_lbm_t* h, int32_t instance, uint32_t mask, float* out, int64_t out_elems,
                    double* host_diag) {
    int rc = check_instance(h, instance);
    if (rc) return rc;
    Instance& in = h->inst[instance];
    const uint32_t comp = mask & 0xFFFFu;
    if (mask & 0x7FFF0000u) return fail(PWFA_ERR_PARAM, "unknown bits in mask");
    const int nbits = __builtin_popcount(comp);
    StepArgs a = make_args(in);
    if (nbits > 0) {
        if (!out) return fail(PWFA_ERR_PARAM, "out is NULL");
        if (out_elems < (int64_t)nbits * in.g.N) return fail(PWFA_ERR_PARAM, "out_elems too small for the mask");
        const bool dev = is_device_ptr(out);
        float* dst = out;
        const size_t bytes = sizeof(float) * (size_t)nbits * in.g.N;
        if (!dev) {
            rc = ensure_staging(h, bytes);
            if (rc) return rc;
            dst = static_cast<float*>(h->staging);
        }
        PWFA_CUDA(launch_export_fields(a, in.p.storage, mask, dst, h->stream), "export kernel");
        if (!dev) {
            PWFA_CUDA(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, h->stream), "cudaMemcpyAsync");
            PWFA_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
        }
    }
    if (host_diag) {
        const double dx3 = in.p.dx * in.p.dx * in.p.dx;
        PWFA_CUDA(launch_diag(a, in.p.storage, dx3, h->d_partials, h->d_diag, h->stream), "diag kernel");
        PWFA_CUDA(cudaMemcpyAsync(host_diag, h->d_diag, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
                  "cudaMemcpyAsync");
        PWFA_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
        if (host_diag[7] > 0 || host_diag[5] < 0) {
            char buf[160];
            std::snprintf(buf, sizeof buf, "instance %d unstable: %g non-finite nodes, min n = %g", instance,
                          host_diag[7], host_diag[5]);
            return fail(PWFA_ERR_UNSTABLE, buf);
        }
    }
    return PWFA_OK;
}

int pwfa_lbm_fields(pwfa_lbm_t* h, int32_t instance, uint32_t mask, float* out, int64_t out_elems,
                    double* host_diag) {
    return debug_after(h, fields_impl(h, instance, mask, out, out_elems, host_diag));
}

int pwfa_lbm_linecut(pwfa_lbm_t* h, int32_t instance, double r, double n_star, float* out, int64_t out_elems,
                     double* bubble_length) {
    int rc = check_instance(h, instance);
    if (rc) return rc;
    Instance& in = h->inst[instance];
    const int nz = in.g.nz;
    if (!out || out_elems < 2 * (int64_t)nz) return fail(PWFA_ERR_PARAM, "out must hold 2 * nz floats");
    if (!std::isfinite(r)) return fail(PWFA_ERR_PARAM, "r must be finite");
    const bool dev = is_device_ptr(out);
    float* dst = out;
    const size_t bytes = sizeof(float) * 2 * (size_t)nz;
    if (!dev || bubble_length) {
        rc = ensure_staging(h, bytes);
        if (rc) return rc;
        dst = static_cast<float*>(h->staging);
    }
    PWFA_CUDA(launch_linecut(make_args(in), in.p.storage, r, dst, h->stream), "linecut kernel");
    if (dst != out) PWFA_CUDA(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDefault, h->stream), "cudaMemcpyAsync");
    if (bubble_length) {
        std::vector<float> hn(nz);
        PWFA_CUDA(cudaMemcpyAsync(hn.data(), dst, sizeof(float) * nz, cudaMemcpyDeviceToHost, h->stream),
                  "cudaMemcpyAsync");
        PWFA_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
        int64_t count = 0;
        for (int k = 0; k < nz; ++k) count += hn[k] < n_star ? 1 : 0;
        *bubble_length = count * in.p.dx;
    }
    if (!dev) PWFA_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return PWFA_OK;
}

int pwfa_lbm_get_state(pwfa_lbm_t* h, int32_t instance, float* f, float* E, float* B) {
    int rc = check_instance(h, instance);
    if (rc) return rc;
    Instance& in = h->inst[instance];
    const int64_t N = in.g.N;
    StepArgs a = make_args(in);
    if (f) {
        const size_t bytes = sizeof(float) * (size_t)kPop * N;
        const bool dev = is_device_ptr(f);
        float* dst = f;
        if (!dev) {
            rc = ensure_staging(h, bytes);
            if (rc) return rc;
            dst = static_cast<float*>(h->staging);
        }
        PWFA_CUDA(launch_export_f(a, in.p.storage, dst, h->stream), "export kernel");
        if (!dev) PWFA_CUDA(cudaMemcpyAsync(f, dst, bytes, cudaMemcpyDeviceToHost, h->stream), "cudaMemcpyAsync");
    }
    const size_t vb = sizeof(float) * (size_t)N;
    for (int c = 0; c < 3; ++c) {
        if (E) PWFA_CUDA(cudaMemcpyAsync(E + c * N, in.E[c], vb, cudaMemcpyDefault, h->stream), "cudaMemcpyAsync E");
        if (B) PWFA_CUDA(cudaMemcpyAsync(B + c * N, in.B[in.bcur][c], vb, cudaMemcpyDefault, h->stream),
                         "cudaMemcpyAsync B");
    }
    PWFA_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return PWFA_OK;
}

int pwfa_lbm_set_state(pwfa_lbm_t* h, int32_t instance, const float* f, const float* E, const float* B) {
    int rc = check_instance(h, instance);
    if (rc) return rc;
    h->batch_valid = false;
    Instance& in = h->inst[instance];
    in.lookahead = false;
    const int64_t N = in.g.N;
    if (f) {
        const size_t bytes = sizeof(float) * (size_t)kPop * N;
        const float* src = f;
        if (!is_device_ptr(f)) {
            rc = ensure_staging(h, bytes);
            if (rc) return rc;
            PWFA_CUDA(cudaMemcpyAsync(h->staging, f, bytes, cudaMemcpyHostToDevice, h->stream), "cudaMemcpyAsync");
            src = static_cast<const float*>(h->staging);
        }
        PWFA_CUDA(launch_import_f(in.g, src, in.f[in.fcur], in.p.storage, (float)in.p.n0, h->stream),
                  "import kernel");
    }
    const size_t vb = sizeof(float) * (size_t)N;
    for (int c = 0; c < 3; ++c) {
        if (E) PWFA_CUDA(cudaMemcpyAsync(in.E[c], E + c * N, vb, cudaMemcpyDefault, h->stream), "cudaMemcpyAsync E");
        if (B) PWFA_CUDA(cudaMemcpyAsync(in.B[in.bcur][c], B + c * N, vb, cudaMemcpyDefault, h->stream),
                         "cudaMemcpyAsync B");
    }
    // Open grids: components on or outside the conducting walls are zero.
    if ((E || B) && !in.g.periodic) PWFA_CUDA(launch_zero_walls(make_args(in), h->stream), "wall kernel");
    PWFA_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return PWFA_OK;
}

int64_t pwfa_lbm_steps_done(pwfa_lbm_t* h, int32_t instance) {
    int rc = check_instance(h, instance);
    if (rc) return rc;
    return h->inst[instance].steps;
}

int pwfa_lbm_set_particles(pwfa_lbm_t* h, int32_t instance, int64_t n, const float* xp, double weight) {
    int rc = check_instance(h, instance);
    if (rc) return rc;
    Instance& in = h->inst[instance];
    if (in.p.driver != PWFA_DRIVER_PIC) return fail(PWFA_ERR_PARAM, "the instance was not created with the PIC driver");
    if (n < 0 || (n > 0 && !xp)) return fail(PWFA_ERR_PARAM, "bad particle array");
    if (!(weight >= 0) || !std::isfinite(weight)) return fail(PWFA_ERR_PARAM, "weight must be finite and >= 0");
    PWFA_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (in.particles) cudaFree(in.particles);
    in.particles = nullptr;
    in.np = 0;
    if (n > 0) {
        if (dev_alloc((void**)&in.particles, sizeof(float) * 6 * (size_t)n) != cudaSuccess) {
            cudaGetLastError();
            return alloc_fail("cudaMalloc of the particle array failed");
        }
        PWFA_CUDA(cudaMemcpyAsync(in.particles, xp, sizeof(float) * 6 * (size_t)n, cudaMemcpyDefault, h->stream),
                  "particle copy");
        PWFA_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    }
    in.np = n;
    in.pweight = weight;
    return PWFA_OK;
}

int pwfa_lbm_get_particles(pwfa_lbm_t* h, int32_t instance, float* out) {
    int rc = check_instance(h, instance);
    if (rc) return rc;
    Instance& in = h->inst[instance];
    if (in.np == 0) return PWFA_OK;
    if (!out) return fail(PWFA_ERR_PARAM, "out is NULL");
    PWFA_CUDA(cudaMemcpyAsync(out, in.particles, sizeof(float) * 6 * (size_t)in.np, cudaMemcpyDefault, h->stream),
              "particle copy");
    PWFA_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    return PWFA_OK;
}

int64_t pwfa_lbm_window_planes(pwfa_lbm_t* h, int32_t instance) {
    int rc = check_instance(h, instance);
    if (rc) return rc;
    const Instance& in = h->inst[instance];
    return window_planes_at(in.p, in.steps);
}

int pwfa_lbm_profile(pwfa_lbm_t* h, int32_t enable) {
    if (!h) return fail(PWFA_ERR_PARAM, "null handle");
    if (enable && h->events.empty()) {
        h->events.resize(2 * kEventPairs);
        for (auto& e : h->events) PWFA_CUDA(cudaEventCreate(&e), "cudaEventCreate");
    }
    if (!enable) {
        int rc = fold_events(h);
        if (rc) return rc;
    }
    h->profiling = enable != 0;
    return PWFA_OK;
}

int pwfa_lbm_kernel_times(pwfa_lbm_t* h, double* ms, int64_t* launches) {
    if (!h) return fail(PWFA_ERR_PARAM, "null handle");
    int rc = fold_events(h);
    if (rc) return rc;
    PWFA_CUDA(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    for (int k = 0; k < PWFA_KERNEL_KINDS; ++k) {
        if (ms) ms[k] = h->ms[k];
        if (launches) launches[k] = h->launches[k];
        h->ms[k] = 0;
        h->launches[k] = 0;
    }
    return PWFA_OK;
}

int pwfa_lbm_set_launch(pwfa_lbm_t* h, int32_t instance, int32_t bx, int32_t by) {
    int rc = check_instance(h, instance);
    if (rc) return rc;
    if (bx < 1 || by < 1 || bx * by > PWFA_FLUID_MAX_THREADS || (bx * by) % 32)
        return fail(PWFA_ERR_PARAM, "block shape must be a multiple of 32 threads, at most 128");
    h->inst[instance].bx = bx;
    h->inst[instance].by = by;
    h->batch_valid = false;
    return PWFA_OK;
}

int pwfa_lbm_set_fluid_variant(pwfa_lbm_t* h, int32_t instance, int32_t variant) {
    int rc = check_instance(h, instance);
    if (rc) return rc;
    if (variant != PWFA_FLUID_DIRECT && variant != PWFA_FLUID_STAGED) return fail(PWFA_ERR_PARAM, "unknown variant");
    h->inst[instance].variant = variant;
    h->batch_valid = false;
    return PWFA_OK;
}

int pwfa_lbm_get_fluid_variant(pwfa_lbm_t* h, int32_t instance, int32_t* variant) {
    int rc = check_instance(h, instance);
    if (rc) return rc;
    if (variant) *variant = h->inst[instance].variant;
    return PWFA_OK;
}

int pwfa_lbm_get_launch(pwfa_lbm_t* h, int32_t instance, int32_t* bx, int32_t* by) {
    int rc = check_instance(h, instance);
    if (rc) return rc;
    if (bx) *bx = h->inst[instance].bx;
    if (by) *by = h->inst[instance].by;
    return PWFA_OK;
}

int pwfa_lbm_autotune(pwfa_lbm_t* h, int32_t reps) {
    if (!h) return fail(PWFA_ERR_PARAM, "null handle");
    if (reps < 1) return fail(PWFA_ERR_PARAM, "reps must be >= 1");
    // {bx, by, variant}: direct shapes, then the staged kernel's 128-thread
    // tiles (the batched path's per-node phases take tiles of consecutive
    // nodes instead; the shapes serve the per-instance steps)
    static const int cand_all[][3] = {{32, 4, 0}, {64, 2, 0}, {128, 1, 0}, {32, 4, 1}, {64, 2, 1}, {128, 1, 1}};
    const int ncand = (int)(sizeof cand_all / sizeof cand_all[0]);
    h->batch_valid = false;
    cudaEvent_t e0, e1;
    PWFA_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
    PWFA_CUDA(cudaEventCreate(&e1), "cudaEventCreate");
    int rc = PWFA_OK;
    for (auto& in : h->inst) {
        float best = 1e30f;
        int bb[3] = {in.bx, in.by, in.variant};
        for (int ci = 0; ci < ncand; ++ci) {
            const int* c = cand_all[ci];
            if (c[0] > 2 * in.g.nx && c[0] > 32) continue;  // mostly idle lanes
            if (c[0] * c[1] > PWFA_FLUID_MAX_THREADS) continue;
            in.bx = c[0];
            in.by = c[1];
            in.variant = c[2];
            StepArgs a = make_args(in);
            a.src_shift = 0;  // time a plain step even if the next one moves the window
            cudaError_t e = launch_fluid(a, in.p.storage, in.p.collision, h->stream);  // warm
            if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
            for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_fluid(a, in.p.storage, in.p.collision, h->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) { rc = cuda_fail(e, "autotune"); break; }
            if (ms < best) { best = ms; bb[0] = c[0]; bb[1] = c[1]; bb[2] = c[2]; }
        }
        in.bx = bb[0];
        in.by = bb[1];
        in.variant = bb[2];
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

int pwfa_lbm_set_field_fusion(pwfa_lbm_t* h, int32_t mode) {
    if (!h) return fail(PWFA_ERR_PARAM, "null handle");
    if (mode != PWFA_FUSION_OFF && mode != PWFA_FUSION_AUTO && mode != PWFA_FUSION_ON)
        return fail(PWFA_ERR_PARAM, "unknown field-fusion mode");
    h->field_fusion = mode;
    h->batch_valid = false;  // the batched graph holds the field step's form
    return PWFA_OK;
}

int pwfa_lbm_set_batching(pwfa_lbm_t* h, int32_t enable) {
    if (!h) return fail(PWFA_ERR_PARAM, "null handle");
    h->batching = enable != 0;
    h->batch_valid = false;
    return PWFA_OK;
}

int pwfa_lbm_set_stream(pwfa_lbm_t* h, void* cuda_stream) {
    if (!h) return fail(PWFA_ERR_PARAM, "null handle");
    cudaStream_t next = static_cast<cudaStream_t>(cuda_stream);
    if (next != h->stream) {
        // the new stream's work follows everything already queued on the old
        // one (no host wait)
        cudaEvent_t done;
        PWFA_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming), "cudaEventCreate");
        cudaError_t e = cudaEventRecord(done, h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(next, done, 0);
        cudaEventDestroy(done);
        if (e != cudaSuccess) return cuda_fail(e, "stream switch");
    }
    h->stream = next;
    return PWFA_OK;
}

int pwfa_lbm_destroy(pwfa_lbm_t* h) {
    if (!h) return PWFA_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    for (auto& in : h->inst) free_instance(in);
    if (h->d_partials) cudaFree(h->d_partials);
    if (h->staging) cudaFree(h->staging);
    for (auto& e : h->events) cudaEventDestroy(e);
    batch_release(h);
    if (h->d_entries) cudaFree(h->d_entries);
    if (h->d_steps) cudaFree(h->d_steps);
    if (h->d_tile_inst) cudaFree(h->d_tile_inst);
    if (h->d_step_records) cudaFree(h->d_step_records);
    if (h->d_step_diag) cudaFree(h->d_step_diag);
    if (h->d_step_scratch) cudaFree(h->d_step_scratch);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    delete h;
    return PWFA_OK;
}

}  // extern "C"
