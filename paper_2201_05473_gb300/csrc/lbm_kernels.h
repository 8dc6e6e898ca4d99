// Host-side launchers of the LBM plasma-wakefield kernels (internal to the
// library; the public interface is include/pwfa_lbm.h).
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace pwfa {

// Device allocation of the library (cudaMalloc with the test hook
// PWFA_FAIL_ALLOC_AT: the n-th allocation of the process fails).
cudaError_t dev_alloc(void** p, size_t bytes);

// Launch bounds of the fluid kernels: blocks of at most 128 threads; for the
// regularized form five per SM with FP32 storage (a 96-register budget) and
// six with the 16-bit forms (80 registers; a few values spill to L1), four
// (128 registers) for BGK and stream-only. With its first moments taken right after the gather the
// regularized kernel fits those budgets and the extra warps hide the pull's
// latency (production grid: FP32 3.24 -> 3.17 ms at five blocks against four;
// BF16 2.05 -> 1.86 ms at five, 1.83 ms at six; FP32 at six: 3.46 ms). BGK
// and stream-only carry every pulled value itself through the source
// computation and would spill at 96.
#ifndef PWFA_FLUID_MAX_THREADS
#define PWFA_FLUID_MAX_THREADS 128
#endif
#ifndef PWFA_FLUID_MIN_BLOCKS
#define PWFA_FLUID_MIN_BLOCKS 5
#endif
#ifndef PWFA_FLUID_MIN_BLOCKS_16
#define PWFA_FLUID_MIN_BLOCKS_16 6
#endif
template <int ST, int COLL>
struct FluidOcc {
    static constexpr int blocks = COLL == 1 ? (ST == 0 ? PWFA_FLUID_MIN_BLOCKS : PWFA_FLUID_MIN_BLOCKS_16) : 4;
};
// The batched fluid phase parks BGK's pulled values of lattices 2 and 3 in
// shared memory between the moments and the collision (fluid_rest), which
// lets it run at 96 registers and five blocks per SM instead of 128 and
// four: 64-instance scan 10.99 -> 10.62 ms per step. The single-instance
// kernel keeps them in registers (3.266 against 3.280 ms parked).
#ifndef PWFA_BGK_STASH
#define PWFA_BGK_STASH 1
#endif
template <int ST, int COLL>
struct BatchFluidOcc {
    static constexpr bool park = COLL == 0 && PWFA_BGK_STASH;
    static constexpr int blocks = park ? 5 : FluidOcc<ST, COLL>::blocks;
};

// Where the fused diagnostics of a step go. The fluid launch writes one FP32
// record of 8 values per warp (sum n, sum n p_x, p_y, p_z, field energy /
// dx^3, min n, min -|beta|^2, non-finite count); when the step's Faraday
// launch took the field energy (nenergy > 0) it wrote one FP32 value per warp
// to energy and the fluid records carry 0 there. Both are combined in FP64
// into out[8] (scratch: kDiagBlocks FP64 records).
struct DiagOut {
    float* records;
    int64_t capacity;
    float* energy;
    int64_t energy_capacity;
    int64_t nenergy;
    double* scratch;
    double* out;
    double dxcube;
};

// Fused fluid step: pull streaming (Eq. 6), moments, Lorentz source (Eqs. 4,
// 10), collision (Eq. 7 or regularized), Eq. 14 boundary nodes, node current.
// With d != NULL it also reduces the FP64 diagnostics of the entering state.
cudaError_t launch_fluid(const StepArgs& a, int storage, int collision, cudaStream_t s,
                         const DiagOut* d = nullptr);

// The same fluid step that also stores each node's lattice sums A_l into
// a.mom ([4][N] FP32): the adjoint's recomputed forward steps keep them for
// the reverse step, which needs nothing else of the populations.
cudaError_t launch_fluid_mom(const StepArgs& a, int storage, int collision, cudaStream_t s);

// Reduce the nrec fluid records and d.nenergy energy records of a fused step
// into d.out: up to kDiagBlocks blocks combine contiguous chunks into
// d.scratch, one block combines those (a single block over the ~2.6e5
// records of a 512x256x256 grid was latency-bound at ~1 ms).
cudaError_t launch_diag_finish_step(const DiagOut& d, int64_t nrec, cudaStream_t s);

// Faraday, dB/dt = -curl E: Bn = Bc - dt curl_h E (Yee, Eq. 5). With energy
// != NULL each warp also writes the field energy (|E|^2 + |Bc|^2)/2 of its
// nodes, per dx^3, to energy[warp] (faraday_energy_records(g) records).
cudaError_t launch_faraday(const StepArgs& a, cudaStream_t s, float* energy = nullptr);
int64_t faraday_energy_records(const Grid& g);

// Ampere, dE/dt = curl B - J: E += dt (curl_h Bn - J_edge - J_b(t_{n+1})).
cudaError_t launch_ampere(const StepArgs& a, cudaStream_t s);

// Ampere of this step fused with Faraday of the next (rigid driver only):
// out.E := E + dt (curl_h Bn - J_edge - J_b) (a.E unchanged), out.B := the
// next step's B(t_{n+2}) = Bn - dt curl_h out.E. out.E must not alias a.E and
// out.B none of a.E, a.Bn, a.J (out.B is normally a.Bc's buffer).
struct FieldPair {
    float* E[3];
    float* B[3];
};
cudaError_t launch_ampere_faraday(const StepArgs& a, const FieldPair& out, cudaStream_t s);
// Tiles of the fused field step over a grid: tx x ty per z-slab, tz slabs.
void fused_field_tiles(const Grid& g, int* tx, int* ty, int* tz);

// Open grids: zero the Yee components of E and B(t_n) that lie on or outside
// the conducting walls (tangential E, normal B, components past the grid).
cudaError_t launch_zero_walls(const StepArgs& a, cudaStream_t s);

// Moving window (open grids): Eo, Bo := E, B moved down one plane (box node
// k takes node k + 1), zero on the top plane and on the conducting walls.
struct WindowMove {
    Grid g;
    const float* E[3];
    const float* B[3];
    float* Eo[3];
    float* Bo[3];
};
cudaError_t launch_window_move(const WindowMove& w, cudaStream_t s);

// PIC driver: push np macro-electrons (xp[6][np]: x, y, z at t_{n+1/2},
// p_x, p_y, p_z at t_n) with the step's fields and add the current of their
// moves to Jb (E-edge arrays, zero outside a.jbox: Ampere clears what it
// consumes), growing the node box a.jbox to cover every deposit. weight:
// electrons per macro-particle in units of n0 (c/omega_p)^3.
cudaError_t launch_push_deposit(const StepArgs& a, float* xp, int64_t np, double weight, float* const Jb[3],
                                cudaStream_t s);

// Initial condition: stored populations whose pull gives the plasma at rest,
// f = w_i n0 prof(r) (lattice 0), 0 (momentum lattices).
cudaError_t launch_init(const Grid& g, void* f, int storage, float n0, const double* d_profile,
                        int n_profile, double profile_rmax, double dx, cudaStream_t s);

// Export the pre-collision populations f^n as FP32 [4][19][N].
cudaError_t launch_export_f(const StepArgs& a, int storage, float* out, cudaStream_t s);

// Import FP32 pre-collision populations [4][19][N] into the stored layout.
cudaError_t launch_import_f(const Grid& g, const float* in, void* f, int storage, float n0, cudaStream_t s);

// Node fields selected by a PWFA_FIELD_* mask into out, one block of N per bit.
cudaError_t launch_export_fields(const StepArgs& a, int storage, unsigned mask, float* out, cudaStream_t s);

// Line cut along z at offset r from the axis: out[0..nz) density,
// out[nz..2nz) node-averaged E_z (bilinear in x, y).
cudaError_t launch_linecut(const StepArgs& a, int storage, double r, float* out, cudaStream_t s);

// The built-in gradient objective's slab (plane k, x range [rows[2 j],
// rows[2 j + 1]) in row j): the FP64 sum of E_z over it into out[0], or
// Ez_bar := value on it.
cudaError_t launch_witness_sum(const Grid& g, const float* Ez, int k, const int* rows, double* out, cudaStream_t s);
cudaError_t launch_witness_seed(const Grid& g, float* Ezbar, int k, const int* rows, float value, cudaStream_t s);

// FP64 diagnostics: partial sums per block into partials (nblocks x 8), then
// reduced into out[8] (device).
constexpr int kDiagBlocks = 1024;
constexpr int kDiagThreads = 256;
cudaError_t launch_diag(const StepArgs& a, int storage, double dxcube, double* partials, double* out,
                        cudaStream_t s);

}  // namespace pwfa
