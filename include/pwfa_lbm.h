/*
 * pwfa_lbm.h - C ABI of the GB300 lattice-Boltzmann plasma-wakefield step.
 *
 * Method: Parise et al., "Lattice Boltzmann simulations of plasma wakefield
 * acceleration", arXiv:2201.05473. The electron plasma is a cold relativistic
 * fluid (Eq. 2) advanced as four D3Q19 advection-diffusion lattices for
 * A = (n, n p_x, n p_y, n p_z) (Eq. 4 generalised to Cartesian momentum),
 * each with BGK collision (Eq. 7), equilibrium Eq. 9 in lattice units
 * (c_s^2 = 1/3, diffusivity D = (tau - 1/2)/3 of Eq. 12), source S_i = w_i F dt
 * (Eq. 10) with the Lorentz force F = -n (E + beta x B) (Eq. 4), and
 * equilibrium boundary nodes (Eq. 14). It is coupled to Maxwell's equations
 * (Eq. 5) on a Yee grid (FDTD) through the current J = -n beta, and driven by
 * a rigid bi-Gaussian electron bunch moving at c along +z.
 *
 * Units: time 1/omega_p, length c/omega_p, density n0, momentum m_e c,
 * E and B in m_e c omega_p / e.
 *
 * Conventions shared by every call:
 *   - Grid nodes x_i = i dx, i = 0..nx-1 (same for y, z); z is the driver's
 *     propagation axis. Every node array is [z][y][x], x fastest.
 *   - Yee staggering: E_x at (i+1/2, j, k), E_y at (i, j+1/2, k), E_z at
 *     (i, j, k+1/2); B_x at (i, j+1/2, k+1/2), B_y at (i+1/2, j, k+1/2),
 *     B_z at (i+1/2, j+1/2, k). Each stored as an [z][y][x] array indexed by
 *     the integer part of its position.
 *   - D3Q19 order: 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 = (1,1,0),
 *     (-1,-1,0), (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1),
 *     (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1). Populations are exchanged as
 *     [lattice 0..3][q 0..18][z][y][x].
 *   - Time levels: after s steps the populations and B are at t_s = s dt and
 *     E at t_{s+1/2}.
 *   - Every call returns PWFA_OK (0) or a negative PWFA_ERR_* code; the
 *     message of the last failure on the calling thread is returned by
 *     pwfa_lbm_last_error(). No C++ exception crosses this boundary.
 *   - Pointers named dev_* must be device memory; pointers named out/in may
 *     be host or device memory (the library checks with
 *     cudaPointerGetAttributes and copies as needed). Caller-owned memory is
 *     never retained after a call returns.
 *   - All device work is ordered on the stream given at create (or set with
 *     pwfa_lbm_set_stream). Calls that return data to host memory synchronise
 *     that stream; the others are asynchronous.
 */
#ifndef PWFA_LBM_H
#define PWFA_LBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PWFA_OK 0
#define PWFA_ERR_PARAM (-1)    /* invalid argument or parameter set */
#define PWFA_ERR_CUDA (-2)     /* a CUDA runtime call or kernel launch failed */
#define PWFA_ERR_UNSTABLE (-3) /* diagnostics found a non-finite value or n < 0 */
#define PWFA_ERR_TIMEOUT (-4)  /* a bounded device-side wait expired (reserved: no kernel of this
                                  library waits on another, so no call returns it at present) */
#define PWFA_ERR_ALLOC (-5)    /* device memory allocation failed: the device had no room (a
                                  cudaMalloc the runtime refuses for another reason, e.g.
                                  inside the caller's stream capture, returns PWFA_ERR_CUDA) */
#define PWFA_ERR_STATE (-6)    /* call not valid in the handle's current state */

/* Collision operator of every lattice. */
#define PWFA_BGK 0          /* Eq. 7: f* = f - (f - f^eq)/tau + w_i F dt */
#define PWFA_REGULARIZED 1  /* BGK on the first-order Hermite projection of f - f^eq
                               (the paper names "more complicated" operators without
                               defining one; this is the builder's choice) */
#define PWFA_STREAM_ONLY 2  /* no collision and no source: pure streaming (testing) */

/* Storage format of the populations (compute is always FP32). */
#define PWFA_F32 0
#define PWFA_BF16 1  /* deviations f - w_i n0 (lattice 0) and f (lattices 1-3), bf16 */
#define PWFA_F16 2   /* same deviations in IEEE binary16 */

/* Boundary treatment. */
#define PWFA_OPEN 0      /* Eq. 14: boundary nodes = f^eq of the clamped interior
                            node ("free flux"); conducting walls for the fields */
#define PWFA_PERIODIC 1  /* every axis wraps */

typedef struct {
    int32_t nx, ny, nz;    /* grid nodes; each >= 3 */
    double dx;             /* node spacing in c/omega_p, > 0 */
    double dt;             /* time step in 1/omega_p; 0 selects 0.17628 dx, the
                              paper's c dt / dz (Sec. IV); must satisfy
                              dt < dx / sqrt(3) (Yee Courant limit) */
    double tau;            /* BGK relaxation time in lattice units, > 0.5 (Eq. 12) */
    int32_t collision;     /* PWFA_BGK / PWFA_REGULARIZED / PWFA_STREAM_ONLY */
    int32_t storage;       /* PWFA_F32 / PWFA_BF16 / PWFA_F16 */
    int32_t boundary;      /* PWFA_OPEN / PWFA_PERIODIC */
    int32_t couple;        /* 1: Lorentz source + Maxwell update; 0: fluid only */
    double n0;             /* background electron density (normalised, >= 0) */
    const double* profile; /* host array of n_profile radial multipliers of n0 at
                              r_j = j profile_rmax / (n_profile - 1), linear in
                              between, last value beyond; NULL = uniform. Copied
                              at create. r is measured from the axis
                              x_c = (nx-1) dx / 2, y_c = (ny-1) dx / 2. */
    int32_t n_profile;     /* 0 or >= 1 */
    double profile_rmax;   /* > 0 when n_profile >= 2 */
    double alpha;          /* driver peak density n_b / n0 (Eq. 15's alpha) */
    double sigma_r;        /* driver rms radius, > 0 */
    double sigma_z;        /* driver rms length, > 0 */
    double z0;             /* driver centre at t = 0; it moves as z0 + t */
    double n_floor;        /* p = A / max(n, n_floor); 0 selects 1e-6 */
    int32_t moving_window; /* 1: the box follows the driver (Sec. II's moving
                              window; open boundary, single-instance stepping
                              and no adjoint recording). After n steps it has
                              moved W_n = max(0, floor((z0 + n dt - window_z)
                              / dx)) planes along +z: a step with W_{n+1} >
                              W_n first moves the streaming source, E and B
                              down one plane, drops the bottom plane and
                              fills the top plane with the initial plasma at
                              rest and zero fields (conducting walls imposed
                              on the moved fields), then steps as usual with
                              the driver at its lab position. 0: fixed box. */
    double window_z;       /* box coordinate at which the driver centre is held
                              once the window moves (c/omega_p) */
    int32_t driver;        /* PWFA_DRIVER_RIGID: the rigid bi-Gaussian bunch
                              (alpha, sigma_r, sigma_z, z0); PWFA_DRIVER_PIC:
                              macro-electrons set by pwfa_lbm_set_particles
                              (Eq. 1; single-instance stepping, no moving
                              window, no adjoint) */
} pwfa_lbm_params;

#define PWFA_DRIVER_RIGID 0
#define PWFA_DRIVER_PIC 1

typedef struct pwfa_lbm pwfa_lbm_t;

/* Create n_instances independent simulations (params is an array of that
 * length), allocate their device state and set the initial condition: a cold
 * plasma at rest with density n0 * profile(r), E = B = 0 (Sec. IV test case).
 * cuda_stream is a cudaStream_t (NULL = legacy default stream). The handle
 * owns all device memory it allocates. On failure *out is NULL. */
int pwfa_lbm_create(const pwfa_lbm_params* params, int32_t n_instances,
                    void* cuda_stream, pwfa_lbm_t** out);

/* Advance every instance by nsteps (>= 0) time steps: Faraday, fused
 * pull-stream + moments + Lorentz source + collision (Eqs. 6-10, 14), Ampere
 * with J = -n beta and the driver current. Asynchronous on the stream. A
 * caller that captures this call into a graph of its own records kernels
 * whose arguments (buffer parity, driver time of a single instance) are
 * fixed at capture, and the handle counts the steps once: replaying such a
 * graph repeats those steps rather than continuing the run. For repeated
 * steps use nsteps (the batched path replays its own graphs, whose driver
 * time advances on the device). */
int pwfa_lbm_step(pwfa_lbm_t* h, int32_t nsteps);

/* Gradients by the discrete adjoint (the paper has no adjoint; this
 * differentiates the scheme above exactly, step by step in reverse).
 *
 * pwfa_lbm_record resets the instance to its initial condition (t = 0) and
 * advances it nsteps, keeping a checkpoint of the full state every
 * ckpt_every steps (0 selects ceil(sqrt(nsteps))) plus the final state. The
 * instance is left at step nsteps. Device memory: (nsteps/ckpt_every + 1)
 * states of 76 N populations + 6 N field values; one segment of K =
 * ckpt_every recomputed steps (two population buffers, the E and B of its
 * states, 6 (K + 1) N values, and the four lattice sums of each step, 4 K N:
 * the reverse step needs nothing else of the populations); ~174 N floats of
 * adjoint scratch; PWFA_ERR_ALLOC if it does not fit. The last segment
 * runs as the reverse sweep would recompute it, into the segment storage,
 * so the next pwfa_lbm_adjoint_step reverses it without recomputing it; with
 * ckpt_every >= nsteps (one segment of nsteps steps, when memory allows)
 * that sweep recomputes nothing. */
int pwfa_lbm_record(pwfa_lbm_t* h, int32_t instance, int32_t nsteps, int32_t ckpt_every);

/* Gradient of an objective L of the raw Yee E after T recorded steps with
 * respect to theta = (alpha, sigma_r, sigma_z, profile[0..n_profile-1]),
 * written to host_grad (n_grad >= 3 + n_profile doubles, host).
 *   seed_E  dL/dE, [3][z][y][x] FP32 (host or device) for
 *           L = sum(seed_E * E(t_{T+1/2})); or NULL for the built-in witness
 *           loss of pwfa_lbm_witness_loss after T steps (the library seeds
 *           -1/count on its slab).
 *   nsteps  T >= 1: run the forward with checkpoints first (as
 *           pwfa_lbm_record(h, instance, nsteps, ckpt_every)) unless the
 *           instance already holds a recording of T steps (with ckpt_every
 *           checkpoints when ckpt_every > 0); 0: use the existing recording
 *           (PWFA_ERR_STATE if there is none).
 *   ckpt_every  checkpoint interval of a new recording; 0 selects
 *           ceil(sqrt(T)).
 * Each segment is recomputed from its checkpoint, then reversed: transposed
 * Ampere (with the driver's parameter derivatives), transposed fluid step
 * (J = -n beta(p*), collision, equilibrium, Lorentz source, beta(p), the
 * n-floor branch, Eq. 14 boundary nodes, transposed pull), transposed node
 * averages and Faraday; the initial populations give the profile
 * derivative. Adjoint state is FP32, parameter gradients are accumulated in
 * FP64. n_profile <= 256. The instance ends at step T. Synchronises. */
int pwfa_lbm_adjoint_step(pwfa_lbm_t* h, int32_t instance, const float* seed_E, int32_t nsteps,
                          int32_t ckpt_every, double* host_grad, int32_t n_grad);

/* The built-in gradient objective at the instance's current step T (the
 * witness loss of the differentiable form): host_loss receives
 * L = -mean(E_z) over the witness slab, the layer of E_z edges
 * z = (k + 1/2) dx nearest z_w = z0 + T dt - 3 pi (1.5 plasma wavelengths
 * 2 pi c/omega_p behind the driver centre; k kept in 1..nz-2) over the
 * transverse nodes off the walls with r <= 1 c/omega_p of the axis. The slab
 * does not depend on the driver parameters. FP64 sum; synchronises.
 * PWFA_ERR_PARAM if the slab holds no edge. */
int pwfa_lbm_witness_loss(pwfa_lbm_t* h, int32_t instance, double* host_loss);

/* Advance every instance by nsteps (>= 1) like pwfa_lbm_step and return the
 * FP64 diagnostics of the state entering the last step, fused into that
 * step's fluid kernel (no extra pass over the populations): host_diag
 * receives 8 doubles per instance in the order of pwfa_lbm_fields'
 * host_diag. Synchronises the stream; PWFA_ERR_UNSTABLE (after filling
 * host_diag) if an instance has non-finite moments or n < 0. */
int pwfa_lbm_step_diag(pwfa_lbm_t* h, int32_t nsteps, double* host_diag);

/* Field export masks for pwfa_lbm_fields. */
#define PWFA_FIELD_N (1u << 0)   /* electron density n = sum of lattice 0 */
#define PWFA_FIELD_UX (1u << 1)  /* beta_x = p_x / sqrt(1 + p^2) */
#define PWFA_FIELD_UY (1u << 2)
#define PWFA_FIELD_UZ (1u << 3)
#define PWFA_FIELD_EX (1u << 4)
#define PWFA_FIELD_EY (1u << 5)
#define PWFA_FIELD_EZ (1u << 6)
#define PWFA_FIELD_BX (1u << 7)
#define PWFA_FIELD_BY (1u << 8)
#define PWFA_FIELD_BZ (1u << 9)
#define PWFA_FIELD_JX (1u << 10) /* plasma current of the last step, at nodes */
#define PWFA_FIELD_JY (1u << 11)
#define PWFA_FIELD_JZ (1u << 12)
#define PWFA_FIELD_PX (1u << 13) /* momentum density A_k = n p_k */
#define PWFA_FIELD_PY (1u << 14)
#define PWFA_FIELD_PZ (1u << 15)
#define PWFA_RAW_YEE (1u << 31)  /* E, B as raw staggered Yee arrays instead of
                                    node averages */

/* Export the selected fields of one instance at its current time level into
 * out (host or device), one [z][y][x] block of nx*ny*nz floats per set bit
 * in increasing bit order. out_elems must be >= (#bits) * nodes; out may be
 * NULL when only diagnostics are wanted. E and B are averaged to the nodes
 * (E from its two edges, B from its four faces) unless PWFA_RAW_YEE is set.
 * host_diag (nullable, 8 doubles, host) receives FP64 reductions over the
 * instance: [0] sum n, [1..3] sum n p_k, [4] field energy 1/2 sum(E^2+B^2) dx^3,
 * [5] min n, [6] max |beta|, [7] count of non-finite moments. A non-NULL
 * host_diag synchronises the stream and returns PWFA_ERR_UNSTABLE (after
 * filling host_diag) when [7] > 0 or [5] < 0. */
int pwfa_lbm_fields(pwfa_lbm_t* h, int32_t instance, uint32_t mask, float* out,
                    int64_t out_elems, double* host_diag);

/* Line cut and bubble length (Sec. IV observables). out (host or device,
 * >= 2 nz floats) receives, along z, the electron density n and the
 * node-averaged E_z at transverse offset r (c/omega_p) from the driver axis
 * along +x, bilinear between the four surrounding nodes. bubble_length
 * (nullable, host) receives L_b = dz * #{k : n_k < n_star} on that line: the
 * paper's bubble length, counted with the threshold n* = 0.95 (pass r = 0
 * for the axis). Synchronises the stream when out is host memory or
 * bubble_length is given. */
int pwfa_lbm_linecut(pwfa_lbm_t* h, int32_t instance, double r, double n_star, float* out, int64_t out_elems,
                     double* bubble_length);

/* Full state of one instance: pre-collision populations f^n
 * [4][19][z][y][x], raw Yee E (t_{n+1/2}) and B (t_n) [3][z][y][x]. Any of the
 * three pointers may be NULL. Host or device memory. In open mode the
 * boundary-node populations are not independent state: they are exported
 * and re-derived as f^eq of the clamped interior node (Eq. 14). */
int pwfa_lbm_get_state(pwfa_lbm_t* h, int32_t instance, float* f, float* E, float* B);
int pwfa_lbm_set_state(pwfa_lbm_t* h, int32_t instance, const float* f,
                       const float* E, const float* B);

/* Steps taken by an instance so far (>= 0), or a negative error code. */
int64_t pwfa_lbm_steps_done(pwfa_lbm_t* h, int32_t instance);

/* Planes the moving window of an instance has advanced so far (0 for a fixed
 * box), or a negative error code: box node k sits at lab z = (k + W) dx. */
int64_t pwfa_lbm_window_planes(pwfa_lbm_t* h, int32_t instance);

/* PIC driver (Eq. 1): n macro-electrons, xp[6][n] FP32 (host or device) =
 * x, y, z (box coordinates, c/omega_p) at t_{n+1/2} and p_x, p_y, p_z (m_e c)
 * at t_n, each of weight electrons in units of n0 (c/omega_p)^3. Each step,
 * after the fluid, they are pushed by the Boris scheme with E(t_{n+1/2}) and
 * the mean of B(t_n), B(t_{n+1}) interpolated trilinearly from each Yee
 * component, moved by dt p/gamma, and the current of the move is deposited
 * on the E edges by Esirkepov's charge-conserving scheme (linear shape);
 * Ampere subtracts it in place of the rigid J_b. Particles outside an open
 * grid see no field and deposit only on in-grid edges; periodic grids wrap
 * them. PWFA_ERR_PARAM unless the instance was created with
 * PWFA_DRIVER_PIC. Replaces any previous particle set. */
int pwfa_lbm_set_particles(pwfa_lbm_t* h, int32_t instance, int64_t n, const float* xp, double weight);

/* Current particles, out[6][n] as above (host or device); n from the last
 * pwfa_lbm_set_particles. Synchronises. */
int pwfa_lbm_get_particles(pwfa_lbm_t* h, int32_t instance, float* out);

/* Kernel kinds reported by pwfa_lbm_kernel_times. */
#define PWFA_KERNEL_FARADAY 0 /* Yee B update */
#define PWFA_KERNEL_FLUID 1   /* fused stream + moments + source + collide */
#define PWFA_KERNEL_AMPERE 2  /* Yee E update with plasma and driver current */
#define PWFA_KERNEL_AUX 3     /* moving-window field moves, PIC push and deposit */
#define PWFA_KERNEL_ADJ_FLUID 4 /* adjoint: transposed fluid step (boundary and interior nodes) */
#define PWFA_KERNEL_ADJ_FIELD 5 /* adjoint: transposed Ampere, node averages and Faraday */
#define PWFA_KERNEL_KINDS 6

/* Per-kernel device timing, off by default. While enabled, each step records
 * a CUDA event pair around every kernel it launches on the handle's stream
 * (no synchronisation is added). */
int pwfa_lbm_profile(pwfa_lbm_t* h, int32_t enable);

/* Synchronise the stream and return, per kernel kind, the device time in ms
 * accumulated while profiling was enabled (ms, nullable, PWFA_KERNEL_KINDS
 * doubles) and the number of launches (launches, nullable, PWFA_KERNEL_KINDS
 * int64, counted whether or not profiling is on) since the previous call;
 * both accumulators are then reset. */
int pwfa_lbm_kernel_times(pwfa_lbm_t* h, double* ms, int64_t* launches);

/* Thread-block shape (bx * by threads, bx along x) of the fused fluid kernel
 * for one instance. bx, by >= 1, bx * by a multiple of 32 and at most 128;
 * PWFA_ERR_PARAM otherwise. */
int pwfa_lbm_set_launch(pwfa_lbm_t* h, int32_t instance, int32_t bx, int32_t by);
int pwfa_lbm_get_launch(pwfa_lbm_t* h, int32_t instance, int32_t* bx, int32_t* by);

/* Fluid kernel variants. DIRECT: one thread per node, the 76 pulled values
 * loaded straight into registers. STAGED: persistent 128-thread tiles,
 * software pipelined: each thread's pulled values of its next tile (76 FP32
 * words, or 38 words of 16-bit lattice pairs) arrive in shared memory by
 * cp.async while it computes the current node; needs bx * by = 128 (other
 * shapes run the direct kernel). */
#define PWFA_FLUID_DIRECT 0
#define PWFA_FLUID_STAGED 1
int pwfa_lbm_set_fluid_variant(pwfa_lbm_t* h, int32_t instance, int32_t variant);
int pwfa_lbm_get_fluid_variant(pwfa_lbm_t* h, int32_t instance, int32_t* variant);

/* Autotune the fluid kernel's block shape and variant of every instance: time reps
 * launches (>= 1) of each candidate shape with CUDA events and keep the
 * fastest. The kernel is re-run on the current state without advancing it,
 * so the simulation state is unchanged. Synchronises the stream. */
int pwfa_lbm_autotune(pwfa_lbm_t* h, int32_t reps);

/* Batched path, on by default. A handle with 2..65535 instances that share
 * storage, collision, boundary and coupling and use the rigid driver in a
 * fixed box advances them together: each phase of a step is one launch over
 * the tiles of every instance (the fluid step on 128-node tiles, then Ampere
 * fused with the next step's Faraday on z-marching field tiles; with
 * PWFA_FUSION_OFF, Faraday, fluid and Ampere), and two steps at a time are
 * replayed from a captured CUDA graph whose field launches advance the
 * driver's step counters themselves (an odd remainder step runs per
 * instance). The instance table and graph are rebuilt lazily after any call
 * that changes an instance's state, launch shape or the field-fusion mode.
 * enable = 0 advances the instances one after another with ordinary
 * launches. */
int pwfa_lbm_set_batching(pwfa_lbm_t* h, int32_t enable);

/* Field-step fusion. For a coupled instance with the rigid driver and a
 * fixed box, the Ampere update of step n (Eq. 5) can run in one kernel with
 * the Faraday update of step n+1: B(t_n+1) is read once for both, and step
 * n+1 starts without its Faraday launch. Results are those of the separate
 * kernels, bit for bit. The kernel-time kind PWFA_KERNEL_AMPERE then covers
 * the fused kernel. Modes: OFF (separate launches), AUTO (the default: fused
 * on grids of 4 Mi nodes or more, where it is faster, and in the batched
 * path, whose field launch spans every instance), ON (always);
 * PWFA_ERR_PARAM for another value. In the adjoint sweep the transposed
 * node averages and Faraday update run as one kernel unless the mode is
 * OFF (the same results, bit for bit). */
#define PWFA_FUSION_OFF 0
#define PWFA_FUSION_AUTO 1
#define PWFA_FUSION_ON 2
int pwfa_lbm_set_field_fusion(pwfa_lbm_t* h, int32_t mode);

/* Re-target all later work of the handle to another cudaStream_t (NULL:
 * the legacy default stream). The new stream waits for the work already
 * queued on the old one (an event, no host wait), so the switch may come
 * while kernels are in flight. */
int pwfa_lbm_set_stream(pwfa_lbm_t* h, void* cuda_stream);

/* FP64 diagnostics of a state the caller holds in device memory, computed
 * without allocating anything. The paper has no counterpart: this serves
 * callers that must not let a library call cudaMalloc/cudaFree, such as an
 * in-situ analysis hook inside another code, or an application that owns a
 * fixed device-memory budget through its own pool (cudaFree also
 * synchronises the whole device and would stall its other streams).
 *   dev_f   pre-collision populations f^n, [4][19][z][y][x] FP32 (the
 *           layout of pwfa_lbm_get_state), device memory
 *   dev_E, dev_B  raw Yee E and B, [3][z][y][x] FP32, device memory
 *   dev_out 8 doubles, device memory, the same quantities as the host_diag
 *           of pwfa_lbm_fields: sum n, sum n p_k (3), field energy
 *           1/2 sum(E^2 + B^2) dx^3, min n, max |beta|, non-finite count
 *   n_floor density floor of p = A / max(n, n_floor); 0 selects 1e-6, a
 *           negative or NaN value is rejected with PWFA_ERR_PARAM
 * Work is enqueued on cuda_stream (a cudaStream_t, NULL = legacy default
 * stream) and not synchronised. Scratch is a fixed 1 MiB array inside the
 * library that every GPU which loads it holds until exit; grids of more than
 * 67,108,864 nodes are rejected with PWFA_ERR_PARAM. The first call on each
 * device looks up that array's device address (cudaGetSymbolAddress), so make
 * the first call on a device before any stream capture. All calls share the
 * array: calls that overlap on the GPU (different streams, or several host
 * threads) race and must be serialised by the caller. */
int pwfa_lbm_diag_noalloc(int32_t nx, int32_t ny, int32_t nz, double dx, double n_floor,
                          const float* dev_f, const float* dev_E, const float* dev_B,
                          double* dev_out, void* cuda_stream);

/* Release every device allocation of the handle. Accepts NULL. */
int pwfa_lbm_destroy(pwfa_lbm_t* h);

/* Message of the last failure on the calling thread ("" if none). The
 * pointer stays valid until the next call on this thread. */
const char* pwfa_lbm_last_error(void);

/* ------------------------------------------------------------------------
 * 2D-axisymmetric (z, r) form: the paper's own geometry (Sec. III).
 *
 * Three D2Q9 advection-diffusion lattices on the (z, r) plane for
 * A = (n, n p_z, n p_r) (Eq. 4), BGK collision (Eq. 7) to the equilibrium of
 * Eq. 9 (lattice units, c_s^2 = 1/3), u = beta(p) dt/dx (Eq. 2), pull
 * streaming (Eq. 6), and the cylindrical terms of Eq. 13 added to every
 * lattice's source: S_i = w_i dt (F + D (1/r) dA/dr - A u_r / r), with
 * D = (tau - 1/2)/3 dx^2/dt (Eq. 12) and dA/dr the central difference of the
 * node moments. Fields: cylindrical Yee TM (E_z, E_r, B_theta),
 * dB_theta/dt = dE_z/dr - dE_r/dz, dE_r/dt = -dB_theta/dz - J_r,
 * dE_z/dt = (1/r) d(r B_theta)/dr - J_z - J_b, with J = -n beta and the rigid
 * driver J_b = -n_b z_hat; conducting z walls and outer wall.
 *
 * Grid: nodes (z_k = k dx, r_j = (j - 1/2) dx), k = 0..nz-1, j = 0..nr-1;
 * row 0 is the mirror image of row 1 (cylindrical symmetry: the axis lies
 * between them), rows 1..nr-2 hold the plasma, row nr-1 and the planes
 * k = 0, nz-1 are Eq. 14 boundary nodes (equilibrium of the clamped interior
 * node). E_z sits at (z_{k+1/2}, r_j), E_r at (z_k, j dx), B_theta at
 * (z_{k+1/2}, j dx). Arrays are [..][z][r], r fastest. Initial state: plasma
 * at rest of density n0, zero fields. */
typedef struct {
    int32_t nz, nr;        /* nodes along z; rows along r including the mirror
                              and outer rows; each >= 3 */
    double dx;             /* dz = dr in c/omega_p, > 0 */
    double dt;             /* 0 selects 0.17628 dx; must be < dx / sqrt(2) */
    double tau;            /* > 0.5 */
    int32_t collision;     /* PWFA_BGK or PWFA_STREAM_ONLY */
    int32_t couple;        /* 1: Lorentz source + Maxwell update; 0: fluid only */
    double n0;             /* plasma density (normalised, >= 0) */
    double alpha, sigma_r, sigma_z, z0;  /* driver: peak n_b/n0, rms sizes, centre at t = 0 */
    double n_floor;        /* 0 selects 1e-6 */
} pwfa_axi_params;

typedef struct pwfa_axi pwfa_axi_t;

/* Allocate the device state and set the initial condition. cuda_stream is a
 * cudaStream_t (NULL = legacy default stream). */
int pwfa_axi_create(const pwfa_axi_params* params, void* cuda_stream, pwfa_axi_t** out);

/* Advance nsteps (>= 0): the fused Faraday + fluid step, then Ampere with
 * the driver at t_{n+1}. Asynchronous on the stream. */
int pwfa_axi_step(pwfa_axi_t* h, int32_t nsteps);

/* out[6][nz][nr] (host or device FP32): n, beta_z, beta_r of the current
 * state, then the raw Yee E_z, E_r (t_{n+1/2}) and B_theta (t_n).
 * Synchronises the stream. */
int pwfa_axi_fields(pwfa_axi_t* h, float* out);

/* The stored streaming source (post-collision populations of the last
 * step, [3][9][nz][nr], D2Q9 order rest, +z, -z, +r, -r, (+z,+r), (-z,-r),
 * (+z,-r), (-z,+r)); the pre-collision state of every interior node is its
 * pull f_i(x) = S_i(x - xi_i). Host or device FP32; synchronises. */
int pwfa_axi_get_source(pwfa_axi_t* h, float* fs);
int pwfa_axi_set_source(pwfa_axi_t* h, const float* fs);

/* Steps taken so far (>= 0), or a negative error code. */
int64_t pwfa_axi_steps_done(pwfa_axi_t* h);

/* Accumulated device time (ms) of the step's kernels since the last call:
 * ms[2] the fused Faraday + fluid kernel, ms[3] Ampere (ms[0], ms[1] stay
 * zero: Faraday's law and the node moments run inside the fluid kernel),
 * from CUDA event pairs recorded while enabled (pwfa_axi_profile).
 * Synchronises. */
int pwfa_axi_profile(pwfa_axi_t* h, int32_t enable);
int pwfa_axi_kernel_times(pwfa_axi_t* h, double* ms, int64_t* launches);

/* Release the device state. Accepts NULL. */
int pwfa_axi_destroy(pwfa_axi_t* h);

#ifdef __cplusplus
}
#endif

#endif /* PWFA_LBM_H */
