// Device-side building blocks of the GB300 LBM plasma-wakefield step.
//
// D3Q19 velocity set (Sec. III uses D2Q9; the 3D analogue keeps the same
// construction: rest particle, nearest neighbours, diagonals), storage codecs
// for the populations, and the argument blocks passed to every kernel.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace pwfa {

constexpr int kQ = 19;   // velocities per lattice
constexpr int kL = 4;    // lattices: n, n p_x, n p_y, n p_z (Eq. 4)
constexpr int kPop = kQ * kL;

// Canonical D3Q19 order: 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 the edge
// diagonals (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1) (1,0,-1)
// (-1,0,1) (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1). Opposites are (2m-1, 2m).
__host__ __device__ __forceinline__ constexpr int xi_x(int q) {
    return (q == 1 || q == 7 || q == 9 || q == 11 || q == 13) ? 1
         : (q == 2 || q == 8 || q == 10 || q == 12 || q == 14) ? -1 : 0;
}
__host__ __device__ __forceinline__ constexpr int xi_y(int q) {
    return (q == 3 || q == 7 || q == 10 || q == 15 || q == 17) ? 1
         : (q == 4 || q == 8 || q == 9 || q == 16 || q == 18) ? -1 : 0;
}
__host__ __device__ __forceinline__ constexpr int xi_z(int q) {
    return (q == 5 || q == 11 || q == 14 || q == 15 || q == 18) ? 1
         : (q == 6 || q == 12 || q == 13 || q == 16 || q == 17) ? -1 : 0;
}
// Lattice weights: 1/3 rest, 1/18 axis, 1/36 diagonal (c_s^2 = 1/3).
__host__ __device__ __forceinline__ constexpr float wq(int q) {
    return q == 0 ? (1.0f / 3.0f) : (q <= 6 ? (1.0f / 18.0f) : (1.0f / 36.0f));
}

// ------------------------------------------------------------ storage codecs
// FP32 stores f itself. BF16/FP16 store the deviation from the plasma at rest
// (w_i n0 for lattice 0, 0 for the momentum lattices) so that the short
// mantissa resolves the perturbation rather than the background. FP16 also
// scales the deviation by 2^10 / w_i: without it the small deviations of
// lattice 0 (w_i dn ~ 1e-6) fall into FP16's subnormal range; with it FP16
// holds |deviation / w_i| up to ~64 (n p <= 64) at full relative precision.
__host__ __device__ __forceinline__ constexpr float dev_base(int l, int q, float n0) {
    return l == 0 ? wq(q) * n0 : 0.0f;
}
constexpr float kF16Scale = 1024.0f;

template <int ST> struct Codec;

template <> struct Codec<0> {
    using T = float;
    static __device__ __forceinline__ float load(const T* p, int, int, float) { return __ldg(p); }
    static __device__ __forceinline__ void store(T* p, float v, int, int, float) { __stcs(p, v); }
};
// The 16-bit codecs also move the pair of lattices (l0, l0 + 1) that share a
// 32-bit word (see pop_elem): p points at the word's first (even) element.
template <> struct Codec<1> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float load(const T* p, int l, int q, float n0) {
        return __bfloat162float(__ldg(p)) + dev_base(l, q, n0);
    }
    static __device__ __forceinline__ void store(T* p, float v, int l, int q, float n0) {
        *p = __float2bfloat16_rn(v - dev_base(l, q, n0));
    }
    static __device__ __forceinline__ void from_word(uint32_t u, int l0, int q, float n0, float& v0, float& v1) {
        const float2 w = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
        v0 = w.x + dev_base(l0, q, n0);
        v1 = w.y + dev_base(l0 + 1, q, n0);
    }
    static __device__ __forceinline__ void load2(const T* p, int l0, int q, float n0, float& v0, float& v1) {
        from_word(__ldg(reinterpret_cast<const unsigned int*>(p)), l0, q, n0, v0, v1);
    }
    static __device__ __forceinline__ void store2(T* p, float v0, float v1, int l0, int q, float n0) {
        *reinterpret_cast<__nv_bfloat162*>(p) =
            __floats2bfloat162_rn(v0 - dev_base(l0, q, n0), v1 - dev_base(l0 + 1, q, n0));
    }
    // stored units: f = kappa(q) s + dev_base (raw access, no conversion)
    static __host__ __device__ constexpr float kappa(int) { return 1.0f; }
    static __device__ __forceinline__ void load2raw(const T* p, float& s0, float& s1) {
        const unsigned int u = __ldg(reinterpret_cast<const unsigned int*>(p));
        const float2 w = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
        s0 = w.x;
        s1 = w.y;
    }
    static __device__ __forceinline__ void store2raw(T* p, float s0, float s1) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(s0, s1);
    }
};
template <> struct Codec<2> {
    using T = __half;
    static __device__ __forceinline__ float load(const T* p, int l, int q, float n0) {
        return __half2float(__ldg(p)) * (wq(q) / kF16Scale) + dev_base(l, q, n0);
    }
    static __device__ __forceinline__ void store(T* p, float v, int l, int q, float n0) {
        *p = __float2half_rn((v - dev_base(l, q, n0)) * (kF16Scale / wq(q)));
    }
    static __device__ __forceinline__ void from_word(uint32_t u, int l0, int q, float n0, float& v0, float& v1) {
        const float2 w = __half22float2(*reinterpret_cast<const __half2*>(&u));
        v0 = w.x * (wq(q) / kF16Scale) + dev_base(l0, q, n0);
        v1 = w.y * (wq(q) / kF16Scale) + dev_base(l0 + 1, q, n0);
    }
    static __device__ __forceinline__ void load2(const T* p, int l0, int q, float n0, float& v0, float& v1) {
        from_word(__ldg(reinterpret_cast<const unsigned int*>(p)), l0, q, n0, v0, v1);
    }
    static __device__ __forceinline__ void store2(T* p, float v0, float v1, int l0, int q, float n0) {
        *reinterpret_cast<__half2*>(p) = __floats2half2_rn((v0 - dev_base(l0, q, n0)) * (kF16Scale / wq(q)),
                                                            (v1 - dev_base(l0 + 1, q, n0)) * (kF16Scale / wq(q)));
    }
    static __host__ __device__ constexpr float kappa(int q) { return wq(q) / kF16Scale; }
    static __device__ __forceinline__ void load2raw(const T* p, float& s0, float& s1) {
        const unsigned int u = __ldg(reinterpret_cast<const unsigned int*>(p));
        const float2 w = __half22float2(*reinterpret_cast<const __half2*>(&u));
        s0 = w.x;
        s1 = w.y;
    }
    static __device__ __forceinline__ void store2raw(T* p, float s0, float s1) {
        *reinterpret_cast<__half2*>(p) = __floats2half2_rn(s0, s1);
    }
};

// ------------------------------------------------------------ debug builds
// With PWFA_DEBUG defined, the step kernels check each element index they
// compute against the extent of the array it addresses before the access.
// An index outside [lo, hi) is recorded in the instance's debug word (dbg[0]:
// site of the first failure, dbg[1]: its index, dbg[2]: failures counted) and
// replaced by lo, so nothing outside the allocation is read or written; the
// host then fails the call with PWFA_ERR_STATE. Release builds compile the
// checks away. Sites: 1 pulled source node, 2 stored node, 3 node-average
// field read, 4 Faraday, 5 Ampere, 6 fused field step, 7 adjoint scatter.
#ifdef PWFA_DEBUG
static __device__ __noinline__ void debug_record(unsigned* dbg, unsigned site, long long i) {
    if (!dbg) return;
    if (atomicCAS(dbg, 0u, site) == 0u) dbg[1] = (unsigned)i;
    atomicAdd(dbg + 2, 1u);
}
template <class I>
__device__ __forceinline__ I debug_index(unsigned* dbg, I i, long long lo, long long hi, unsigned site) {
    const long long v = (long long)i;
    if (v < lo || v >= hi) {
        debug_record(dbg, site, v);
        return (I)lo;
    }
    return i;
}
#define PWFA_CHECK(dbg, i, lo, hi, site) ::pwfa::debug_index((dbg), (i), (long long)(lo), (long long)(hi), (site))
#else
#define PWFA_CHECK(dbg, i, lo, hi, site) (i)
#endif

// ------------------------------------------------------------ kernel args
struct Grid {
    int nx, ny, nz;
    int64_t N;        // nx * ny * nz
    int64_t Np;       // population nodes: N (plus, with a moving window, one
                      // trailing plane of fresh plasma) rounded up to 32
    int periodic;     // 1: every axis wraps; 0: open (Eq. 14) + conducting walls
};

// Population layout in HBM: four lattice blocks of 19 * Np elements; inside
// a block, nodes are grouped in chunks of 32 and a chunk holds its 19
// populations one after another: (q, node) sits at
// (node / 32) * 19 * 32 + q * 32 + node % 32. A warp's 19 loads of one lattice
// thus fall in one 2.4 KB region (FP32) instead of 19 far-apart planes.
__host__ __device__ __forceinline__ uint32_t pop_off(int q, uint32_t node) {
    return (node >> 5) * (uint32_t)(kQ * 32) + (uint32_t)q * 32u + (node & 31u);
}
__host__ __device__ __forceinline__ int64_t lattice_stride(const Grid& g) { return (int64_t)kQ * g.Np; }

// Element index of population (l, i) at chunked offset off (LS = 19 Np).
// FP32 keeps one block per lattice. The 16-bit forms pair the lattices
// (0, 1) and (2, 3) in 32-bit words, so that a thread's loads and stores each
// move two values: pair block p holds 19 Np words and word off holds
// {lattice 2p, lattice 2p + 1}. Both forms take 76 Np elements.
template <int ST>
__host__ __device__ __forceinline__ int64_t pop_elem(int l, uint32_t off, int64_t LS) {
    return ST == 0 ? (int64_t)l * LS + off : (int64_t)(l >> 1) * 2 * LS + 2 * (int64_t)off + (l & 1);
}

// One instance's device state as the step kernels see it.
struct StepArgs {
    Grid g;
    const void* fin;      // stored post-collision populations, 76 planes of N
    void* fout;
    const float* E[3];    // Yee E at t_{n+1/2}
    const float* Bc[3];   // Yee B at t_n
    float* Bn[3];         // Yee B at t_{n+1} (written by Faraday)
    float* Eout[3];       // E updated in place by Ampere
    float* J[3];          // node current -n beta(p*) of the step
    float omega;          // 1 / tau
    float lat;            // dt / dx: physical velocity -> lattice units
    float dt;
    float cdt;            // dt / dx for the curls
    float n_floor;
    float n0;             // background (deviation storage base)
    int couple;
    // driver: J_b,z = -alpha exp(-r^2/(2 sr^2) - (z - zc)^2/(2 sz^2)) at t_{n+1}
    float alpha, inv2sr2, inv2sz2, zc, dx;
    float* Jb[3];         // PIC driver: deposited current on the E edges (else null);
                          // Ampere zeroes what it consumes, so the arrays stay
                          // zero outside the box of the last deposit
    int* jbox;            // PIC driver: [lo x, y, z, hi x, y, z] node box of this
                          // step's deposit (hi < lo: none)
    int* jbox_next;       // the other step parity's box, emptied by Ampere
    uint32_t src_shift;   // added to every pulled source node: nx*ny on a step
                          // that moves the window (the streaming source is
                          // read one plane up), else 0
    int bx, by;           // fluid kernel block shape (autotuned per instance)
    int staged;           // 1: software-pipelined fluid kernel (FP32 storage), 128-thread tiles
    unsigned* dbg;        // debug builds: the instance's index-error word (see PWFA_CHECK)
    float* mom;           // adjoint recompute (launch_fluid_mom): each node's lattice
                          // sums A_l are stored here too ([4][N]); unused otherwise
};

// Elements of the zero guard in front of every Yee/current array (one x-y
// plane, one row and one element): the lowest index a node average reads.
__host__ __device__ __forceinline__ int64_t guard_elems(const Grid& g) {
    return (int64_t)g.nx * g.ny + g.nx + 1;
}

__device__ __forceinline__ int wrapi(int a, int n) {
    return a < 0 ? a + n : (a >= n ? a - n : a);
}

}  // namespace pwfa
