/*
 * FP64 CPU oracle of the lattice-Boltzmann plasma-wakefield step.
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference arm load this library. The GPU library shares no
 * code, header, table or helper with it.
 *
 * What it computes (Parise et al., arXiv:2201.05473), one time step:
 *   - the electron plasma as four advection-diffusion lattices (Sec. III,
 *     "three LBM descriptions" generalised to three Cartesian momentum
 *     components): A = (n, n p_x, n p_y, n p_z), Eq. 4;
 *   - each lattice D3Q19 with BGK collision (Eq. 7), equilibrium Eq. 9 read in
 *     lattice units (c_s^2 = 1/3, consistent with D = (tau - 1/2)/3 of Eq. 12),
 *     source S_i = w_i F dt (Eq. 10) and pull streaming (Eq. 6);
 *   - the advecting velocity u = beta(p) of Eq. 2 (third line), shared by all
 *     four lattices (Eq. 4), in lattice units u = beta dt/dx;
 *   - the Lorentz source F = -n (E + beta x B) of Eq. 4;
 *   - boundary nodes set to the equilibrium of the zero-gradient ("free flux")
 *     extrapolated moments, Eq. 14;
 *   - Maxwell's equations (Eq. 5) on a Yee grid with FDTD leapfrog, Faraday's
 *     law with Maxwell's sign dB/dt = -curl E, currents J_e = -n beta (electron
 *     charge -1) and a rigid bi-Gaussian electron driver J_b = -n_b z_hat
 *     moving at c.
 *
 * Units: time 1/omega_p, length c/omega_p, density n0, momentum m_e c,
 * fields m_e c omega_p / e. Then dB/dt = -curl E, dE/dt = curl B - J.
 *
 * Time staggering (the paper leaves it open; this is the reading used):
 *   at the start of step n the fluid (populations f^n) and B sit at t_n and E
 *   sits at t_{n+1/2}. One step:
 *     1. Faraday   B(t_{n+1}) = B(t_n) - dt curl E
 *     2. collide   every node, force with E and B(t_{n+1/2}) = mean of the two
 *                  B levels, both averaged to the node
 *     3. stream    pull, f^{n+1}(x) = f*(x - xi_i)
 *     4. boundary  (open mode) boundary nodes := f^eq of the moments of the
 *                  clamped interior node, Eq. 14
 *     5. Ampere    E += dt (curl B(t_{n+1}) - J), with the plasma current
 *                  J = -n beta(p*) built from the post-collision momentum
 *                  p* = (A_k + F_k dt)/n and the driver current at t_{n+1}.
 *   For a uniform plasma this reduces exactly to the symplectic recurrence
 *   p' = p - dt E, E' = E + dt beta(p'), i.e. the cold-plasma oscillation at
 *   omega_p with the leapfrog phase error.
 *
 * Boundaries: "open" = Eq. 14 equilibrium boundary nodes for the lattices plus
 * perfectly conducting walls for the fields (tangential E and normal B stay
 * zero on the six outer planes); "periodic" wraps every axis.
 *
 * Moving window (Sec. II: the simulation box moves with the driver; open
 * mode only). After n steps the box has moved W_n = max(0, floor((z0 + n dt
 * - window_z) / dx)) planes along +z, so the driver centre, once it reaches
 * window_z, stays within one cell of it. A step n with W_{n+1} > W_n first
 * moves the box one plane: the streaming source (the post-collision
 * populations of the previous step), E and the current B level move down one
 * plane, the bottom plane leaves the box, the top plane is filled with
 * unperturbed plasma at rest (the streaming source of the initial state,
 * zero fields), the conducting walls are imposed on the moved fields, and the
 * pre-collision populations are pulled again from the moved source. The
 * step then runs as usual, the driver evaluated at lab position z + W dx.
 *
 * PIC driver (Eq. 1, instead of the rigid bunch): macro-electrons of weight
 * w (electrons in units of n0 (c/omega_p)^3) with positions at t_{n+1/2} (the
 * time level of E) and momenta at t_n (that of B). In step n, after the
 * fluid, each is pushed by the Boris scheme (charge/mass -1) with E(t_{n+1/2})
 * and the mean of B(t_n), B(t_{n+1}), both interpolated trilinearly from each
 * component's own Yee lattice at x_{n+1/2}, to p_{n+1}; it moves to
 * x_{n+3/2} = x_{n+1/2} + dt p_{n+1}/gamma_{n+1}, and the current of that
 * move is deposited on the E edges by the charge-conserving scheme of
 * Esirkepov (Comput. Phys. Commun. 135, 2001) for the linear (cloud-in-cell)
 * shape, so that the driver's charge obeys the discrete continuity equation
 * exactly; Ampere subtracts it as J_b. Particles outside an open grid see no
 * field and deposit only on in-grid edges.
 *
 * The scalar type is a template parameter so that the same step can run on
 * forward-mode dual numbers for derivatives.
 */
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#include <new>

namespace {

// ---------------------------------------------------------------- D3Q19 set
// Canonical order: rest, 6 axis neighbours, 12 edge diagonals; opposite pairs
// are (2m-1, 2m). Weights 1/3, 1/18, 1/36 (c_s^2 = 1/3).
const int NQ = 19;
const int NL = 4;
const int XI[NQ][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

double weight(int q) {
    if (q == 0) return 1.0 / 3.0;
    if (q <= 6) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

enum { COLL_BGK = 0, COLL_REG = 1, COLL_NONE = 2 };
enum { BND_OPEN = 0, BND_PERIODIC = 1 };

// ---------------------------------------------------------------- scalars
// Forward-mode dual number with ND tangent directions.
template <int ND>
struct Dual {
    double v;
    double d[ND];
    Dual() : v(0.0) { for (int k = 0; k < ND; ++k) d[k] = 0.0; }
    Dual(double x) : v(x) { for (int k = 0; k < ND; ++k) d[k] = 0.0; }
};
template <int ND> Dual<ND> operator+(const Dual<ND>& a, const Dual<ND>& b) {
    Dual<ND> r; r.v = a.v + b.v; for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] + b.d[k]; return r; }
template <int ND> Dual<ND> operator-(const Dual<ND>& a, const Dual<ND>& b) {
    Dual<ND> r; r.v = a.v - b.v; for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] - b.d[k]; return r; }
template <int ND> Dual<ND> operator-(const Dual<ND>& a) {
    Dual<ND> r; r.v = -a.v; for (int k = 0; k < ND; ++k) r.d[k] = -a.d[k]; return r; }
template <int ND> Dual<ND> operator*(const Dual<ND>& a, const Dual<ND>& b) {
    Dual<ND> r; r.v = a.v * b.v; for (int k = 0; k < ND; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k]; return r; }
template <int ND> Dual<ND> operator/(const Dual<ND>& a, const Dual<ND>& b) {
    Dual<ND> r; r.v = a.v / b.v;
    for (int k = 0; k < ND; ++k) { r.d[k] = (a.d[k] - r.v * b.d[k]) / b.v; }
    return r; }
template <int ND> Dual<ND>& operator+=(Dual<ND>& a, const Dual<ND>& b) { a = a + b; return a; }
template <int ND> Dual<ND>& operator-=(Dual<ND>& a, const Dual<ND>& b) { a = a - b; return a; }
template <int ND> Dual<ND> sqrt(const Dual<ND>& a) {
    Dual<ND> r; r.v = std::sqrt(a.v);
    for (int k = 0; k < ND; ++k) { r.d[k] = a.d[k] / (2.0 * r.v); }
    return r; }
template <int ND> Dual<ND> exp(const Dual<ND>& a) {
    Dual<ND> r; r.v = std::exp(a.v);
    for (int k = 0; k < ND; ++k) { r.d[k] = a.d[k] * r.v; }
    return r; }
template <int ND> double val(const Dual<ND>& a) { return a.v; }
inline double val(double a) { return a; }
using std::sqrt;
using std::exp;

// ---------------------------------------------------------------- params
}  // namespace

extern "C" {
typedef struct {
    int32_t nx, ny, nz;
    double dx, dt, tau;
    int32_t collision;   /* 0 BGK (Eq. 7), 1 regularized BGK, 2 none (stream only) */
    int32_t boundary;    /* 0 open (Eq. 14 + conducting walls), 1 periodic */
    int32_t couple;      /* 1 Lorentz force + Maxwell update, 0 fluid only */
    double n0;
    const double* profile; /* radial multiplier of n0, n_profile points, or null */
    int32_t n_profile;
    double profile_rmax;
    double alpha, sigma_r, sigma_z, z0; /* driver: peak n_b/n0, rms sizes, centre at t=0 */
    double n_floor;
    int32_t moving_window; /* 1: the box follows the driver (open mode only) */
    double window_z;       /* box position held by the driver centre once reached */
    int32_t driver;        /* 0 rigid bi-Gaussian bunch, 1 macro-particles (PIC, Eq. 1) */
} oracle_params;
}

namespace {

template <class S>
struct Sim {
    oracle_params p;
    // parameters that may carry tangents
    S alpha, sigma_r, sigma_z;
    std::vector<S> prof;
    int nx, ny, nz;
    int64_t N;
    int64_t step_count = 0;
    std::vector<S> f, fs, fn;          // AoS populations [node][lattice][q]
    std::vector<S> E[3], B[3], Bn[3];  // Yee arrays [k][j][i]
    std::vector<S> Jn[3];              // node current of the last step
    std::vector<S> Fn[4];              // node source of the last step
    std::vector<S> EN[3], BN[3];       // node fields used by the last step
    bool fs_valid = true;              // fs is the streaming source of f
    bool shift_failed = false;         // a window move found no valid source
    // PIC driver: x, y, z (t_{n+1/2}), p_x, p_y, p_z (t_n); weight; the
    // driver current of the last step on the E edges
    std::vector<S> P[6];
    double pw = 0.0;
    std::vector<S> Jb[3];

    int64_t idx(int i, int j, int k) const { return ((int64_t)k * ny + j) * nx + i; }
    bool periodic() const { return p.boundary == BND_PERIODIC; }
    int wrap(int a, int n) const { return ((a % n) + n) % n; }

    // Value of a Yee array at integer index (i,j,k): wraps when periodic,
    // zero outside the grid otherwise.
    S at(const std::vector<S>& a, int i, int j, int k) const {
        if (periodic()) return a[idx(wrap(i, nx), wrap(j, ny), wrap(k, nz))];
        if (i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz) return S(0.0);
        return a[idx(i, j, k)];
    }

    bool boundary_node(int i, int j, int k) const {
        if (periodic()) return false;
        return i == 0 || j == 0 || k == 0 || i == nx - 1 || j == ny - 1 || k == nz - 1;
    }
    static int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

    // Radial density multiplier: piecewise linear over r_j = j rmax/(np-1),
    // held at the last value beyond rmax.
    S profile_at(double r) const {
        if (prof.empty()) return S(1.0);
        int np = (int)prof.size();
        if (np == 1) return prof[0];
        double h = p.profile_rmax / (np - 1);
        if (r >= p.profile_rmax) return prof[np - 1];
        double t = r / h;
        int j = (int)std::floor(t);
        if (j >= np - 1) return prof[np - 1];
        double fr = t - j;
        return S(1.0 - fr) * prof[j] + S(fr) * prof[j + 1];
    }
    double radius(int i, int j) const {
        double xc = 0.5 * (nx - 1) * p.dx, yc = 0.5 * (ny - 1) * p.dx;
        double x = i * p.dx - xc, y = j * p.dx - yc;
        return std::sqrt(x * x + y * y);
    }

    // Equilibrium of Eq. 9 in lattice units (c_s^2 = 1/3).
    static S feq(int q, const S& A, const S u[3]) {
        S xu = S((double)XI[q][0]) * u[0] + S((double)XI[q][1]) * u[1] + S((double)XI[q][2]) * u[2];
        S uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        return S(weight(q)) * A * (S(1.0) + S(3.0) * xu + S(4.5) * xu * xu - S(1.5) * uu);
    }

    // Moments of one node's populations: A_l = sum_i f_{l,i} (Eq. 8, first
    // line), p = A_{1..3}/max(n, n_floor), beta = p / sqrt(1 + |p|^2) (Eq. 2).
    void moments(const S* fnode, S A[NL], S pvec[3], S beta[3]) const {
        for (int l = 0; l < NL; ++l) {
            S s(0.0);
            for (int q = 0; q < NQ; ++q) s += fnode[l * NQ + q];
            A[l] = s;
        }
        S nn = val(A[0]) > p.n_floor ? A[0] : S(p.n_floor);
        for (int c = 0; c < 3; ++c) pvec[c] = A[c + 1] / nn;
        S g = sqrt(S(1.0) + pvec[0] * pvec[0] + pvec[1] * pvec[1] + pvec[2] * pvec[2]);
        for (int c = 0; c < 3; ++c) beta[c] = pvec[c] / g;
    }

    void init() {
        nx = p.nx; ny = p.ny; nz = p.nz;
        N = (int64_t)nx * ny * nz;
        f.assign(N * NL * NQ, S(0.0));
        fs.assign(N * NL * NQ, S(0.0));
        fn.assign(N * NL * NQ, S(0.0));
        for (int c = 0; c < 3; ++c) {
            E[c].assign(N, S(0.0)); B[c].assign(N, S(0.0)); Bn[c].assign(N, S(0.0));
            Jn[c].assign(N, S(0.0)); EN[c].assign(N, S(0.0)); BN[c].assign(N, S(0.0));
        }
        for (int l = 0; l < NL; ++l) Fn[l].assign(N, S(0.0));
        // Initial state: cold plasma at rest, density n0 * profile(r), i.e.
        // f = f^eq(A = (n0 prof, 0, 0, 0), u = 0) = w_i n0 prof. Open-mode
        // boundary nodes take the value of their clamped interior node (Eq. 14).
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    int ic = i, jc = j;
                    if (boundary_node(i, j, k)) { ic = clampi(i, 1, nx - 2); jc = clampi(j, 1, ny - 2); }
                    S n = S(p.n0) * profile_at(radius(ic, jc));
                    S* fnode = &f[idx(i, j, k) * NL * NQ];
                    for (int q = 0; q < NQ; ++q) fnode[q] = S(weight(q)) * n;
                    fresh_source(i, j, &fs[idx(i, j, k) * NL * NQ]);
                }
        fs_valid = true;
    }

    // Streaming source of the plasma at rest: the post-collision populations
    // whose pull gives f = w_i n0 prof(r) at every node, i.e. f*_i(x) =
    // w_i n0 prof(r(x + xi_i)) on lattice 0 (transverse position wrapped, or
    // clamped to the interior on open grids) and zero on the momentum lattices.
    void fresh_source(int i, int j, S* fnode) const {
        for (int l = 0; l < NL; ++l)
            for (int q = 0; q < NQ; ++q) fnode[l * NQ + q] = S(0.0);
        for (int q = 0; q < NQ; ++q) {
            int si = i + XI[q][0], sj = j + XI[q][1];
            if (periodic()) { si = wrap(si, nx); sj = wrap(sj, ny); }
            else { si = clampi(si, 1, nx - 2); sj = clampi(sj, 1, ny - 2); }
            fnode[q] = S(weight(q)) * S(p.n0) * profile_at(radius(si, sj));
        }
    }

    // Planes the moving window has advanced after n steps.
    int64_t window_planes(int64_t n) const {
        if (!p.moving_window) return 0;
        const double v = std::floor((p.z0 + (double)n * p.dt - p.window_z) / p.dx);
        return v > 0.0 ? (int64_t)v : 0;
    }

    // Driver density n_b at (x, y, z) and time t: alpha * exp(-r^2/2 sr^2 - (z - z0 - t)^2 / 2 sz^2).
    S driver(double x, double y, double z, double t) const {
        double xc = 0.5 * (nx - 1) * p.dx, yc = 0.5 * (ny - 1) * p.dx;
        double r2 = (x - xc) * (x - xc) + (y - yc) * (y - yc);
        double zeta = z - p.z0 - t;
        S a = S(-r2) / (S(2.0) * sigma_r * sigma_r) - S(zeta * zeta) / (S(2.0) * sigma_z * sigma_z);
        return alpha * exp(a);
    }

    // ---- active Yee components (open mode = conducting walls) ----
    bool act_bx(int i, int j, int k) const { return periodic() || (i >= 1 && i <= nx - 2 && j <= ny - 2 && k <= nz - 2); }
    bool act_by(int i, int j, int k) const { return periodic() || (i <= nx - 2 && j >= 1 && j <= ny - 2 && k <= nz - 2); }
    bool act_bz(int i, int j, int k) const { return periodic() || (i <= nx - 2 && j <= ny - 2 && k >= 1 && k <= nz - 2); }
    bool act_ex(int i, int j, int k) const { return periodic() || (i <= nx - 2 && j >= 1 && j <= ny - 2 && k >= 1 && k <= nz - 2); }
    bool act_ey(int i, int j, int k) const { return periodic() || (i >= 1 && i <= nx - 2 && j <= ny - 2 && k >= 1 && k <= nz - 2); }
    bool act_ez(int i, int j, int k) const { return periodic() || (i >= 1 && i <= nx - 2 && j >= 1 && j <= ny - 2 && k <= nz - 2); }

    // 1. Faraday: Bn = B - dt curl E. E_x at (i+1/2,j,k), E_y at (i,j+1/2,k),
    //    E_z at (i,j,k+1/2); B_x at (i,j+1/2,k+1/2) and cyclic.
    void faraday() {
        const S c(p.dt / p.dx);
#pragma omp parallel for schedule(static)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    int64_t o = idx(i, j, k);
                    Bn[0][o] = act_bx(i, j, k)
                        ? B[0][o] - c * ((at(E[2], i, j + 1, k) - at(E[2], i, j, k)) - (at(E[1], i, j, k + 1) - at(E[1], i, j, k)))
                        : S(0.0);
                    Bn[1][o] = act_by(i, j, k)
                        ? B[1][o] - c * ((at(E[0], i, j, k + 1) - at(E[0], i, j, k)) - (at(E[2], i + 1, j, k) - at(E[2], i, j, k)))
                        : S(0.0);
                    Bn[2][o] = act_bz(i, j, k)
                        ? B[2][o] - c * ((at(E[1], i + 1, j, k) - at(E[1], i, j, k)) - (at(E[0], i, j + 1, k) - at(E[0], i, j, k)))
                        : S(0.0);
                }
    }

    // Fields at a node: E averaged over the two adjacent edges, B = mean of the
    // two time levels averaged over the four adjacent faces.
    void node_fields(int i, int j, int k, S e[3], S b[3]) const {
        e[0] = S(0.5) * (at(E[0], i - 1, j, k) + at(E[0], i, j, k));
        e[1] = S(0.5) * (at(E[1], i, j - 1, k) + at(E[1], i, j, k));
        e[2] = S(0.5) * (at(E[2], i, j, k - 1) + at(E[2], i, j, k));
        auto bh = [&](int c, int a, int bb, int cc) { return S(0.5) * (at(B[c], a, bb, cc) + at(Bn[c], a, bb, cc)); };
        b[0] = S(0.25) * (bh(0, i, j, k) + bh(0, i, j - 1, k) + bh(0, i, j, k - 1) + bh(0, i, j - 1, k - 1));
        b[1] = S(0.25) * (bh(1, i, j, k) + bh(1, i - 1, j, k) + bh(1, i, j, k - 1) + bh(1, i - 1, j, k - 1));
        b[2] = S(0.25) * (bh(2, i, j, k) + bh(2, i - 1, j, k) + bh(2, i, j - 1, k) + bh(2, i - 1, j - 1, k));
    }

    // 2. Collision + source at every node (Eqs. 6, 7, 9, 10).
    void collide() {
        const double tau = p.tau;
        const double lat = p.dt / p.dx;  // physical velocity -> lattice units
#pragma omp parallel for schedule(static)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    int64_t o = idx(i, j, k);
                    const S* fo = &f[o * NL * NQ];
                    S* fso = &fs[o * NL * NQ];
                    S A[NL], pv[3], beta[3];
                    moments(fo, A, pv, beta);
                    S e[3] = {S(0.0), S(0.0), S(0.0)}, b[3] = {S(0.0), S(0.0), S(0.0)};
                    if (p.couple) node_fields(i, j, k, e, b);
                    for (int c = 0; c < 3; ++c) { EN[c][o] = e[c]; BN[c][o] = b[c]; }
                    // Lorentz source, Eq. 4: F_0 = 0, F_k = -n (E + beta x B)_k
                    S F[NL];
                    F[0] = S(0.0);
                    F[1] = -A[0] * (e[0] + beta[1] * b[2] - beta[2] * b[1]);
                    F[2] = -A[0] * (e[1] + beta[2] * b[0] - beta[0] * b[2]);
                    F[3] = -A[0] * (e[2] + beta[0] * b[1] - beta[1] * b[0]);
                    if (!p.couple || p.collision == COLL_NONE) for (int l = 0; l < NL; ++l) F[l] = S(0.0);
                    for (int l = 0; l < NL; ++l) Fn[l][o] = F[l];
                    S u[3] = {beta[0] * S(lat), beta[1] * S(lat), beta[2] * S(lat)};
                    for (int l = 0; l < NL; ++l) {
                        const S* fl = fo + l * NQ;
                        S* fsl = fso + l * NQ;
                        if (p.collision == COLL_NONE) {
                            for (int q = 0; q < NQ; ++q) fsl[q] = fl[q];
                            continue;
                        }
                        S fe[NQ];
                        for (int q = 0; q < NQ; ++q) fe[q] = feq(q, A[l], u);
                        if (p.collision == COLL_BGK) {
                            // Eq. 7: f* = f - (f - f^eq)/tau + w_i F dt
                            for (int q = 0; q < NQ; ++q)
                                fsl[q] = fl[q] - (fl[q] - fe[q]) / S(tau) + S(weight(q) * p.dt) * F[l];
                        } else {
                            // Regularized: keep only the first Hermite moment of
                            // the non-equilibrium part, Pi = sum_i xi_i (f_i - f_i^eq),
                            // f* = f^eq + (1 - 1/tau) 3 w_i xi_i . Pi + w_i F dt.
                            S Pi[3] = {S(0.0), S(0.0), S(0.0)};
                            for (int q = 0; q < NQ; ++q)
                                for (int c = 0; c < 3; ++c)
                                    if (XI[q][c] != 0) Pi[c] += S((double)XI[q][c]) * (fl[q] - fe[q]);
                            for (int q = 0; q < NQ; ++q) {
                                S xp = S((double)XI[q][0]) * Pi[0] + S((double)XI[q][1]) * Pi[1] + S((double)XI[q][2]) * Pi[2];
                                fsl[q] = fe[q] + S((1.0 - 1.0 / tau) * 3.0 * weight(q)) * xp + S(weight(q) * p.dt) * F[l];
                            }
                        }
                    }
                    // Plasma current for Ampere: J = -n beta(p*), p* the
                    // post-collision momentum (A_k + F_k dt) / max(n, n_floor).
                    S nn = val(A[0]) > p.n_floor ? A[0] : S(p.n_floor);
                    S ps[3];
                    for (int c = 0; c < 3; ++c) ps[c] = (A[c + 1] + F[c + 1] * S(p.dt)) / nn;
                    S g = sqrt(S(1.0) + ps[0] * ps[0] + ps[1] * ps[1] + ps[2] * ps[2]);
                    for (int c = 0; c < 3; ++c) Jn[c][o] = -A[0] * ps[c] / g;
                }
    }

    // 3. Pull streaming, f^{n+1}_i(x) = f*_i(x - xi_i) (Eq. 6).
    // 4. Open boundary: boundary nodes := f^eq(A(x_c), u(x_c)), x_c the
    //    clamped interior node, moments taken after streaming (Eq. 14).
    void stream() {
#pragma omp parallel for schedule(static)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    if (boundary_node(i, j, k)) continue;
                    int64_t o = idx(i, j, k);
                    for (int q = 0; q < NQ; ++q) {
                        int si = i - XI[q][0], sj = j - XI[q][1], sk = k - XI[q][2];
                        if (periodic()) { si = wrap(si, nx); sj = wrap(sj, ny); sk = wrap(sk, nz); }
                        int64_t so = idx(si, sj, sk);
                        for (int l = 0; l < NL; ++l) fn[o * NL * NQ + l * NQ + q] = fs[so * NL * NQ + l * NQ + q];
                    }
                }
        if (periodic()) return;
        const double lat = p.dt / p.dx;
#pragma omp parallel for schedule(static)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    if (!boundary_node(i, j, k)) continue;
                    int ic = clampi(i, 1, nx - 2), jc = clampi(j, 1, ny - 2), kc = clampi(k, 1, nz - 2);
                    S A[NL], pv[3], beta[3];
                    moments(&fn[idx(ic, jc, kc) * NL * NQ], A, pv, beta);
                    S u[3] = {beta[0] * S(lat), beta[1] * S(lat), beta[2] * S(lat)};
                    S* fo = &fn[idx(i, j, k) * NL * NQ];
                    for (int l = 0; l < NL; ++l)
                        for (int q = 0; q < NQ; ++q) fo[l * NQ + q] = feq(q, A[l], u);
                }
    }

    // ---- PIC driver
    // Component a at grid coordinates (gx, gy, gz) of its own Yee lattice:
    // trilinear in the eight surrounding values.
    S interp(const std::vector<S>& a, const S& gx, const S& gy, const S& gz) const {
        const int i0 = (int)std::floor(val(gx)), j0 = (int)std::floor(val(gy)), k0 = (int)std::floor(val(gz));
        const S fx = gx - S((double)i0), fy = gy - S((double)j0), fz = gz - S((double)k0);
        S r(0.0);
        for (int c = 0; c < 2; ++c)
            for (int b = 0; b < 2; ++b)
                for (int a2 = 0; a2 < 2; ++a2) {
                    const S wx = a2 ? fx : S(1.0) - fx, wy = b ? fy : S(1.0) - fy, wz = c ? fz : S(1.0) - fz;
                    r += wx * wy * wz * at(a, i0 + a2, j0 + b, k0 + c);
                }
        return r;
    }
    // linear (cloud-in-cell) shape
    static S hat(const S& t) {
        const S at_ = val(t) < 0.0 ? -t : t;
        return val(at_) < 1.0 ? S(1.0) - at_ : S(0.0);
    }
    void add_edge(std::vector<S>& a, int i, int j, int k, const S& v) {
        if (periodic()) { i = wrap(i, nx); j = wrap(j, ny); k = wrap(k, nz); }
        else if (i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz) return;
        a[idx(i, j, k)] += v;
    }
    // Esirkepov's charge-conserving current of one move (grid coordinates in
    // cells, node-centred; |move| < 1 cell per axis), on a 3-node stencil per
    // axis: W_x = dSx (S0y S0z + dSy S0z / 2 + S0y dSz / 2 + dSy dSz / 3) and
    // cyclic, J_x(i + 1/2) = w / (dx^2 dt) sum_{i' <= i} W_x(i').
    void deposit(const S g0[3], const S g1[3]) {
        int base[3];
        S s0[3][3], ds[3][3];
        for (int d = 0; d < 3; ++d) {
            base[d] = (int)std::floor(std::min(val(g0[d]), val(g1[d])));
            for (int m = 0; m < 3; ++m) {
                const S node((double)(base[d] + m));
                s0[d][m] = hat(g0[d] - node);
                ds[d][m] = hat(g1[d] - node) - s0[d][m];
            }
        }
        const S coef(pw / (p.dx * p.dx * p.dt));
        const S half(0.5), third(1.0 / 3.0);
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c) {
                S run(0.0);
                for (int a2 = 0; a2 < 2; ++a2) {
                    run += ds[0][a2] * (s0[1][b] * s0[2][c] + half * ds[1][b] * s0[2][c] + half * s0[1][b] * ds[2][c] +
                                        third * ds[1][b] * ds[2][c]);
                    add_edge(Jb[0], base[0] + a2, base[1] + b, base[2] + c, coef * run);
                }
            }
        for (int a2 = 0; a2 < 3; ++a2)
            for (int c = 0; c < 3; ++c) {
                S run(0.0);
                for (int b = 0; b < 2; ++b) {
                    run += ds[1][b] * (s0[0][a2] * s0[2][c] + half * ds[0][a2] * s0[2][c] + half * s0[0][a2] * ds[2][c] +
                                       third * ds[0][a2] * ds[2][c]);
                    add_edge(Jb[1], base[0] + a2, base[1] + b, base[2] + c, coef * run);
                }
            }
        for (int a2 = 0; a2 < 3; ++a2)
            for (int b = 0; b < 3; ++b) {
                S run(0.0);
                for (int c = 0; c < 2; ++c) {
                    run += ds[2][c] * (s0[0][a2] * s0[1][b] + half * ds[0][a2] * s0[1][b] + half * s0[0][a2] * ds[1][b] +
                                       third * ds[0][a2] * ds[1][b]);
                    add_edge(Jb[2], base[0] + a2, base[1] + b, base[2] + c, coef * run);
                }
            }
    }
    // Boris push of every macro-electron and the deposit of its move
    void push_deposit() {
        for (int c = 0; c < 3; ++c) Jb[c].assign(N, S(0.0));
        const S dt(p.dt), hdt(0.5 * p.dt), inv_dx(1.0 / p.dx);
        const double L[3] = {nx * p.dx, ny * p.dx, nz * p.dx};
        const size_t np = P[0].size();
        for (size_t m = 0; m < np; ++m) {
            const S g[3] = {P[0][m] * inv_dx, P[1][m] * inv_dx, P[2][m] * inv_dx};
            const S h(0.5);
            const S e[3] = {interp(E[0], g[0] - h, g[1], g[2]), interp(E[1], g[0], g[1] - h, g[2]),
                            interp(E[2], g[0], g[1], g[2] - h)};
            const S b[3] = {h * (interp(B[0], g[0], g[1] - h, g[2] - h) + interp(Bn[0], g[0], g[1] - h, g[2] - h)),
                            h * (interp(B[1], g[0] - h, g[1], g[2] - h) + interp(Bn[1], g[0] - h, g[1], g[2] - h)),
                            h * (interp(B[2], g[0] - h, g[1] - h, g[2]) + interp(Bn[2], g[0] - h, g[1] - h, g[2]))};
            // Boris, q/m = -1: half kick, rotation, half kick
            S um[3], up[3], pn[3];
            for (int c = 0; c < 3; ++c) um[c] = P[3 + c][m] - hdt * e[c];
            const S gm = sqrt(S(1.0) + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
            S tv[3];
            for (int c = 0; c < 3; ++c) tv[c] = -hdt * b[c] / gm;
            const S t2 = tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2];
            S sv[3];
            for (int c = 0; c < 3; ++c) sv[c] = S(2.0) * tv[c] / (S(1.0) + t2);
            const S w1[3] = {um[0] + (um[1] * tv[2] - um[2] * tv[1]), um[1] + (um[2] * tv[0] - um[0] * tv[2]),
                             um[2] + (um[0] * tv[1] - um[1] * tv[0])};
            up[0] = um[0] + (w1[1] * sv[2] - w1[2] * sv[1]);
            up[1] = um[1] + (w1[2] * sv[0] - w1[0] * sv[2]);
            up[2] = um[2] + (w1[0] * sv[1] - w1[1] * sv[0]);
            for (int c = 0; c < 3; ++c) pn[c] = up[c] - hdt * e[c];
            const S gn = sqrt(S(1.0) + pn[0] * pn[0] + pn[1] * pn[1] + pn[2] * pn[2]);
            S xn[3], g1[3];
            for (int c = 0; c < 3; ++c) {
                xn[c] = P[c][m] + dt * pn[c] / gn;
                g1[c] = xn[c] * inv_dx;
            }
            deposit(g, g1);
            for (int c = 0; c < 3; ++c) {
                if (periodic()) {
                    const double v = val(xn[c]);
                    if (v < 0.0) xn[c] += S(L[c]);
                    else if (v >= L[c]) xn[c] -= S(L[c]);
                }
                P[c][m] = xn[c];
                P[3 + c][m] = pn[c];
            }
        }
    }

    // 5. Ampere: E += dt (curl B(t_{n+1}) - J_e - J_b), J_e averaged from the
    //    two nodes of each edge, J_b,z = -n_b at t_{n+1} (rigid bunch) or the
    //    deposited current of the PIC driver.
    void ampere() {
        const S c(p.dt / p.dx);
        const S dt(p.dt);
        const double t1 = (step_count + 1) * p.dt;
        const int64_t zshift = window_planes(step_count + 1);  // box position at t_{n+1}
#pragma omp parallel for schedule(static)
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    int64_t o = idx(i, j, k);
                    const bool pic = p.driver == 1;
                    if (act_ex(i, j, k)) {
                        S curl = (at(Bn[2], i, j, k) - at(Bn[2], i, j - 1, k)) - (at(Bn[1], i, j, k) - at(Bn[1], i, j, k - 1));
                        S Je = S(0.5) * (at(Jn[0], i, j, k) + at(Jn[0], i + 1, j, k));
                        if (pic) Je += Jb[0][o];
                        E[0][o] = E[0][o] + c * curl - dt * Je;
                    }
                    if (act_ey(i, j, k)) {
                        S curl = (at(Bn[0], i, j, k) - at(Bn[0], i, j, k - 1)) - (at(Bn[2], i, j, k) - at(Bn[2], i - 1, j, k));
                        S Je = S(0.5) * (at(Jn[1], i, j, k) + at(Jn[1], i, j + 1, k));
                        if (pic) Je += Jb[1][o];
                        E[1][o] = E[1][o] + c * curl - dt * Je;
                    }
                    if (act_ez(i, j, k)) {
                        S curl = (at(Bn[1], i, j, k) - at(Bn[1], i - 1, j, k)) - (at(Bn[0], i, j, k) - at(Bn[0], i, j - 1, k));
                        S Je = S(0.5) * (at(Jn[2], i, j, k) + at(Jn[2], i, j, k + 1));
                        S Jd = pic ? Jb[2][o] : -driver(i * p.dx, j * p.dx, (k + 0.5 + (double)zshift) * p.dx, t1);
                        E[2][o] = E[2][o] + c * curl - dt * (Je + Jd);
                    }
                }
    }

    // Move the box one plane along +z (see the header).
    void shift_window() {
        std::vector<S> src(fs.size());
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    S* d = &src[idx(i, j, k) * NL * NQ];
                    if (k + 1 < nz) {
                        const S* s = &fs[idx(i, j, k + 1) * NL * NQ];
                        for (int m = 0; m < NL * NQ; ++m) d[m] = s[m];
                    } else {
                        fresh_source(i, j, d);
                    }
                }
        fs.swap(src);
        stream();
        f.swap(fn);
        for (int c = 0; c < 3; ++c) {
            std::vector<S> e(N, S(0.0)), b(N, S(0.0));
            for (int k = 0; k + 1 < nz; ++k)
                for (int j = 0; j < ny; ++j)
                    for (int i = 0; i < nx; ++i) {
                        const bool ae = c == 0 ? act_ex(i, j, k) : (c == 1 ? act_ey(i, j, k) : act_ez(i, j, k));
                        const bool ab = c == 0 ? act_bx(i, j, k) : (c == 1 ? act_by(i, j, k) : act_bz(i, j, k));
                        if (ae) e[idx(i, j, k)] = E[c][idx(i, j, k + 1)];
                        if (ab) b[idx(i, j, k)] = B[c][idx(i, j, k + 1)];
                    }
            E[c].swap(e);
            B[c].swap(b);
        }
    }

    void step() {
        if (p.moving_window && window_planes(step_count + 1) > window_planes(step_count)) {
            if (!fs_valid || periodic()) { shift_failed = true; return; }
            shift_window();
        }
        if (p.couple) faraday();
        else for (int c = 0; c < 3; ++c) Bn[c] = B[c];
        collide();
        stream();
        if (p.driver == 1) push_deposit();
        if (p.couple) ampere();
        for (int c = 0; c < 3; ++c) B[c].swap(Bn[c]);
        f.swap(fn);
        fs_valid = true;
        ++step_count;
    }
};

// Layout helpers between the AoS state and the [lattice][q][z][y][x] export.
template <class S>
void export_f(const Sim<S>& s, double* out) {
    for (int l = 0; l < NL; ++l)
        for (int q = 0; q < NQ; ++q)
            for (int64_t o = 0; o < s.N; ++o) out[(int64_t)(l * NQ + q) * s.N + o] = val(s.f[o * NL * NQ + l * NQ + q]);
}

}  // namespace

extern "C" {

void* oracle_create(const oracle_params* prm) {
    if (!prm || prm->nx < 3 || prm->ny < 3 || prm->nz < 3) return nullptr;
    if (prm->driver == 1 && prm->moving_window) return nullptr;
    Sim<double>* s = new (std::nothrow) Sim<double>();
    if (!s) return nullptr;
    s->p = *prm;
    if (prm->profile && prm->n_profile > 0) s->prof.assign(prm->profile, prm->profile + prm->n_profile);
    s->p.profile = nullptr;
    s->alpha = prm->alpha; s->sigma_r = prm->sigma_r; s->sigma_z = prm->sigma_z;
    s->init();
    return s;
}

void oracle_destroy(void* h) { delete static_cast<Sim<double>*>(h); }

int oracle_step(void* h, int32_t nsteps) {
    Sim<double>* s = static_cast<Sim<double>*>(h);
    for (int n = 0; n < nsteps; ++n) {
        s->step();
        if (s->shift_failed) return -1;
    }
    return 0;
}

/* PIC driver macro-electrons: xp[6][n] = x, y, z at t_{n+1/2} and p_x, p_y,
 * p_z at t_n; weight in electrons per n0 (c/omega_p)^3. */
void oracle_set_particles(void* h, int64_t n, const double* xp, double weight) {
    Sim<double>* s = static_cast<Sim<double>*>(h);
    for (int c = 0; c < 6; ++c) s->P[c].assign(xp + c * n, xp + (c + 1) * n);
    s->pw = weight;
}

void oracle_get_particles(void* h, double* out) {
    Sim<double>* s = static_cast<Sim<double>*>(h);
    const size_t n = s->P[0].size();
    for (int c = 0; c < 6; ++c)
        for (size_t m = 0; m < n; ++m) out[c * n + m] = s->P[c][m];
}

/* Driver current of the last step on the E edges, [3][z][y][x] (PIC only). */
void oracle_driver_current(void* h, double* out) {
    Sim<double>* s = static_cast<Sim<double>*>(h);
    for (int c = 0; c < 3; ++c)
        for (int64_t o = 0; o < s->N; ++o) out[c * s->N + o] = s->Jb[c].empty() ? 0.0 : s->Jb[c][o];
}

/* Planes the moving window has advanced so far (0 without a window). */
int64_t oracle_window_planes(void* h) {
    Sim<double>* s = static_cast<Sim<double>*>(h);
    return s->window_planes(s->step_count);
}

/* Set the streaming source (post-collision populations, [lattice][q][z][y][x])
 * and pull the pre-collision state from it (Eq. 6, Eq. 14). */
void oracle_set_source(void* h, const double* in) {
    Sim<double>* s = static_cast<Sim<double>*>(h);
    for (int l = 0; l < NL; ++l)
        for (int q = 0; q < NQ; ++q)
            for (int64_t o = 0; o < s->N; ++o) s->fs[o * NL * NQ + l * NQ + q] = in[(int64_t)(l * NQ + q) * s->N + o];
    s->stream();
    s->f.swap(s->fn);
    s->fs_valid = true;
}

int64_t oracle_steps_done(void* h) { return static_cast<Sim<double>*>(h)->step_count; }

/* Pre-collision populations f^n, [lattice][q][z][y][x]. */
void oracle_get_f(void* h, double* out) { export_f(*static_cast<Sim<double>*>(h), out); }

void oracle_set_f(void* h, const double* in) {
    Sim<double>* s = static_cast<Sim<double>*>(h);
    s->fs_valid = false;  // the streaming source of this state is unknown
    for (int l = 0; l < NL; ++l)
        for (int q = 0; q < NQ; ++q)
            for (int64_t o = 0; o < s->N; ++o) s->f[o * NL * NQ + l * NQ + q] = in[(int64_t)(l * NQ + q) * s->N + o];
}

/* f = f^eq(A, u(A)) at every node, A given as [4][z][y][x]. */
void oracle_set_equilibrium(void* h, const double* A) {
    Sim<double>* s = static_cast<Sim<double>*>(h);
    s->fs_valid = false;
    const double lat = s->p.dt / s->p.dx;
    for (int64_t o = 0; o < s->N; ++o) {
        double Al[NL];
        for (int l = 0; l < NL; ++l) Al[l] = A[l * s->N + o];
        double nn = Al[0] > s->p.n_floor ? Al[0] : s->p.n_floor;
        double pv[3] = {Al[1] / nn, Al[2] / nn, Al[3] / nn};
        double g = std::sqrt(1.0 + pv[0] * pv[0] + pv[1] * pv[1] + pv[2] * pv[2]);
        double u[3] = {pv[0] / g * lat, pv[1] / g * lat, pv[2] / g * lat};
        for (int l = 0; l < NL; ++l)
            for (int q = 0; q < NQ; ++q) s->f[o * NL * NQ + l * NQ + q] = Sim<double>::feq(q, Al[l], u);
    }
}

/* Raw Yee arrays, each [3][z][y][x]: E at t_{n+1/2}, B at t_n. */
void oracle_get_fields(void* h, double* E, double* B) {
    Sim<double>* s = static_cast<Sim<double>*>(h);
    for (int c = 0; c < 3; ++c)
        for (int64_t o = 0; o < s->N; ++o) { E[c * s->N + o] = s->E[c][o]; B[c * s->N + o] = s->B[c][o]; }
}

void oracle_set_fields(void* h, const double* E, const double* B) {
    Sim<double>* s = static_cast<Sim<double>*>(h);
    for (int c = 0; c < 3; ++c)
        for (int64_t o = 0; o < s->N; ++o) { s->E[c][o] = E[c * s->N + o]; s->B[c][o] = B[c * s->N + o]; }
}

/* Node moments of the current populations, [8][z][y][x]:
 * n, beta_x, beta_y, beta_z, A_1, A_2, A_3, |beta|. */
void oracle_moments(void* h, double* out) {
    Sim<double>* s = static_cast<Sim<double>*>(h);
    const int64_t N = s->N;
    for (int64_t o = 0; o < N; ++o) {
        double A[NL], pv[3], beta[3];
        s->moments(&s->f[o * NL * NQ], A, pv, beta);
        out[0 * N + o] = A[0];
        for (int c = 0; c < 3; ++c) { out[(1 + c) * N + o] = beta[c]; out[(4 + c) * N + o] = A[c + 1]; }
        out[7 * N + o] = std::sqrt(beta[0] * beta[0] + beta[1] * beta[1] + beta[2] * beta[2]);
    }
}

/* Quantities of the last step: node current J [3][N], source F [4][N],
 * node fields E [3][N] and B [3][N] used by the force. */
void oracle_last_step(void* h, double* J, double* F, double* En, double* Bnode) {
    Sim<double>* s = static_cast<Sim<double>*>(h);
    const int64_t N = s->N;
    for (int64_t o = 0; o < N; ++o) {
        for (int c = 0; c < 3; ++c) {
            if (J) J[c * N + o] = s->Jn[c][o];
            if (En) En[c * N + o] = s->EN[c][o];
            if (Bnode) Bnode[c * N + o] = s->BN[c][o];
        }
        if (F) for (int l = 0; l < NL; ++l) F[l * N + o] = s->Fn[l][o];
    }
}

/* Global FP64 diagnostics: [0] sum n, [1..3] sum A_k, [4] field energy
 * 1/2 sum (E^2 + B^2) dx^3, [5] min n, [6] max |beta|, [7] non-finite count. */
void oracle_diag(void* h, double* out) {
    Sim<double>* s = static_cast<Sim<double>*>(h);
    double sn = 0, sa[3] = {0, 0, 0}, en = 0, mn = 1e300, mb = 0, bad = 0;
    for (int64_t o = 0; o < s->N; ++o) {
        double A[NL], pv[3], beta[3];
        s->moments(&s->f[o * NL * NQ], A, pv, beta);
        if (!std::isfinite(A[0]) || !std::isfinite(A[1]) || !std::isfinite(A[2]) || !std::isfinite(A[3])) bad += 1;
        sn += A[0];
        for (int c = 0; c < 3; ++c) sa[c] += A[c + 1];
        mn = std::min(mn, A[0]);
        mb = std::max(mb, std::sqrt(beta[0] * beta[0] + beta[1] * beta[1] + beta[2] * beta[2]));
        for (int c = 0; c < 3; ++c) en += s->E[c][o] * s->E[c][o] + s->B[c][o] * s->B[c][o];
    }
    out[0] = sn; out[1] = sa[0]; out[2] = sa[1]; out[3] = sa[2];
    out[4] = 0.5 * en * s->p.dx * s->p.dx * s->p.dx;
    out[5] = mn; out[6] = mb; out[7] = bad;
}

/* Forward-mode derivatives. Parameters theta = (alpha, sigma_r, sigma_z,
 * profile[0 .. n_profile-1]); dirs holds ndir (1..4) tangent directions of
 * length 3 + n_profile. Runs nsteps from the initial state on dual numbers
 * and returns the raw Yee E (value, [3][N]) and its directional derivatives
 * dE ([ndir][3][N]). The same step code as the primal path, templated on the
 * scalar type. */
int oracle_tangent_run(const oracle_params* prm, int32_t nsteps, int32_t ndir, const double* dirs,
                       double* E, double* dE) {
    if (!prm || ndir < 1 || ndir > 4 || nsteps < 0 || prm->driver != 0) return -1;
    using D = Dual<4>;
    Sim<D>* s = new (std::nothrow) Sim<D>();
    if (!s) return -1;
    s->p = *prm;
    const int np = prm->profile && prm->n_profile > 0 ? prm->n_profile : 0;
    const int nt = 3 + np;
    auto seed = [&](double v, int idx) {
        D d(v);
        for (int k = 0; k < ndir; ++k) d.d[k] = dirs[k * nt + idx];
        return d;
    };
    s->alpha = seed(prm->alpha, 0);
    s->sigma_r = seed(prm->sigma_r, 1);
    s->sigma_z = seed(prm->sigma_z, 2);
    for (int j = 0; j < np; ++j) s->prof.push_back(seed(prm->profile[j], 3 + j));
    s->p.profile = nullptr;
    s->init();
    for (int n = 0; n < nsteps; ++n) s->step();
    const int64_t N = s->N;
    for (int c = 0; c < 3; ++c)
        for (int64_t o = 0; o < N; ++o) {
            E[c * N + o] = s->E[c][o].v;
            for (int k = 0; k < ndir; ++k) dE[((int64_t)k * 3 + c) * N + o] = s->E[c][o].d[k];
        }
    delete s;
    return 0;
}

/* Normalised charge of Eq. 15, read with k_p^{+3} (the printed exponent -3
 * is dimensionally inconsistent): Q = (2 pi)^{3/2} sx sy sz alpha k_p^3.
 * Inputs in SI units: sigmas in metres, n0 in m^-3; k_p = omega_p / c;
 * alpha = n_b / n0 with n_b the peak density of a bi-Gaussian of that charge. */
double oracle_qtilde(double charge_coulomb, double sx, double sy, double sz, double n0_m3, double* alpha_out) {
    const double PI = 3.14159265358979323846;
    const double e = 1.602176634e-19, me = 9.1093837015e-31, eps0 = 8.8541878128e-12, c = 299792458.0;
    double nb = charge_coulomb / e / (std::pow(2.0 * PI, 1.5) * sx * sy * sz);
    double alpha = nb / n0_m3;
    if (alpha_out) *alpha_out = alpha;
    double wp = std::sqrt(n0_m3 * e * e / (eps0 * me));
    double kp = wp / c;
    return std::pow(2.0 * PI, 1.5) * sx * sy * sz * alpha * kp * kp * kp;
}

}  // extern "C"
