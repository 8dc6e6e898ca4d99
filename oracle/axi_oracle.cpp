/*
 * FP64 CPU oracle of the 2D-axisymmetric (z, r) form of the method: the
 * paper's own geometry.
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline / reference arm load this library. The GPU library shares no
 * code, header, table or helper with it.
 *
 * What it computes (Parise et al., arXiv:2201.05473):
 *   - three D2Q9 advection-diffusion lattices on the (z, r) plane for
 *     A = (n, n p_z, n p_r) (Eq. 4), BGK collision (Eq. 7) towards the
 *     equilibrium of Eq. 9 in lattice units (c_s^2 = 1/3), u = beta(p) dt/dx
 *     (Eq. 2), pull streaming (Eq. 6);
 *   - the cylindrical terms of Eq. 13 added to the source of every lattice:
 *     S_i = w_i dt (F + D (1/r) dA/dr - A u_r / r), with the physical
 *     diffusivity D = (tau - 1/2)/3 dx^2/dt (Eq. 12) and dA/dr the central
 *     difference of the node moments at r +- dx (the paper gives the terms
 *     of Eq. 13, not their discretisation: this is the reading used);
 *   - the Lorentz source F = -n (E + beta x B) with only E_z, E_r, B_theta
 *     (axisymmetric TM fields): F_z = -n (E_z + beta_r B_theta),
 *     F_r = -n (E_r - beta_z B_theta);
 *   - Maxwell's equations (Eq. 5, Faraday with Maxwell's sign) on a
 *     cylindrical Yee grid: dB_theta/dt = dE_z/dr - dE_r/dz,
 *     dE_r/dt = -dB_theta/dz - J_r, dE_z/dt = (1/r) d(r B_theta)/dr - J_z,
 *     with J = -n beta (electrons) and the rigid driver J_b = -n_b z_hat.
 *
 * Grid: nodes (z_k, r_j) with z_k = k dx (k = 0..nz-1) and
 * r_j = (j - 1/2) dx (j = 0..nr-1). Row 0 (r = -dx/2) is the mirror row of
 * the axis, rows 1..nr-2 are the plasma, row nr-1 the outer boundary row.
 * E_z sits at (z_{k+1/2}, r_j), E_r at (z_k, j dx), B_theta at
 * (z_{k+1/2}, j dx): E_r and B_theta vanish on the axis (j = 0).
 *
 * Boundaries (Eq. 14, free flux + cylindrical symmetry): the z walls and the
 * outer row hold the equilibrium of the clamped interior node's moments and
 * are collided with the Lorentz source of their own node fields (no
 * cylindrical term), as the open boundary of the 3D form; the axis row is the
 * mirror image of row 1 (cylindrical symmetry): its streaming source is row
 * 1's post-collision populations with the r component of every velocity
 * reversed and the sign of the n p_r lattice flipped, and its state the
 * mirror of row 1's. Fields: perfectly conducting z walls and outer wall
 * (tangential E zero); Yee values outside the grid read as zero.
 *
 * Time staggering as in the 3D oracle: the fluid and B at t_n, E at
 * t_{n+1/2}; Faraday, collision with the mean of the two B levels, pull,
 * boundary rows, Ampere with the post-collision current J = -n* beta(p*) and
 * the driver at t_{n+1}.
 */
#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

namespace {

const int AQ = 9;
const int AL = 3;
// (z, r) components: rest, +z, -z, +r, -r, (+z,+r), (-z,-r), (+z,-r), (-z,+r)
const int AXI[AQ][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {-1, -1}, {1, -1}, {-1, 1}};
// the direction with the r component reversed
const int AREFL[AQ] = {0, 1, 2, 4, 3, 7, 8, 5, 6};

double aweight(int q) {
    if (q == 0) return 4.0 / 9.0;
    if (q <= 4) return 1.0 / 9.0;
    return 1.0 / 36.0;
}

}  // namespace

extern "C" {
typedef struct {
    int32_t nz, nr;       /* nodes along z and rows along r (row 0 = axis mirror row) */
    double dx, dt, tau;
    int32_t collision;    /* 0 BGK, 2 stream only */
    int32_t couple;       /* 1 Lorentz source + Maxwell update */
    double n0;
    double alpha, sigma_r, sigma_z, z0;  /* driver */
    double n_floor;
} axi_params;
}

namespace {

struct Axi {
    axi_params p{};
    int nz = 0, nr = 0;
    int64_t N = 0;
    int64_t steps = 0;
    std::vector<double> f, fs, fn;          // [node][lattice][q]
    std::vector<double> Ez, Er, Bt, Btn;    // Yee arrays [k][j]
    std::vector<double> Jz, Jr;             // node current of the last step

    int64_t idx(int k, int j) const { return (int64_t)k * nr + j; }
    double rnode(int j) const { return (j - 0.5) * p.dx; }
    bool boundary(int k, int j) const { return k == 0 || k == nz - 1 || j == 0 || j == nr - 1; }
    static int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

    static double feq(int q, double A, const double u[2]) {
        const double xu = AXI[q][0] * u[0] + AXI[q][1] * u[1];
        const double uu = u[0] * u[0] + u[1] * u[1];
        return aweight(q) * A * (1.0 + 3.0 * xu + 4.5 * xu * xu - 1.5 * uu);
    }

    // A_l = sum_i f_l,i; p = A_{1,2} / max(n, n_floor); beta = p / sqrt(1 + p^2)
    void moments(const double* fnode, double A[AL], double beta[2]) const {
        for (int l = 0; l < AL; ++l) {
            double s = 0.0;
            for (int q = 0; q < AQ; ++q) s += fnode[l * AQ + q];
            A[l] = s;
        }
        const double nn = A[0] > p.n_floor ? A[0] : p.n_floor;
        const double pz = A[1] / nn, pr = A[2] / nn;
        const double g = std::sqrt(1.0 + pz * pz + pr * pr);
        beta[0] = pz / g;
        beta[1] = pr / g;
    }

    void init() {
        nz = p.nz; nr = p.nr;
        N = (int64_t)nz * nr;
        f.assign(N * AL * AQ, 0.0);
        fs.assign(N * AL * AQ, 0.0);
        fn.assign(N * AL * AQ, 0.0);
        Ez.assign(N, 0.0); Er.assign(N, 0.0); Bt.assign(N, 0.0); Btn.assign(N, 0.0);
        Jz.assign(N, 0.0); Jr.assign(N, 0.0);
        for (int64_t o = 0; o < N; ++o)
            for (int q = 0; q < AQ; ++q) f[o * AL * AQ + q] = aweight(q) * p.n0;
    }

    // driver density at (z, r) and time t
    double driver(double z, double r, double t) const {
        const double zeta = z - p.z0 - t;
        return p.alpha * std::exp(-r * r / (2.0 * p.sigma_r * p.sigma_r) - zeta * zeta / (2.0 * p.sigma_z * p.sigma_z));
    }

    // active Yee components (conducting z walls and outer wall; axis values 0)
    bool act_ez(int k, int j) const { return k <= nz - 2 && j >= 1 && j <= nr - 2; }
    bool act_er(int k, int j) const { return k >= 1 && k <= nz - 2 && j >= 1 && j <= nr - 2; }
    bool act_bt(int k, int j) const { return k <= nz - 2 && j >= 1 && j <= nr - 2; }

    // 1. Faraday: dB_theta/dt = dE_z/dr - dE_r/dz
    void faraday() {
        const double c = p.dt / p.dx;
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < nr; ++j) {
                const int64_t o = idx(k, j);
                Btn[o] = act_bt(k, j)
                    ? Bt[o] - c * ((Er[idx(k + 1, j)] - Er[o]) - (Ez[idx(k, j + 1)] - Ez[o]))
                    : 0.0;
            }
    }

    // Yee value at (k, j), zero outside the grid
    double at(const std::vector<double>& a, int k, int j) const {
        if (k < 0 || j < 0 || k >= nz || j >= nr) return 0.0;
        return a[idx(k, j)];
    }

    // node fields: E_z mean of its two z edges, E_r of its two r edges, B_theta
    // mean of the four surrounding values of both time levels
    void node_fields(int k, int j, double& ez, double& er, double& bt) const {
        ez = 0.5 * (at(Ez, k - 1, j) + at(Ez, k, j));
        er = 0.5 * (at(Er, k, j - 1) + at(Er, k, j));
        double s = 0.0;
        for (int dk = -1; dk <= 0; ++dk)
            for (int dj = -1; dj <= 0; ++dj) s += at(Bt, k + dk, j + dj) + at(Btn, k + dk, j + dj);
        bt = s / 8.0;
    }

    // the axis row as the mirror image of row 1 (cylindrical symmetry)
    void mirror_axis(std::vector<double>& a) const {
        for (int k = 0; k < nz; ++k) {
            const double* src = &a[idx(k, 1) * AL * AQ];
            double* dst = &a[idx(k, 0) * AL * AQ];
            for (int l = 0; l < AL; ++l)
                for (int q = 0; q < AQ; ++q) dst[l * AQ + q] = (l == 2 ? -1.0 : 1.0) * src[l * AQ + AREFL[q]];
        }
    }

    // 2. collision + source (the cylindrical terms on interior nodes only),
    //    then the axis row mirrors row 1. Node currents J = -n* beta(p*) of
    //    the post-collision moments.
    void collide() {
        const double lat = p.dt / p.dx;
        const double om = 1.0 / p.tau;
        const double D = (p.tau - 0.5) / 3.0 * p.dx * p.dx / p.dt;
        std::vector<double> Am(N * AL), Bm(N * 2);
        for (int64_t o = 0; o < N; ++o) moments(&f[o * AL * AQ], &Am[o * AL], &Bm[o * 2]);
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < nr; ++j) {
                const int64_t o = idx(k, j);
                const double* fo = &f[o * AL * AQ];
                double* fso = &fs[o * AL * AQ];
                const double* A = &Am[o * AL];
                const double* beta = &Bm[o * 2];
                if (j == 0) continue;  // the mirror of row 1, filled below
                if (p.collision == 2) {
                    for (int m = 0; m < AL * AQ; ++m) fso[m] = fo[m];
                    const double nn = A[0] > p.n_floor ? A[0] : p.n_floor;
                    const double g = std::sqrt(1.0 + (A[1] / nn) * (A[1] / nn) + (A[2] / nn) * (A[2] / nn));
                    Jz[o] = -A[0] * (A[1] / nn) / g;
                    Jr[o] = -A[0] * (A[2] / nn) / g;
                    continue;
                }
                double F[AL] = {0.0, 0.0, 0.0};
                if (p.couple) {
                    double ez, er, bt;
                    node_fields(k, j, ez, er, bt);
                    F[1] = -A[0] * (ez + beta[1] * bt);
                    F[2] = -A[0] * (er - beta[0] * bt);
                }
                double S[AL] = {F[0], F[1], F[2]};
                if (!boundary(k, j)) {
                    // cylindrical terms of Eq. 13
                    const double r = rnode(j);
                    for (int l = 0; l < AL; ++l) {
                        const double dAdr = (Am[idx(k, j + 1) * AL + l] - Am[idx(k, j - 1) * AL + l]) / (2.0 * p.dx);
                        S[l] += D * dAdr / r - A[l] * beta[1] / r;
                    }
                }
                const double u[2] = {beta[0] * lat, beta[1] * lat};
                for (int l = 0; l < AL; ++l)
                    for (int q = 0; q < AQ; ++q) {
                        const double fl = fo[l * AQ + q];
                        fso[l * AQ + q] = fl - om * (fl - feq(q, A[l], u)) + aweight(q) * S[l] * p.dt;
                    }
                const double ns = A[0] + S[0] * p.dt;
                const double nn = ns > p.n_floor ? ns : p.n_floor;
                const double pz = (A[1] + S[1] * p.dt) / nn, pr = (A[2] + S[2] * p.dt) / nn;
                const double g = std::sqrt(1.0 + pz * pz + pr * pr);
                Jz[o] = -ns * pz / g;
                Jr[o] = -ns * pr / g;
            }
        mirror_axis(fs);
        for (int k = 0; k < nz; ++k) {
            Jz[idx(k, 0)] = Jz[idx(k, 1)];
            Jr[idx(k, 0)] = -Jr[idx(k, 1)];
        }
    }

    // 3. pull streaming of the interior nodes (Eq. 6); 4. the z walls and the
    //    outer row take the equilibrium of the clamped interior node (Eq. 14);
    //    the axis row mirrors row 1
    void stream() {
        const double lat = p.dt / p.dx;
        for (int k = 1; k < nz - 1; ++k)
            for (int j = 1; j < nr - 1; ++j) {
                const int64_t o = idx(k, j);
                for (int q = 0; q < AQ; ++q) {
                    const int64_t so = idx(k - AXI[q][0], j - AXI[q][1]);
                    for (int l = 0; l < AL; ++l) fn[o * AL * AQ + l * AQ + q] = fs[so * AL * AQ + l * AQ + q];
                }
            }
        for (int k = 0; k < nz; ++k)
            for (int j = 1; j < nr; ++j) {
                if (!boundary(k, j)) continue;
                const int kc = clampi(k, 1, nz - 2), jc = clampi(j, 1, nr - 2);
                double A[AL], beta[2];
                moments(&fn[idx(kc, jc) * AL * AQ], A, beta);
                const double u[2] = {beta[0] * lat, beta[1] * lat};
                double* fo = &fn[idx(k, j) * AL * AQ];
                for (int l = 0; l < AL; ++l)
                    for (int q = 0; q < AQ; ++q) fo[l * AQ + q] = feq(q, A[l], u);
            }
        mirror_axis(fn);
    }

    // 5. Ampere: dE_r/dt = -dB_theta/dz - J_r, dE_z/dt = (1/r) d(r B_theta)/dr - J_z - J_b
    void ampere() {
        const double c = p.dt / p.dx, dt = p.dt;
        const double t1 = (steps + 1) * p.dt;
        for (int k = 0; k < nz; ++k)
            for (int j = 0; j < nr; ++j) {
                const int64_t o = idx(k, j);
                if (act_er(k, j)) {
                    const double je = 0.5 * (Jr[o] + Jr[idx(k, j + 1)]);
                    Er[o] = Er[o] - c * (Btn[o] - Btn[idx(k - 1, j)]) - dt * je;
                }
                if (act_ez(k, j)) {
                    const double curl = ((double)j * Btn[o] - (double)(j - 1) * Btn[idx(k, j - 1)]) / (j - 0.5);
                    const double je = 0.5 * (Jz[o] + Jz[idx(k + 1, j)]);
                    const double jb = -driver((k + 0.5) * p.dx, std::fabs(rnode(j)), t1);
                    Ez[o] = Ez[o] + c * curl - dt * (je + jb);
                }
            }
    }

    void step() {
        if (p.couple) faraday();
        else Btn = Bt;
        collide();
        stream();
        if (p.couple) ampere();
        Bt.swap(Btn);
        f.swap(fn);
        ++steps;
    }
};

}  // namespace

extern "C" {

void* axi_create(const axi_params* prm) {
    if (!prm || prm->nz < 3 || prm->nr < 3) return nullptr;
    Axi* s = new (std::nothrow) Axi();
    if (!s) return nullptr;
    s->p = *prm;
    s->init();
    return s;
}

void axi_destroy(void* h) { delete static_cast<Axi*>(h); }

int axi_step(void* h, int32_t nsteps) {
    Axi* s = static_cast<Axi*>(h);
    for (int n = 0; n < nsteps; ++n) s->step();
    return 0;
}

int64_t axi_steps_done(void* h) { return static_cast<Axi*>(h)->steps; }

/* Pre-collision populations, [lattice][q][z][r]. */
void axi_get_f(void* h, double* out) {
    Axi* s = static_cast<Axi*>(h);
    for (int l = 0; l < AL; ++l)
        for (int q = 0; q < AQ; ++q)
            for (int64_t o = 0; o < s->N; ++o) out[(int64_t)(l * AQ + q) * s->N + o] = s->f[o * AL * AQ + l * AQ + q];
}

void axi_set_f(void* h, const double* in) {
    Axi* s = static_cast<Axi*>(h);
    for (int l = 0; l < AL; ++l)
        for (int q = 0; q < AQ; ++q)
            for (int64_t o = 0; o < s->N; ++o) s->f[o * AL * AQ + l * AQ + q] = in[(int64_t)(l * AQ + q) * s->N + o];
}

/* f = f^eq(A, u(A)) at every node, A given as [3][z][r]. */
void axi_set_equilibrium(void* h, const double* A) {
    Axi* s = static_cast<Axi*>(h);
    const double lat = s->p.dt / s->p.dx;
    for (int64_t o = 0; o < s->N; ++o) {
        const double Al[AL] = {A[o], A[s->N + o], A[2 * s->N + o]};
        const double nn = Al[0] > s->p.n_floor ? Al[0] : s->p.n_floor;
        const double pz = Al[1] / nn, pr = Al[2] / nn;
        const double g = std::sqrt(1.0 + pz * pz + pr * pr);
        const double u[2] = {pz / g * lat, pr / g * lat};
        for (int l = 0; l < AL; ++l)
            for (int q = 0; q < AQ; ++q) s->f[o * AL * AQ + l * AQ + q] = Axi::feq(q, Al[l], u);
    }
}

/* Raw Yee arrays [z][r]: E_z, E_r (t_{n+1/2}) and B_theta (t_n). */
void axi_get_fields(void* h, double* Ez, double* Er, double* Bt) {
    Axi* s = static_cast<Axi*>(h);
    for (int64_t o = 0; o < s->N; ++o) { Ez[o] = s->Ez[o]; Er[o] = s->Er[o]; Bt[o] = s->Bt[o]; }
}

void axi_set_fields(void* h, const double* Ez, const double* Er, const double* Bt) {
    Axi* s = static_cast<Axi*>(h);
    for (int64_t o = 0; o < s->N; ++o) { s->Ez[o] = Ez[o]; s->Er[o] = Er[o]; s->Bt[o] = Bt[o]; }
}

/* Node moments [6][z][r]: n, beta_z, beta_r, A_1 = n p_z, A_2 = n p_r, |beta|. */
void axi_moments(void* h, double* out) {
    Axi* s = static_cast<Axi*>(h);
    const int64_t N = s->N;
    for (int64_t o = 0; o < N; ++o) {
        double A[AL], beta[2];
        s->moments(&s->f[o * AL * AQ], A, beta);
        out[o] = A[0];
        out[N + o] = beta[0];
        out[2 * N + o] = beta[1];
        out[3 * N + o] = A[1];
        out[4 * N + o] = A[2];
        out[5 * N + o] = std::sqrt(beta[0] * beta[0] + beta[1] * beta[1]);
    }
}

/* The streaming source (post-collision populations of the last step,
 * [lattice][q][z][r]). */
void axi_get_source(void* h, double* out) {
    Axi* s = static_cast<Axi*>(h);
    for (int l = 0; l < AL; ++l)
        for (int q = 0; q < AQ; ++q)
            for (int64_t o = 0; o < s->N; ++o) out[(int64_t)(l * AQ + q) * s->N + o] = s->fs[o * AL * AQ + l * AQ + q];
}

/* Set the streaming source and pull the pre-collision state from it (Eq. 6,
 * Eq. 14 boundary rows, mirror row). */
void axi_set_source(void* h, const double* in) {
    Axi* s = static_cast<Axi*>(h);
    for (int l = 0; l < AL; ++l)
        for (int q = 0; q < AQ; ++q)
            for (int64_t o = 0; o < s->N; ++o) s->fs[o * AL * AQ + l * AQ + q] = in[(int64_t)(l * AQ + q) * s->N + o];
    s->stream();
    s->f.swap(s->fn);
}

/* Node currents of the last step [z][r] (plasma only). */
void axi_last_current(void* h, double* Jz, double* Jr) {
    Axi* s = static_cast<Axi*>(h);
    for (int64_t o = 0; o < s->N; ++o) { Jz[o] = s->Jz[o]; Jr[o] = s->Jr[o]; }
}

}  // extern "C"
