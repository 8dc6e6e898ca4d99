"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: exact moment
identities of the D3Q19 equilibrium (Eq. 9), exact balance laws of the source
term (Eq. 10), brute-force index streaming (Eq. 6), exact moment recursions and
the diffusivity of Eq. 12, closed-form Yee dispersion (Eq. 5), the cold-plasma
oscillation of Eqs. 2 + 5, the linear-wake wavelength 2 pi c / omega_p, and the
paper's own normalised-charge numbers (Eq. 15, Sec. IV).
"""
import math
import os

import numpy as np
import pytest

from paper_2201_05473_gb300 import workloads as W

# D3Q19 as written from the velocity-set definition: rest, the six axis
# neighbours and the twelve edge diagonals, weights 1/3, 1/18, 1/36.
XI = np.array([[0, 0, 0],
               [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
               [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0],
               [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1],
               [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]])
WQ = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(np.asarray(b).ravel()), 1e-300))


def beta_of(p):
    """Eq. 2, third line, in units of m_e c."""
    return p / np.sqrt(1.0 + np.sum(p * p, axis=0))


def make(oracle_mod, nx, ny, nz, **kw):
    kw.setdefault("dx", 0.2)
    kw.setdefault("dt", W.DT_OVER_DX * kw["dx"])
    kw.setdefault("tau", 0.8)
    return oracle_mod.Oracle(nx, ny, nz, **kw)


# --------------------------------------------------------------------- Eq. 9
def test_velocity_set_is_d3q19_lattice(oracle_mod):
    # isotropy the equilibrium relies on: sum w = 1, sum w xi_a xi_b = delta/3,
    # odd moments vanish, fourth moment isotropic
    assert abs(WQ.sum() - 1) < 1e-15
    assert np.allclose(np.einsum("q,qa,qb->ab", WQ, XI, XI), np.eye(3) / 3, atol=1e-15)
    assert np.allclose(np.einsum("q,qa->a", WQ, XI), 0)
    assert np.allclose(np.einsum("q,qa,qb,qc->abc", WQ, XI, XI, XI), 0)


def test_equilibrium_moments_exact(oracle_mod):
    """Eq. 9 in lattice units: sum f = A, sum xi f = A u, sum xi xi f = A(I/3 + u u)."""
    shape = (3, 4, 5)
    o = make(oracle_mod, 5, 4, 3, boundary=oracle_mod.BND_PERIODIC)
    rng = np.random.default_rng(7)
    A = np.empty((4,) + shape)
    A[0] = 0.5 + rng.random(shape)
    A[1:] = A[0] * rng.uniform(-2, 2, (3,) + shape)
    o.set_equilibrium(A)
    f = o.get_f()
    p = A[1:] / A[0]
    u = beta_of(p) * o.params["dt"] / o.params["dx"]
    for l in range(4):
        s0 = f[l].sum(axis=0)
        s1 = np.einsum("qa,q...->a...", XI, f[l])
        s2 = np.einsum("qa,qb,q...->ab...", XI, XI, f[l])
        assert np.allclose(s0, A[l], rtol=1e-14, atol=1e-15)
        assert np.allclose(s1, A[l] * u, rtol=1e-12, atol=1e-15)
        want2 = A[l] * (np.eye(3)[:, :, None, None, None] / 3 + u[:, None] * u[None, :])
        assert np.allclose(s2, want2, rtol=1e-12, atol=1e-15)


# --------------------------------------------------------------------- Eq. 6
@pytest.mark.parametrize("shape", [(4, 4, 4), (5, 3, 7)])
def test_stream_only_is_exact_permutation(oracle_mod, shape):
    """Collision off: one step moves every population by its lattice vector."""
    nz, ny, nx = shape
    o = make(oracle_mod, nx, ny, nz, collision=oracle_mod.COLL_NONE,
             boundary=oracle_mod.BND_PERIODIC, couple=0)
    f0 = W.integer_populations(shape)
    o.set_f(f0)
    o.step(3)
    got = o.get_f()
    for q in range(19):
        shift = (3 * XI[q][2], 3 * XI[q][1], 3 * XI[q][0])
        want = np.roll(f0[:, q], shift=shift, axis=(1, 2, 3))
        assert np.array_equal(got[:, q], want), q


def test_stream_brute_force_index_table(oracle_mod):
    """4x4x4 periodic: every value lands at (x + xi) mod 4 (explicit table)."""
    o = make(oracle_mod, 4, 4, 4, collision=oracle_mod.COLL_NONE,
             boundary=oracle_mod.BND_PERIODIC, couple=0)
    f0 = W.integer_populations((4, 4, 4))
    o.set_f(f0)
    o.step(1)
    got = o.get_f()
    for l in range(4):
        for q in range(19):
            for z in range(4):
                for y in range(4):
                    for x in range(4):
                        d = ((z + XI[q][2]) % 4, (y + XI[q][1]) % 4, (x + XI[q][0]) % 4)
                        assert got[l, q][d] == f0[l, q, z, y, x]


# -------------------------------------------------------------- Eq. 7 and 10
def _random_state(oracle_mod, o, seed, field_scale=0.05):
    rng = np.random.default_rng(seed)
    o.set_f(W.random_populations(o.shape, seed=seed))
    E = field_scale * rng.standard_normal((3,) + o.shape)
    B = field_scale * rng.standard_normal((3,) + o.shape)
    o.set_fields(E, B)


@pytest.mark.parametrize("collision", [0, 1])
def test_mass_conserved_momentum_balance(oracle_mod, collision):
    """Periodic: sum A_0 is conserved; sum A_k changes by exactly dt sum F_k."""
    o = make(oracle_mod, 6, 5, 4, collision=collision, boundary=oracle_mod.BND_PERIODIC, tau=0.7)
    _random_state(oracle_mod, o, 3)
    dt = o.params["dt"]
    for _ in range(4):
        A_before = o.get_f().sum(axis=1).reshape(4, -1).sum(axis=1)
        o.step(1)
        A_after = o.get_f().sum(axis=1).reshape(4, -1).sum(axis=1)
        F = o.last_step()["F"].reshape(4, -1).sum(axis=1)
        assert abs(A_after[0] - A_before[0]) < 1e-13 * abs(A_before[0])
        assert F[0] == 0 and np.all(np.abs(F[1:]) > 1e-4)  # forcing is really on
        assert np.allclose(A_after[1:] - A_before[1:], dt * F[1:], rtol=1e-11, atol=1e-14)


def test_source_term_and_bgk_tau_one(oracle_mod):
    """BGK at tau = 1 returns f^eq(A, u) + w_i F dt (Eqs. 7, 9, 10), and the
    source is F = -n (E + beta x B) with the node fields used by the step."""
    o = make(oracle_mod, 5, 4, 6, boundary=oracle_mod.BND_PERIODIC, tau=1.0)
    _random_state(oracle_mod, o, 11)
    f0 = o.get_f()
    o.step(1)
    f1 = o.get_f()
    ls = o.last_step()
    dt, dx = o.params["dt"], o.params["dx"]
    A = f0.sum(axis=1)
    beta = beta_of(A[1:] / A[0])
    u = beta * dt / dx
    e, b = ls["E_node"], ls["B_node"]
    F_want = -A[0] * (e + np.cross(beta, b, axis=0))
    assert np.allclose(ls["F"][1:], F_want, rtol=1e-12, atol=1e-15)
    assert np.all(ls["F"][0] == 0)
    xu = np.einsum("qa,a...->q...", XI, u)
    uu = (u * u).sum(axis=0)
    for l in range(4):
        feq = WQ[:, None, None, None] * A[l] * (1 + 3 * xu + 4.5 * xu ** 2 - 1.5 * uu)
        post = feq + WQ[:, None, None, None] * ls["F"][l] * dt
        # undo the streaming of the stored result
        unstreamed = np.stack([np.roll(f1[l, q], shift=(-XI[q][2], -XI[q][1], -XI[q][0]), axis=(0, 1, 2))
                               for q in range(19)])
        assert np.allclose(unstreamed, post, rtol=1e-12, atol=1e-16), l


def test_node_fields_are_yee_averages(oracle_mod):
    """E at a node = mean of its two edges; B = mean of four faces of the two time levels."""
    o = make(oracle_mod, 5, 4, 6, boundary=oracle_mod.BND_PERIODIC)
    _random_state(oracle_mod, o, 5)
    E0, B0 = o.get_fields()
    o.step(1)
    _, B1 = o.get_fields()
    ls = o.last_step()
    r = lambda a, s: np.roll(a, shift=s, axis=(0, 1, 2))
    Ex = 0.5 * (E0[0] + r(E0[0], (0, 0, 1)))
    Ey = 0.5 * (E0[1] + r(E0[1], (0, 1, 0)))
    Ez = 0.5 * (E0[2] + r(E0[2], (1, 0, 0)))
    Bh = 0.5 * (B0 + B1)
    Bx = 0.25 * (Bh[0] + r(Bh[0], (0, 1, 0)) + r(Bh[0], (1, 0, 0)) + r(Bh[0], (1, 1, 0)))
    By = 0.25 * (Bh[1] + r(Bh[1], (0, 0, 1)) + r(Bh[1], (1, 0, 0)) + r(Bh[1], (1, 0, 1)))
    Bz = 0.25 * (Bh[2] + r(Bh[2], (0, 0, 1)) + r(Bh[2], (0, 1, 0)) + r(Bh[2], (0, 1, 1)))
    assert np.allclose(ls["E_node"], np.stack([Ex, Ey, Ez]), atol=1e-15)
    assert np.allclose(ls["B_node"], np.stack([Bx, By, Bz]), atol=1e-15)


# ---------------------------------------------------------------- Eq. 11, 12
def _moment_recursion(tau, M0, u, nsteps):
    """Exact second moment of an equilibrium-started ADE lattice (uniform u):
    from the streaming and BGK rules, R = sum xi f* = M0 u, P = sum xi^2 f
    = M0 (1/3 + u^2), Q_{n+1} = (1-1/tau) Q_n + u Z_n / tau + P,
    Z_{n+1} = Z_n + M0 u, S_{n+1} = S_n + 2[(1-1/tau) Q_n + u Z_n / tau] + P."""
    P = M0 * (1.0 / 3.0 + u * u)
    Q, Z, S = 0.0, 0.0, 0.0  # centred on the initial centroid, equilibrium start
    out = [S]
    for _ in range(nsteps):
        cross = (1 - 1 / tau) * Q + u * Z / tau
        S, Q, Z = S + 2 * cross + P, cross + P, Z + M0 * u
        out.append(S)
    return np.array(out)


@pytest.mark.parametrize("collision,tau", [(0, 1.0), (0, 0.7), (1, 0.7), (0, 0.55)])
def test_ade_variance_growth(oracle_mod, collision, tau):
    """u = 0, no fields: the variance of a density bump follows the exact
    moment recursion and grows at 2D per step with D = (tau - 1/2)/3 (Eq. 12)."""
    nz = 160  # the bump's tails stay > 40 nodes from the wrap for 40 steps
    o = make(oracle_mod, 3, 3, nz, collision=collision, boundary=oracle_mod.BND_PERIODIC,
             couple=0, tau=tau)
    z = np.arange(nz) - nz / 2
    sig = 4.0
    n = 1.0 + 0.1 * np.exp(-z ** 2 / (2 * sig ** 2))
    A = np.zeros((4, nz, 3, 3))
    A[0] = n[:, None, None]
    o.set_equilibrium(A)
    steps = 40
    dn0 = (n - 1.0) * 9
    M0 = dn0.sum()
    S0 = (z ** 2 * dn0).sum()
    var = []
    for k in range(steps + 1):
        if k:
            o.step(1)
        dn = (o.moments()["n"] - 1.0).sum(axis=(1, 2))
        assert abs(dn.sum() - M0) < 1e-11
        var.append((z ** 2 * dn).sum())
    var = np.array(var)
    S_exact = S0 + _moment_recursion(tau, M0, 0.0, steps)
    assert np.allclose(var, S_exact, rtol=1e-10), (var[:5], S_exact[:5])
    D = (tau - 0.5) / 3.0
    growth = (var[-1] - var[-11]) / 10 / M0
    transient = abs(1 - 1 / tau) ** 30
    assert abs(growth - 2 * D) < (1e-3 + 2 * transient) * 2 * D + 1e-9


def test_ade_translation_at_beta(oracle_mod):
    """Uniform momentum p, no fields: the bump's centroid moves exactly
    u = beta(p) dt/dx lattice units per step, p stays uniform."""
    nz = 96
    o = make(oracle_mod, 3, 3, nz, boundary=oracle_mod.BND_PERIODIC, couple=0, tau=0.6)
    z = np.arange(nz) - 30.0
    n = 1.0 + 0.1 * np.exp(-z ** 2 / (2 * 4.0 ** 2))
    p0 = 0.8
    A = np.zeros((4, nz, 3, 3))
    A[0] = n[:, None, None]
    A[3] = p0 * A[0]
    o.set_equilibrium(A)
    u = p0 / math.sqrt(1 + p0 * p0) * o.params["dt"] / o.params["dx"]
    dn0 = (n - 1) * 9
    c0 = (z * dn0).sum() / dn0.sum()
    steps = 80
    o.step(steps)
    m = o.moments()
    dn = (m["n"] - 1).sum(axis=(1, 2))
    c1 = (z * dn).sum() / dn.sum()
    assert abs((c1 - c0) - steps * u) < 1e-9
    assert np.allclose(m["A"][2] / m["n"], p0, rtol=1e-12)


def test_density_floor_sets_the_advecting_velocity(oracle_mod):
    """Plasma thinner than n_floor (the reading p = A / max(n, n_floor)):
    n = 1e-8 uniform with n p_z = 0.8e-6 uniform, so p = 0.8 through the
    floor (the unfloored momentum would be 80). A small bump carried by the
    n p_x lattice (p_x <= 1e-4) then translates at u = beta(0.8) dt/dx lattice
    units per step to O(p_x^2): a floor that is not applied gives
    beta(80) = 0.99992 instead of 0.62."""
    nz = 96
    nfl = 1e-6
    o = make(oracle_mod, 3, 3, nz, boundary=oracle_mod.BND_PERIODIC, couple=0, tau=0.6, n_floor=nfl)
    z = np.arange(nz) - 30.0
    bump = 1e-10 * np.exp(-z ** 2 / (2 * 4.0 ** 2))
    A = np.zeros((4, nz, 3, 3))
    A[0] = 1e-8
    A[1] = bump[:, None, None]
    A[3] = 0.8 * nfl
    o.set_equilibrium(A)
    u = 0.8 / math.sqrt(1 + 0.8 * 0.8) * o.params["dt"] / o.params["dx"]
    c0 = (z * bump).sum() / bump.sum()
    steps = 80
    o.step(steps)
    m = o.moments()
    a1 = m["A"][0].sum(axis=(1, 2))  # the n p_x lattice
    c1 = (z * a1).sum() / a1.sum()
    assert abs((c1 - c0) - steps * u) < 1e-6, (c1 - c0, steps * u)
    assert abs(a1.sum() - 9 * bump.sum()) <= 1e-12 * 9 * bump.sum()


# ------------------------------------------------------------ Eq. 5 (Yee)
@pytest.mark.parametrize("ecomp,axis", [(0, 2), (0, 1), (1, 0), (1, 2), (2, 0), (2, 1)])
def test_yee_vacuum_standing_wave(oracle_mod, ecomp, axis):
    """Vacuum, one Fourier mode of E_a along axis b: E(m) = cos((m+1/2) th)/cos(th/2)
    with sin(th/2) = (dt/dx) sin(k dx/2), the Yee dispersion relation."""
    n = 16
    dims = [4, 4, 4]  # x, y, z
    dims[axis] = n
    o = make(oracle_mod, dims[0], dims[1], dims[2], boundary=oracle_mod.BND_PERIODIC,
             n0=0.0, tau=0.8)
    dx, dt = o.params["dx"], o.params["dt"]
    k = 2 * math.pi * 2 / (n * dx)
    coord = np.arange(n) * dx  # E_a sits at integer positions along b != a
    E = np.zeros((3,) + o.shape)
    prof = np.sin(k * coord)
    shape = [1, 1, 1]
    shape[2 - axis] = n
    E[ecomp] = prof.reshape(shape) * np.ones(o.shape)
    o.set_fields(E, np.zeros_like(E))
    th = 2 * math.asin(dt / dx * math.sin(k * dx / 2))
    for m in range(1, 41):
        o.step(1)
        got, _ = o.get_fields()
        want = E[ecomp] * math.cos((m + 0.5) * th) / math.cos(th / 2)
        assert np.allclose(got[ecomp], want, atol=1e-12), m
        other = [c for c in range(3) if c != ecomp]
        assert np.abs(got[other]).max() < 1e-13


def _div_edges(E, periodic=True):
    r = lambda a, s: np.roll(a, shift=s, axis=(0, 1, 2))
    return (E[0] - r(E[0], (0, 0, 1))) + (E[1] - r(E[1], (0, 1, 0))) + (E[2] - r(E[2], (1, 0, 0)))


def _div_faces(B):
    r = lambda a, s: np.roll(a, shift=s, axis=(0, 1, 2))
    return (r(B[0], (0, 0, -1)) - B[0]) + (r(B[1], (0, -1, 0)) - B[1]) + (r(B[2], (-1, 0, 0)) - B[2])


def test_yee_gauss_identities(oracle_mod):
    """div B is unchanged and div E changes by -dt div J_edge each step, exactly."""
    o = make(oracle_mod, 6, 5, 7, boundary=oracle_mod.BND_PERIODIC, tau=0.7)
    _random_state(oracle_mod, o, 21)
    E0, B0 = o.get_fields()
    dB0 = _div_faces(B0)
    dt = o.params["dt"]
    r = lambda a, s: np.roll(a, shift=s, axis=(0, 1, 2))
    for _ in range(5):
        E_prev, _ = o.get_fields()
        o.step(1)
        E1, B1 = o.get_fields()
        J = o.last_step()["J"]
        Jedge = np.stack([0.5 * (J[0] + r(J[0], (0, 0, -1))),
                          0.5 * (J[1] + r(J[1], (0, -1, 0))),
                          0.5 * (J[2] + r(J[2], (-1, 0, 0)))])
        assert np.allclose(_div_faces(B1), dB0, atol=1e-13)
        assert np.allclose(_div_edges(E1) - _div_edges(E_prev), -dt * _div_edges(Jedge), atol=1e-13)


def test_driver_charge_gauss_law(oracle_mod):
    """Vacuum, driver entering through the z = 0 wall: div E matches the
    driver's charge density -n_b at t_{n+1/2} (J_b = -n_b z, speed c)."""
    nx = ny = 16
    nz = 48
    dx = 0.2
    o = make(oracle_mod, nx, ny, nz, dx=dx, n0=0.0, alpha=1.0, sigma_r=0.8, sigma_z=0.8,
             z0=-3.2, tau=0.8)
    steps = 200
    o.step(steps)
    E, _ = o.get_fields()
    divE = np.zeros(o.shape)
    divE[1:-1, 1:-1, 1:-1] = ((E[0][1:-1, 1:-1, 1:-1] - E[0][1:-1, 1:-1, :-2])
                              + (E[1][1:-1, 1:-1, 1:-1] - E[1][1:-1, :-2, 1:-1])
                              + (E[2][1:-1, 1:-1, 1:-1] - E[2][:-2, 1:-1, 1:-1])) / dx
    t = (steps + 0.5) * o.params["dt"]
    z = np.arange(nz) * dx
    y = np.arange(ny) * dx - (ny - 1) * dx / 2
    x = np.arange(nx) * dx - (nx - 1) * dx / 2
    rho = -np.exp(-(x[None, None, :] ** 2 + y[None, :, None] ** 2) / (2 * 0.8 ** 2)
                  - (z[:, None, None] - (-3.2 + t)) ** 2 / (2 * 0.8 ** 2))
    inner = (slice(2, -2), slice(2, -2), slice(2, -2))
    err = np.abs(divE[inner] - rho[inner]).max() / np.abs(rho).max()
    assert err < 0.02, err


# ------------------------------------------------- Eqs. 2 + 5, uniform plasma
def test_cold_plasma_oscillation_closed_form(oracle_mod):
    """Uniform plasma, small p_z: E_z(n) = delta dt sin(n th)/sin(th) with
    th = 2 asin(dt/2), i.e. omega_p = 1 up to the leapfrog phase error."""
    o = make(oracle_mod, 4, 4, 4, boundary=oracle_mod.BND_PERIODIC, tau=0.9)
    delta = 1e-6
    A = np.zeros((4,) + o.shape)
    A[0] = 1.0
    A[3] = delta
    o.set_equilibrium(A)
    dt = o.params["dt"]
    th = 2 * math.asin(dt / 2)
    for m in range(1, 301):
        o.step(1)
        if m % 25 == 0:
            E, _ = o.get_fields()
            want = delta * dt * math.sin(m * th) / math.sin(th)
            assert np.allclose(E[2], want, rtol=1e-6, atol=1e-12 * delta), m
            assert np.abs(E[:2]).max() < 1e-20


def _uniform_map(p, E, B, dt, steps):
    """Scalar reduction of the coupled step for a uniform plasma (n = 1):
    p* = p - dt (E + beta(p) x B), E' = E + dt beta(p*), B static."""
    out = []
    for _ in range(steps):
        b = p / math.sqrt(1 + p @ p)
        p = p - dt * (E + np.cross(b, B))
        E = E + dt * p / math.sqrt(1 + p @ p)
        out.append((p.copy(), E.copy()))
    return out


@pytest.mark.parametrize("p0", [0.5, 2.0])
def test_relativistic_oscillation(oracle_mod, p0):
    """Large-amplitude uniform oscillation: the 3D scheme equals the scalar
    map; its period matches the Hamiltonian H = sqrt(1+p^2) + E^2/2 of Eq. 2
    + Eq. 5 (continuum) to O(dt^2)."""
    from scipy.integrate import quad
    o = make(oracle_mod, 3, 3, 3, boundary=oracle_mod.BND_PERIODIC, tau=0.9, dx=0.05)
    dt = o.params["dt"]
    A = np.zeros((4,) + o.shape)
    A[0] = 1.0
    A[3] = p0
    o.set_equilibrium(A)
    ref = _uniform_map(np.array([0, 0, p0], float), np.zeros(3), np.zeros(3), dt, 2000)
    Ez = []
    for m in range(2000):
        o.step(1)
        E, _ = o.get_fields()
        Ez.append(E[2].mean())
        if m % 200 == 0:
            mm = o.moments()
            assert abs(mm["A"][2].mean() - ref[m][0][2]) < 1e-11 * (1 + p0)
            assert abs(E[2].mean() - ref[m][1][2]) < 1e-11 * (1 + p0)
    Ez = np.array(Ez)
    # continuum period: T = 4 int_0^pmax dp / sqrt(2 (gmax - sqrt(1 + p^2)))
    gmax = math.sqrt(1 + p0 * p0)
    T, _ = quad(lambda p: 1.0 / math.sqrt(2 * (gmax - math.sqrt(1 + p * p))), 0, p0, limit=200)
    T *= 4
    # measured period from upward zero crossings of E_z (E is at t_{m+1/2})
    t = (np.arange(len(Ez)) + 1.5) * dt
    s = np.sign(Ez)
    idx = np.where((s[:-1] < 0) & (s[1:] > 0))[0]
    tc = t[idx] - Ez[idx] * dt / (Ez[idx + 1] - Ez[idx])
    Tm = np.diff(tc).mean()
    assert abs(Tm - T) / T < 2e-3, (Tm, T)


def test_magnetised_uniform_plasma(oracle_mod):
    """Uniform B_z: the scheme equals the scalar map with the Lorentz force
    -(E + beta x B), and the oscillation splits into the two cutoff
    frequencies omega = (sqrt(B^2 + 4) +- B)/2 of a magnetised cold plasma."""
    o = make(oracle_mod, 3, 3, 3, boundary=oracle_mod.BND_PERIODIC, tau=0.9, dx=0.05)
    dt = o.params["dt"]
    B0 = 0.6
    delta = 1e-5
    A = np.zeros((4,) + o.shape)
    A[0] = 1.0
    A[1] = delta
    o.set_equilibrium(A)
    Bf = np.zeros((3,) + o.shape)
    Bf[2] = B0
    o.set_fields(np.zeros_like(Bf), Bf)
    steps = 1200
    ref = _uniform_map(np.array([delta, 0, 0]), np.zeros(3), np.array([0, 0, B0]), dt, steps)
    px, py = [], []
    for m in range(steps):
        o.step(1)
        mm = o.moments()
        px.append(mm["A"][0].mean())
        py.append(mm["A"][1].mean())
        if m % 100 == 0:
            assert abs(px[-1] - ref[m][0][0]) < 1e-12 * delta * 1e3
            assert abs(py[-1] - ref[m][0][1]) < 1e-12 * delta * 1e3
    # electron gyration sense: beta along +x in B along +z turns towards +y
    assert py[5] > 0
    # continuum linear solution: P = p_x + i p_y, dP/dt = -eps + i B P, deps/dt = P
    wR = (math.sqrt(B0 ** 2 + 4) + B0) / 2
    wL = (math.sqrt(B0 ** 2 + 4) - B0) / 2
    # P(t) = a e^{i wR t} + b e^{-i wL t}, P(0) = delta, P'(0) = i B delta
    # a + b = delta, i wR a - i wL b = i B delta
    a = delta * (B0 + wL) / (wR + wL)
    b = delta - a
    t = (np.arange(steps) + 1) * dt
    P = a * np.exp(1j * wR * t) + b * np.exp(-1j * wL * t)
    got = np.array(px) + 1j * np.array(py)
    err = np.abs(got - P).max() / delta
    assert err < 0.05, err


# --------------------------------------------------------------- boundaries
def test_open_boundary_equilibrium_of_clamped_node(oracle_mod):
    """Eq. 14: after a step, each boundary node holds f^eq of the moments of
    the clamped interior node."""
    nx, ny, nz = 6, 5, 7
    o = make(oracle_mod, nx, ny, nz, boundary=oracle_mod.BND_OPEN, tau=0.7)
    _random_state(oracle_mod, o, 4)
    o.step(2)
    f = o.get_f()
    A = f.sum(axis=1)
    dt, dx = o.params["dt"], o.params["dx"]
    checked = 0
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if 0 < x < nx - 1 and 0 < y < ny - 1 and 0 < z < nz - 1:
                    continue
                c = (min(max(z, 1), nz - 2), min(max(y, 1), ny - 2), min(max(x, 1), nx - 2))
                Ac = A[(slice(None),) + c]
                u = beta_of(Ac[1:] / Ac[0]) * dt / dx
                xu = XI @ u
                for l in range(4):
                    feq = WQ * Ac[l] * (1 + 3 * xu + 4.5 * xu ** 2 - 1.5 * (u @ u))
                    assert np.allclose(f[l, :, z, y, x], feq, rtol=1e-12, atol=1e-16)
                checked += 1
    assert checked == nx * ny * nz - (nx - 2) * (ny - 2) * (nz - 2)


def test_conducting_walls(oracle_mod):
    """Open mode: tangential E and normal B stay zero on the six walls."""
    o = make(oracle_mod, 12, 10, 16, alpha=0.5, sigma_r=0.6, sigma_z=0.6, z0=-1.0, tau=0.6)
    o.step(30)
    E, B = o.get_fields()
    assert np.abs(E).max() > 1e-4
    # x walls (i = 0, nx-1): E_y, E_z tangential, B_x normal
    for i in (0, -1):
        assert np.all(E[1][:, :, i] == 0) and np.all(E[2][:, :, i] == 0) and np.all(B[0][:, :, i] == 0)
        assert np.all(E[0][:, i, :] == 0) and np.all(E[2][:, i, :] == 0) and np.all(B[1][:, i, :] == 0)
        assert np.all(E[0][i, :, :] == 0) and np.all(E[1][i, :, :] == 0) and np.all(B[2][i, :, :] == 0)


def test_uniform_plasma_at_rest_is_steady(oracle_mod):
    o = make(oracle_mod, 7, 6, 9, tau=0.51)
    o.step(20)
    m = o.moments()
    E, B = o.get_fields()
    assert np.allclose(m["n"], 1.0, atol=1e-15)
    assert np.abs(m["beta"]).max() == 0
    assert np.abs(E).max() == 0 and np.abs(B).max() == 0


def test_radial_profile_initial_density(oracle_mod):
    prof = np.array([1.0, 1.5, 2.0, 2.5])
    nx = ny = 9
    dx = 0.25
    rmax = 0.9
    o = make(oracle_mod, nx, ny, 5, dx=dx, profile=prof, profile_rmax=rmax, boundary=oracle_mod.BND_PERIODIC)
    n = o.moments()["n"]
    c = (nx - 1) * dx / 2
    for y in range(ny):
        for x in range(nx):
            r = math.hypot(x * dx - c, y * dx - c)
            want = 1.0 + 1.5 * min(r, rmax) / rmax
            assert abs(n[2, y, x] - want) < 1e-13


def test_wake_mirror_symmetry(oracle_mod):
    w = W.parity_small().replace(nz=32, steps=40)
    o = make(oracle_mod, w.nx, w.ny, w.nz, dx=w.dx, tau=w.tau, alpha=w.alpha,
             sigma_r=w.sigma_r, sigma_z=w.sigma_z, z0=-1.0)
    o.step(40)
    m = o.moments()
    n = m["n"]
    assert np.abs(n - n[:, :, ::-1]).max() < 1e-12
    assert np.abs(n - n[:, ::-1, :]).max() < 1e-12
    assert np.abs(n - n.transpose(0, 2, 1)).max() < 1e-12


# ------------------------------------------------------------- linear wake
def test_linear_wake_wavelength(oracle_mod):
    """n_b/n0 = 0.01: on-axis E_z behind the driver oscillates with the plasma
    wavelength 2 pi c/omega_p (Sec. IV defines k_p = omega_p/c), and its
    amplitude matches linear theory for a bi-Gaussian driver."""
    nx = ny = 24
    nz = 96
    dx = 0.2
    sr = sz = 0.5
    alpha = 0.01
    o = make(oracle_mod, nx, ny, nz, dx=dx, tau=0.505, alpha=alpha, sigma_r=sr, sigma_z=sz, z0=-2.0)
    dt = o.params["dt"]
    steps = 460
    o.step(steps)
    E, _ = o.get_fields()
    # on-axis value: the axis sits between the four central nodes
    ez = E[2][:, ny // 2 - 1:ny // 2 + 1, nx // 2 - 1:nx // 2 + 1].mean(axis=(1, 2))
    zb = -2.0 + (steps + 0.5) * dt
    z = (np.arange(nz) + 0.5) * dx
    sel = (z < zb - 1.5) & (z > zb - 13.0)
    zz, ee = z[sel], ez[sel]
    s = np.sign(ee)
    i = np.where(s[:-1] != s[1:])[0]
    zc = zz[i] - ee[i] * (zz[i + 1] - zz[i]) / (ee[i + 1] - ee[i])
    half = np.diff(zc)
    assert len(half) >= 2
    lam = 2 * half.mean()
    assert abs(lam - 2 * math.pi) / (2 * math.pi) < 0.02, (lam, zc)
    # linear theory, on axis: E_z = alpha sqrt(2 pi) k sz exp(-sz^2/2) R cos(..),
    # R = (sr^2/2) exp(sr^2/2) E1(sr^2/2)
    from scipy.special import exp1
    a = sr * sr / 2
    R = a * math.exp(a) * exp1(a)
    amp = alpha * math.sqrt(2 * math.pi) * sz * math.exp(-sz * sz / 2) * R
    near = (z < zb - 0.5) & (z > zb - 2 * math.pi - 0.5)
    got = np.abs(ez[near]).max()
    assert abs(got - amp) / amp < 0.2, (got, amp)


# ------------------------------------------------------------ Eq. 15 (golden)
def test_qtilde_paper_values(oracle_mod):
    """Sec. IV: 0.024/0.120/0.240 nC, sigma_x = sigma_y = 8.9 um, sigma_z = 17.7 um,
    n0 = 1e16 cm^-3 give Q = 0.1/0.5/1 (Eq. 15 with k_p^3)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "qtilde_paper.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for charge_nc, sx_um, sy_um, sz_um, n0_cm3, q_paper in rows:
        q, alpha = oracle_mod.qtilde(float(charge_nc) * 1e-9, float(sx_um) * 1e-6,
                                     float(sy_um) * 1e-6, float(sz_um) * 1e-6, float(n0_cm3) * 1e6)
        assert abs(q - float(q_paper)) / float(q_paper) < 0.02, (q, q_paper)
    q, alpha = oracle_mod.qtilde(0.024e-9, 8.9e-6, 8.9e-6, 17.7e-6, 1e22)
    assert abs(alpha - 0.68) < 0.01


# ------------------------------------------------- forward-mode derivatives
def test_tangent_mode_matches_central_differences(oracle_mod):
    """Dual-number derivatives of E after the coupled step (driver, profile)
    equal central finite differences of the FP64 primal at h = 1e-3 and 1e-5."""
    nx, ny, nz, dx = 10, 10, 16, 0.2
    dt = W.DT_OVER_DX * dx
    prof = np.ones(8)
    kw = dict(nx=nx, ny=ny, nz=nz, dx=dx, dt=dt, tau=0.6, profile=prof, profile_rmax=0.9,
              alpha=0.5, sigma_r=0.5, sigma_z=0.5, z0=-0.5)
    steps = 40
    rng = np.random.default_rng(3)
    dirs = np.zeros((4, 3 + len(prof)))
    dirs[0, 0] = 1.0           # d/d alpha
    dirs[1, 1] = 1.0           # d/d sigma_r
    dirs[2, 2] = 1.0           # d/d sigma_z
    dirs[3, 3:] = rng.standard_normal(len(prof))  # a profile direction
    E, dE = oracle_mod.tangent_run(steps, dirs, **kw)
    o = oracle_mod.Oracle(**kw)
    o.step(steps)
    E0, _ = o.get_fields()
    assert np.array_equal(E, E0)  # same primal on dual numbers

    def primal(theta):
        a, sr, sz = theta[:3]
        k = dict(kw, alpha=a, sigma_r=sr, sigma_z=sz, profile=np.array(theta[3:]))
        oo = oracle_mod.Oracle(**k)
        oo.step(steps)
        return oo.get_fields()[0]

    theta0 = np.array([0.5, 0.5, 0.5] + list(prof))
    for k in range(4):
        for h in (1e-3, 1e-5):
            fd = (primal(theta0 + h * dirs[k]) - primal(theta0 - h * dirs[k])) / (2 * h)
            err = np.linalg.norm(fd - dE[k]) / np.linalg.norm(dE[k])
            # central differences: truncation O(h^2) at 1e-3, round-off O(eps/h) at 1e-5
            assert err < (1e-5 if h == 1e-3 else 1e-7), (k, h, err)
