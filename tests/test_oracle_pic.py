"""Pins of the oracle's PIC driver (Eq. 1: macro-electrons pushed in E + beta x B,
their current deposited on the Yee grid).

Against: the Boris rotation's exact closed form in a uniform B (|p| kept,
angle 2 atan(B dt / 2 gamma) per step, electron sense), exact acceleration in
a uniform E, the discrete continuity equation of the deposited current
against charge densities built here from the particle positions, and the
rigid-bunch limit of an ultra-relativistic bunch (sampling noise falling as
the particle count grows).
"""
import math

import numpy as np

from paper_2201_05473_gb300 import workloads as W


def make(oracle_mod, nx, ny, nz, **kw):
    kw.setdefault("dx", 0.2)
    kw.setdefault("dt", W.DT_OVER_DX * kw["dx"])
    kw.setdefault("tau", 0.8)
    return oracle_mod.Oracle(nx, ny, nz, driver=1, **kw)


def test_boris_rotation_in_uniform_B(oracle_mod):
    o = make(oracle_mod, 4, 4, 4, boundary=oracle_mod.BND_PERIODIC, n0=0.0)
    B0 = 0.7
    E = np.zeros((3, 4, 4, 4))
    B = np.zeros((3, 4, 4, 4))
    B[2] = B0
    o.set_fields(E, B)
    p0 = 0.5
    xp = np.zeros((6, 1))
    xp[:3, 0] = 0.33
    xp[3, 0] = p0
    o.set_particles(xp, 0.0)
    dt = o.params["dt"]
    th = 2 * math.atan(B0 * dt / (2 * math.sqrt(1 + p0 * p0)))
    for m in range(1, 41):
        o.step(1)
        px, py, pz = o.get_particles()[3:, 0]
        assert abs(math.hypot(px, py) - p0) < 1e-14 and pz == 0.0
        assert abs(px - p0 * math.cos(m * th)) < 1e-13 and abs(py - p0 * math.sin(m * th)) < 1e-13, m


def test_uniform_E_acceleration(oracle_mod):
    o = make(oracle_mod, 4, 4, 4, boundary=oracle_mod.BND_PERIODIC, n0=0.0)
    E0 = 0.3
    E = np.zeros((3, 4, 4, 4))
    E[2] = E0
    o.set_fields(E, np.zeros((3, 4, 4, 4)))
    xp = np.zeros((6, 1))
    xp[:3, 0] = 0.41
    xp[5, 0] = 2.0
    o.set_particles(xp, 0.0)
    dt = o.params["dt"]
    z = xp[2, 0]
    for m in range(1, 31):
        o.step(1)
        q = o.get_particles()[:, 0]
        pz = 2.0 - E0 * dt * m  # dp/dt = -E for an electron
        assert abs(q[5] - pz) < 1e-13
        z = (z + dt * pz / math.sqrt(1 + pz * pz)) % 0.8
        assert abs(q[2] - z) < 1e-12


def _cic_charge(xp, weight, shape, dx):
    """rho at the nodes from the particle positions, linear shape, charge -w."""
    nz, ny, nx = shape
    rho = np.zeros(shape)
    for x, y, z in xp[:3].T:
        g = np.array([x, y, z]) / dx
        i0 = np.floor(g).astype(int)
        f = g - i0
        for c in range(2):
            for b in range(2):
                for a in range(2):
                    w = (f[0] if a else 1 - f[0]) * (f[1] if b else 1 - f[1]) * (f[2] if c else 1 - f[2])
                    rho[i0[2] + c, i0[1] + b, i0[0] + a] -= weight * w / dx ** 3
    return rho


def test_deposit_obeys_discrete_continuity(oracle_mod):
    """For particles inside the box, (rho(t_{n+3/2}) - rho(t_{n+1/2}))/dt +
    div J_b = 0 at every node, to round-off, with rho built here from the
    positions (linear shape) and J_b the deposited current on the E edges."""
    nx, ny, nz, dx = 10, 9, 12, 0.2
    o = make(oracle_mod, nx, ny, nz, dx=dx, tau=0.7)
    rng = np.random.default_rng(4)
    n = 40
    xp = np.zeros((6, n))
    xp[0] = rng.uniform(3, 6, n) * dx
    xp[1] = rng.uniform(3, 5, n) * dx
    xp[2] = rng.uniform(3, 8, n) * dx
    xp[3:] = rng.normal(0, 2.0, (3, n))
    weight = 0.01
    o.set_particles(xp, weight)
    dt = o.params["dt"]
    for _ in range(3):
        x0 = o.get_particles()
        o.step(1)
        x1 = o.get_particles()
        J = o.driver_current()
        rho0 = _cic_charge(x0, weight, o.shape, dx)
        rho1 = _cic_charge(x1, weight, o.shape, dx)
        div = np.zeros(o.shape)
        div[:, :, 1:] += (J[0][:, :, 1:] - J[0][:, :, :-1]) / dx
        div[:, :, 0] += J[0][:, :, 0] / dx
        div[:, 1:, :] += (J[1][:, 1:, :] - J[1][:, :-1, :]) / dx
        div[:, 0, :] += J[1][:, 0, :] / dx
        div[1:] += (J[2][1:] - J[2][:-1]) / dx
        div[0] += J[2][0] / dx
        res = (rho1 - rho0) / dt + div
        assert np.abs(res).max() < 1e-11 * np.abs(div).max(), np.abs(res).max()
        assert np.abs(div).max() > 0


def _pic_vs_rigid(oracle_mod, n_particles, steps=120):
    w = W.parity_small().replace(nx=16, ny=16, nz=40, z0=1.5)
    kw = dict(dx=w.dx, dt=w.dt, tau=w.tau, alpha=w.alpha, sigma_r=w.sigma_r, sigma_z=w.sigma_z, z0=w.z0)
    rigid = oracle_mod.Oracle(w.nx, w.ny, w.nz, **kw)
    pic = oracle_mod.Oracle(w.nx, w.ny, w.nz, driver=1, **kw)
    xp, weight = W.bunch_particles(n_particles, w.alpha, w.sigma_r, w.sigma_z, w.z0, w.dt, w.nx, w.ny, w.dx)
    pic.set_particles(xp, weight)
    rigid.step(steps)
    pic.step(steps)
    Er, _ = rigid.get_fields()
    Ep, _ = pic.get_fields()
    return float(np.linalg.norm(Ep[2] - Er[2]) / np.linalg.norm(Er[2]))


def test_ultrarelativistic_bunch_approaches_the_rigid_driver(oracle_mod):
    """gamma = 5000, no energy spread: the PIC bunch's wake E_z approaches the
    rigid bi-Gaussian's as the sampling noise falls (4x the particles: about
    half the difference; linear shape vs point values of the rigid current
    leave a small floor)."""
    e1 = _pic_vs_rigid(oracle_mod, 4000)
    e2 = _pic_vs_rigid(oracle_mod, 16000)
    print(e1, e2)
    assert e2 < 0.15 and e2 < 0.75 * e1, (e1, e2)
