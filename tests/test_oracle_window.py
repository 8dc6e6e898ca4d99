"""Pins of the oracle's moving window (Sec. II: the box follows the driver).

The window moves the box one plane along +z whenever the driver centre,
once past window_z, has advanced a cell. Pinned against: translation
invariance of a z-uniform plasma, exact index arithmetic of the move on a
pure-streaming integer state (the moved streaming source is pulled twice,
fresh plasma entering at the top), and the linear-wake wavelength
2 pi c/omega_p and amplitude seen in the moving box after the driver has
crossed twice the box length.
"""
import math

import numpy as np

from paper_2201_05473_gb300 import workloads as W

XI = np.array([[0, 0, 0],
               [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
               [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0],
               [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1],
               [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]])
WQ = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def planes(n, z0, dt, dx, wz):
    return max(0, math.floor((z0 + n * dt - wz) / dx))


def test_window_schedule_and_uniform_invariance(oracle_mod):
    """A uniform plasma at rest (no driver) is a steady state, and it is
    unchanged by any number of window moves; the window advances one plane per
    cell the driver centre moves past window_z."""
    nx, ny, nz, dx = 8, 8, 12, 0.2
    dt = W.DT_OVER_DX * dx
    kw = dict(dx=dx, dt=dt, tau=0.7, alpha=0.0, n0=1.3, z0=-1.0)
    ref = oracle_mod.Oracle(nx, ny, nz, **kw)
    o = oracle_mod.Oracle(nx, ny, nz, moving_window=1, window_z=-1.0, **kw)
    f0 = o.get_f()
    moved = []
    for n in range(1, 41):
        o.step(1)
        moved.append(o.window_planes)
        assert o.window_planes == planes(n, -1.0, dt, dx, -1.0)
    assert moved[-1] == 7 and len(set(moved)) == 8  # one plane at a time
    ref.step(40)
    # steady to round-off (the collision rounds f - (f - f^eq)/tau)
    np.testing.assert_allclose(o.get_f(), f0, rtol=1e-14, atol=0)
    np.testing.assert_allclose(o.get_f(), ref.get_f(), rtol=1e-14, atol=0)
    E, B = o.get_fields()
    assert np.abs(E).max() == 0.0 and np.abs(B).max() == 0.0


def test_window_move_is_one_plane_of_the_streaming_source(oracle_mod):
    """Stream-only lattices, no fields: after a step that moves the window,
    f_i(x) = S_i(x + z_hat - 2 xi_i) for the streaming source S set before the
    step (the moved source is pulled once to rebuild the state, then once by
    the step), and the unperturbed plasma's source w_i n0 (lattice 0), 0
    (momentum lattices) wherever x + z_hat - 2 xi_i leaves the top plane.
    Without the move the same nodes hold S_i(x - 2 xi_i)."""
    nx, ny, nz, dx = 7, 6, 9, 0.2
    dt = W.DT_OVER_DX * dx
    N = nx * ny * nz
    # window_z such that the first step moves the box by one plane
    z0 = 0.0
    wz = z0 - dx + 0.5 * dt
    assert planes(0, z0, dt, dx, wz) == 0 and planes(1, z0, dt, dx, wz) == 1
    S = np.empty((4, 19, nz, ny, nx))
    node = np.arange(N, dtype=np.float64).reshape(nz, ny, nx)
    for l in range(4):
        for q in range(19):
            S[l, q] = (l * 19 + q) * N + node + 1.0
    common = dict(dx=dx, dt=dt, tau=0.7, collision=oracle_mod.COLL_NONE, couple=0, alpha=0.0, z0=z0)
    mv = oracle_mod.Oracle(nx, ny, nz, moving_window=1, window_z=wz, **common)
    st = oracle_mod.Oracle(nx, ny, nz, **common)
    for o in (mv, st):
        o.set_source(S)
        o.step(1)
    assert mv.window_planes == 1 and st.window_planes == 0
    fm, fs = mv.get_f(), st.get_f()
    checked = 0
    for z in range(1, nz - 1):
        for y in range(1, ny - 1):
            for x in range(1, nx - 1):
                for q in range(19):
                    sx, sy, sz = x - XI[q, 0], y - XI[q, 1], z - XI[q, 2]
                    if not (1 <= sx <= nx - 2 and 1 <= sy <= ny - 2 and 1 <= sz <= nz - 2):
                        continue  # the first pull lands on an Eq. 14 boundary node
                    tx, ty, tz = x - 2 * XI[q, 0], y - 2 * XI[q, 1], z - 2 * XI[q, 2]
                    for l in range(4):
                        want = S[l, q, tz + 1, ty, tx] if tz + 1 <= nz - 1 else (WQ[q] if l == 0 else 0.0)
                        assert fm[l, q, z, y, x] == want, (l, q, z, y, x)
                        assert fs[l, q, z, y, x] == S[l, q, tz, ty, tx]
                        checked += 1
    assert checked > 4000


def test_linear_wake_in_the_moving_window(oracle_mod):
    """n_b/n0 = 0.01 driver held at z = 16 of a 19.2-long box while it crosses
    one and a half box lengths: behind it the on-axis E_z keeps the
    plasma wavelength 2 pi c/omega_p (within 2 %) and the linear-theory
    amplitude (within 20 %), evaluated at the driver's box position z0 + t -
    W dx."""
    nx = ny = 24
    nz = 96
    dx = 0.2
    sr = sz = 0.5
    alpha = 0.01
    z0, wz = -2.0, 16.0
    dt = W.DT_OVER_DX * dx
    o = oracle_mod.Oracle(nx, ny, nz, dx=dx, dt=dt, tau=0.505, alpha=alpha, sigma_r=sr, sigma_z=sz,
                          z0=z0, moving_window=1, window_z=wz)
    steps = 1400
    o.step(steps)
    Wn = o.window_planes
    assert Wn == planes(steps, z0, dt, dx, wz) and Wn > 1.5 * nz
    E, _ = o.get_fields()
    ez = E[2][:, ny // 2 - 1:ny // 2 + 1, nx // 2 - 1:nx // 2 + 1].mean(axis=(1, 2))
    zb = z0 + (steps + 0.5) * dt - Wn * dx  # driver centre in the box
    assert abs(zb - wz) <= dx
    z = (np.arange(nz) + 0.5) * dx
    sel = (z < zb - 1.5) & (z > 0.8)
    zz, ee = z[sel], ez[sel]
    s = np.sign(ee)
    i = np.where(s[:-1] != s[1:])[0]
    zc = zz[i] - ee[i] * (zz[i + 1] - zz[i]) / (ee[i + 1] - ee[i])
    half = np.diff(zc)
    assert len(half) >= 2
    lam = 2 * half.mean()
    assert abs(lam - 2 * math.pi) / (2 * math.pi) < 0.02, (lam, zc)
    from scipy.special import exp1
    a = sr * sr / 2
    amp = alpha * math.sqrt(2 * math.pi) * sz * math.exp(-sz * sz / 2) * a * math.exp(a) * exp1(a)
    near = (z < zb - 0.5) & (z > zb - 2 * math.pi - 0.5)
    got = np.abs(ez[near]).max()
    assert abs(got - amp) / amp < 0.2, (got, amp)
