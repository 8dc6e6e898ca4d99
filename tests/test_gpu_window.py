"""GPU moving window against the FP64 oracle and against the exact index
arithmetic of a one-plane move (pure streaming, integer populations)."""
import math

import numpy as np
import pytest

import oracle
from paper_2201_05473_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2201_05473_gb300 import lbm  # noqa: E402

XI = np.array([[0, 0, 0],
               [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
               [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0],
               [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1],
               [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]])
WQ = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def window_case(collision=W.BGK):
    # the parity workload's physics (n_b/n0 = 0.1) in a 20x20x48 box; the
    # driver enters from z0 = -2 and is held at z = 1 once it gets there
    return W.parity_small().replace(nx=20, ny=20, nz=48, collision=collision,
                                    moving_window=1, window_z=1.0)


@pytest.mark.parametrize("collision", [W.BGK, W.REGULARIZED])
def test_window_parity_with_oracle(collision):
    """200 steps, the box moves 20 planes: n, beta, E_z within rel-L2 1e-5."""
    w = window_case(collision)
    steps = 200
    o = oracle.Oracle(w.nx, w.ny, w.nz, w.dx, w.dt, w.tau, collision=w.collision, alpha=w.alpha,
                      sigma_r=w.sigma_r, sigma_z=w.sigma_z, z0=w.z0, moving_window=1, window_z=w.window_z)
    o.step(steps)
    with lbm.Simulation(w) as sim:
        sim.step(steps)
        assert sim.window_planes() == o.window_planes == 20
        m = lbm.FIELD_N | lbm.FIELD_UX | lbm.FIELD_UY | lbm.FIELD_UZ | lbm.FIELD_EZ | lbm.RAW_YEE
        g = sim.fields(m).cpu().numpy().astype(np.float64)
    om = o.moments()
    E, _ = o.get_fields()
    errs = {"n": rel(g[0], om["n"]), "beta": rel(g[1:4], om["beta"]), "Ez": rel(g[4], E[2])}
    print(errs)
    assert max(errs.values()) <= 1e-5, errs


def test_window_with_16bit_storage():
    """The moving window with populations stored as FP16 / BF16 deviations:
    the plane of fresh plasma that enters at the top of the box must decode
    to the plasma at rest (deviation zero). 200 steps, 20 moves, against the
    oracle: FP16 within the reduced-precision bar 1e-3 on n, beta and E_z;
    BF16 recorded and guarded at about three times its GB300 level (BF16
    misses the bar; see the precision tests). GB300: FP16 n 3.3e-6, beta
    1.5e-4, E_z 2.4e-5; BF16 n 1.4e-5, beta 1.2e-3, E_z 2.3e-4."""
    steps = 200
    base = window_case(W.BGK)
    o = oracle.Oracle(base.nx, base.ny, base.nz, base.dx, base.dt, base.tau, collision=base.collision,
                      alpha=base.alpha, sigma_r=base.sigma_r, sigma_z=base.sigma_z, z0=base.z0, moving_window=1,
                      window_z=base.window_z)
    o.step(steps)
    om = o.moments()
    E, _ = o.get_fields()
    m = lbm.FIELD_N | lbm.FIELD_UX | lbm.FIELD_UY | lbm.FIELD_UZ | lbm.FIELD_EZ | lbm.RAW_YEE
    errs = {}
    for st in (W.F16, W.BF16):
        with lbm.Simulation(base.replace(storage=st)) as sim:
            sim.step(steps)
            assert sim.window_planes() == 20
            g = sim.fields(m).cpu().numpy().astype(np.float64)
        errs[st] = {"n": rel(g[0], om["n"]), "beta": rel(g[1:4], om["beta"]), "Ez": rel(g[4], E[2])}
    print("window, 16-bit storage vs oracle:", errs)
    assert max(errs[W.F16].values()) <= 1e-3, errs
    assert max(errs[W.BF16].values()) <= 4e-3, errs


def test_window_move_is_exact_on_integer_populations():
    """Stream-only lattices, no fields, a window move on the first step: the
    state after it is F_i(x + z_hat - xi_i) for the state F set before it,
    bit for bit, and the fresh plasma w_i n0 (lattice 0), 0 (momentum
    lattices) where the pull reaches the plane above the box."""
    nz, ny, nx = 9, 6, 7
    dx = 0.2
    dt = W.DT_OVER_DX * dx
    z0 = 0.0
    wz = z0 - dx + 0.5 * dt  # first step moves the box
    w = W.parity_small().replace(nx=nx, ny=ny, nz=nz, collision=W.STREAM_ONLY, couple=0, alpha=0.0,
                                 z0=z0, moving_window=1, window_z=wz)
    F = W.integer_populations((nz, ny, nx))
    with lbm.Simulation(w) as sim:
        sim.set_state(F)
        sim.step(1)
        assert sim.window_planes() == 1
        G = sim.get_state()[0].cpu().numpy().astype(np.float64)
    inner = lambda x, y, z: 1 <= x <= nx - 2 and 1 <= y <= ny - 2 and 1 <= z <= nz - 2
    moved = fresh = 0
    for z in range(1, nz - 1):
        for y in range(1, ny - 1):
            for x in range(1, nx - 1):
                for q in range(19):
                    if not inner(x - XI[q, 0], y - XI[q, 1], z - XI[q, 2]):
                        continue
                    sx, sy, sz = x - XI[q, 0], y - XI[q, 1], z + 1 - XI[q, 2]
                    for l in range(4):
                        if z + 1 - 2 * XI[q, 2] == nz:
                            want = WQ[q] * w.n0 if l == 0 else 0.0
                            fresh += 1
                        elif inner(sx, sy, sz):
                            want = F[l, q, sz, sy, sx]
                            moved += 1
                        else:
                            continue
                        assert G[l, q, z, y, x] == np.float32(want), (l, q, z, y, x)
    assert moved > 1000 and fresh > 50


def test_window_uniform_plasma_and_restrictions():
    """A uniform plasma without driver stays uniform through window moves;
    the adjoint recording refuses a moving window; several moving-window
    instances step one by one (no batched table)."""
    w = W.parity_small().replace(nx=12, ny=12, nz=24, alpha=0.0, moving_window=1, window_z=-2.0)
    with lbm.Simulation([w, w.replace(nz=20)]) as sim:
        sim.step(30)
        assert sim.window_planes(0) == math.floor((w.z0 + 30 * w.dt - w.window_z) / w.dx) == 5
        for i in range(2):
            n = sim.fields(lbm.FIELD_N, i).cpu().numpy()
            assert np.abs(n - 1.0).max() < 1e-5
        with pytest.raises(lbm.LBMError):
            sim.record(4, 2)
