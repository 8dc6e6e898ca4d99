"""GPU PIC driver (Eq. 1) against the FP64 oracle on the same macro-electrons,
and the Boris rotation's closed form."""
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


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def test_pic_parity_with_oracle():
    """4000 macro-electrons (gamma = 5000, the parity workload's bunch) in a
    16x16x40 box, 120 steps: fields, moments and particles against the oracle.
    Tolerance from the FP32 positions: each step's advance z += dt beta rounds
    to half an ulp of z (z <= 8: 4.8e-7), a random walk of ~5e-6 after 120
    steps, i.e. 2.6e-5 of a cell in the deposited current's shape weights:
    fields and moments within rel-L2 5e-5, particles within 1e-5."""
    w = W.parity_small().replace(nx=16, ny=16, nz=40, z0=1.5, driver=1)
    xp, weight = W.bunch_particles(4000, w.alpha, w.sigma_r, w.sigma_z, w.z0, w.dt, w.nx, w.ny, w.dx)
    o = oracle.Oracle(w.nx, w.ny, w.nz, w.dx, w.dt, w.tau, alpha=w.alpha, sigma_r=w.sigma_r,
                      sigma_z=w.sigma_z, z0=w.z0, driver=1)
    o.set_particles(xp, weight)
    o.step(120)
    with lbm.Simulation(w) as sim:
        sim.set_particles(xp, weight)
        sim.step(120)
        g = sim.fields(lbm.FIELD_N | lbm.FIELD_UZ | lbm.FIELD_EZ | lbm.FIELD_EX | lbm.RAW_YEE).cpu().numpy()
        pg = sim.get_particles().cpu().numpy().astype(np.float64)
    E, _ = o.get_fields()
    m = o.moments()
    po = o.get_particles()
    # (components come in mask-bit order: n, beta_z, E_x, E_z)
    errs = {"n": rel(g[0], m["n"]), "beta_z": rel(g[1], m["beta"][2]), "Ex": rel(g[2], E[0]), "Ez": rel(g[3], E[2]),
            "x": rel(pg[:3], po[:3]), "p_perp": rel(pg[3:5], po[3:5]), "pz": rel(pg[5], po[5])}
    print(errs)
    assert max(errs[k] for k in ("n", "beta_z", "Ex", "Ez")) <= 5e-5, errs
    assert max(errs[k] for k in ("x", "p_perp", "pz")) <= 1e-5, errs


def test_pic_boris_rotation():
    w = W.parity_small().replace(nx=4, ny=4, nz=4, boundary=W.PERIODIC, n0=0.0, alpha=0.0, driver=1)
    B0, p0 = 0.7, 0.5
    xp = np.zeros((6, 1), dtype=np.float32)
    xp[:3, 0] = 0.33
    xp[3, 0] = p0
    with lbm.Simulation(w) as sim:
        B = np.zeros((3, 4, 4, 4), dtype=np.float32)
        B[2] = B0
        sim.set_state(E=np.zeros((3, 4, 4, 4), dtype=np.float32), B=B)
        sim.set_particles(xp, 0.0)
        th = 2 * math.atan(B0 * w.dt / (2 * math.sqrt(1 + p0 * p0)))
        for m in range(1, 21):
            sim.step(1)
            q = sim.get_particles().cpu().numpy()[:, 0]
            assert abs(math.hypot(q[3], q[4]) - p0) < 1e-6
            assert abs(q[3] - p0 * math.cos(m * th)) < 2e-6 and abs(q[4] - p0 * math.sin(m * th)) < 2e-6, m


def test_pic_restrictions():
    w = W.parity_small().replace(nx=8, ny=8, nz=12)
    with lbm.Simulation(w) as sim:
        with pytest.raises(lbm.LBMError):
            sim.set_particles(np.zeros((6, 2), dtype=np.float32), 1.0)
    with lbm.Simulation(w.replace(driver=1)) as sim:
        with pytest.raises(lbm.LBMError):
            sim.record(4, 2)
