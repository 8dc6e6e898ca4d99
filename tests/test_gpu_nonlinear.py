"""The production physics on the GPU: the non-linear regime of Sec. IV.

1. Parity with the FP64 oracle at the production workload's physics
   (n_b/n0 = 1, sigma_r = 0.3, sigma_z = 0.5, dx = 0.05, tau = 0.53,
   regularized collision, open box) on a reduced 160x64x64 box, the driver
   starting inside it at z0 = 4 sigma_z, 400 steps: relative L2 <= 1e-5 on
   n, beta and E_z every 50 steps, while the plasma is driven far from rest
   (min n < 0.5, max |beta| > 0.1).
2. The production workload itself (512x256x256, 2000 steps, the driver
   entering through the z = 0 wall): every moment finite and n > 0 at every
   hundredth step (tau = 0.53 keeps it stable), x/y mirror symmetry of the
   wake, and the FP64 diagnostics equal to direct reductions of the exported
   fields.
"""
import numpy as np
import pytest

import oracle
from paper_2201_05473_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2201_05473_gb300 import lbm  # noqa: E402

TOL = 1e-5


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def test_nonlinear_production_physics_parity():
    w = W.production().replace(nx=64, ny=64, nz=160, z0=2.0)
    oracle.build()
    o = oracle.Oracle(w.nx, w.ny, w.nz, w.dx, w.dt, w.tau, collision=w.collision, alpha=w.alpha,
                      sigma_r=w.sigma_r, sigma_z=w.sigma_z, z0=w.z0, n_floor=w.n_floor)
    m = lbm.FIELD_N | lbm.FIELD_UX | lbm.FIELD_UY | lbm.FIELD_UZ | lbm.FIELD_EZ | lbm.RAW_YEE
    rows = []
    with lbm.Simulation(w) as sim:
        for s in range(50, 401, 50):
            o.step(50)
            sim.step(50)
            g = sim.fields(m).cpu().numpy().astype(np.float64)
            mo = o.moments()
            E, _ = o.get_fields()
            rows.append({"step": s, "n": rel(g[0], mo["n"]), "beta": rel(g[1:4], mo["beta"]),
                         "Ez": rel(g[4], E[2]), "min_n": float(mo["n"].min()),
                         "max_beta": float(np.abs(mo["beta"]).max())})
    o.close()
    for r in rows:
        print(r)
    for r in rows:
        assert r["n"] <= TOL and r["beta"] <= TOL and r["Ez"] <= TOL, r
    # the regime is the non-linear one
    assert rows[-1]["min_n"] < 0.5 and max(r["max_beta"] for r in rows) > 0.1, rows[-1]


def test_production_workload_2000_steps():
    w = W.production()
    with lbm.Simulation(w) as sim:
        for _ in range(20):
            d = sim.step_diag(100)[0]  # raises on a non-finite moment or n < 0
            assert d[7] == 0 and d[5] > 0, d
        assert sim.steps_done() == 2000
        d = sim.diag()
        assert d[7] == 0 and 0 < d[5] < 0.5, d  # the bubble is there and n stays positive
        mask = lbm.FIELD_N | lbm.FIELD_UX | lbm.FIELD_UY | lbm.FIELD_UZ | lbm.FIELD_PX | lbm.FIELD_PY | lbm.FIELD_PZ
        f = sim.fields(mask)
        assert bool(torch.isfinite(f).all())
        n = f[0]
        # mirror symmetry of the wake about the driver axis (between nodes)
        assert (n - n.flip(2)).abs().max().item() < 1e-4
        assert (n - n.flip(1)).abs().max().item() < 1e-4
        # FP64 diagnostics against direct reductions of the exports
        assert abs(float(n.double().sum()) - d[0]) <= 1e-9 * d[0]
        for c in range(3):
            ref = float(f[4 + c].double().sum())
            assert abs(ref - d[1 + c]) <= 1e-6 * max(abs(ref), 1.0), (c, ref, d[1 + c])
        assert float(n.min()) == pytest.approx(d[5], rel=1e-7)
        beta = f[1:4].double()
        assert float(beta.pow(2).sum(0).sqrt().max()) == pytest.approx(d[6], rel=1e-6)
        _, E, B = sim.get_state()
        energy = 0.5 * float(E.double().pow(2).sum() + B.double().pow(2).sum()) * w.dx ** 3
        assert energy == pytest.approx(d[4], rel=1e-9)


def test_production_workload_16bit_storage_2000_steps():
    """The production workload's 2000 steps with populations stored as BF16
    and FP16 deviations: every moment finite and n > 0 throughout (checked by
    the fused diagnostics every 100 steps), the bubble present at the end,
    and the relative L2 distance to the FP32 run at step 2000 recorded. In
    this non-linear regime no accuracy bar is stated for the 16-bit forms
    (the precision bar belongs to the 256x128x128 linear-driver form); the
    asserted bounds are regression guards at about three times the measured
    distances (GB300: FP16 n 1.3e-4, beta_z 3.4e-3, E_z 3.2e-3; BF16 n
    1.7e-3, beta_z 3.1e-2, E_z 2.6e-2), and FP16 must stay closer than
    BF16."""
    mask = lbm.FIELD_N | lbm.FIELD_UZ | lbm.FIELD_EZ | lbm.RAW_YEE
    runs = {}
    for st in (W.F32, W.F16, W.BF16):
        with lbm.Simulation(W.production().replace(storage=st)) as sim:
            for _ in range(20):
                d = sim.step_diag(100)[0]  # raises on a non-finite moment or n < 0
                assert d[7] == 0 and d[5] > 0, (st, d)
            assert 0 < sim.diag()[5] < 0.5
            runs[st] = sim.fields(mask).double()
    dist = {}
    for st in (W.F16, W.BF16):
        dist[st] = [float((runs[st][c] - runs[W.F32][c]).norm() / runs[W.F32][c].norm()) for c in range(3)]
    print("16-bit storage vs FP32 after 2000 production steps (n, beta_z, E_z):", dist)
    assert all(a < b for a, b in zip(dist[W.F16], dist[W.BF16]))
    assert max(dist[W.F16]) < 1e-2 and max(dist[W.BF16]) < 1e-1, dist
