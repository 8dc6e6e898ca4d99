"""Reduced-precision population storage (BF16 / FP16 deviations from the
plasma at rest, FP32 compute) against the FP64 oracle on the precision form:
the 64x32x32 workload's physics (n_b/n0 = 0.1, sigma = 0.5, dx = 0.2, BGK)
on 256x128x128 nodes, errors of n, beta and E_z every 100 steps up to 1000.

Bars: FP32 storage <= 1e-5 after 200 steps; reduced-precision storage
<= 1e-3 at every step. FP16 (deviations scaled by 2^10 / w_i) meets it.
BF16 misses it: its 8-bit significand rounds every stored population of the
momentum lattices by up to 2^-9 relative each step, which leaves beta at
1.2e-3 after 100 steps and 2.8e-3 after 1000 (E_z passes 1e-3 near step
550). Stochastic rounding of the BF16 stores was measured and is worse
(3.4e-3 on beta at step 1000): the per-step rounding noise, not a bias,
sets the error. The BF16 test holds the measured table (within 50 %) as a
regression guard; it is not a bar."""
import numpy as np
import pytest

import oracle
from paper_2201_05473_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2201_05473_gb300 import lbm  # noqa: E402

STEPS = list(range(100, 1001, 100))

# BF16 errors measured on a GB300 (n, beta, E_z at steps 100..1000; the
# larger of two runs that differed in the rounding of the driver current)
BF16_MEASURED = {
    "n": [1.08e-6, 4.19e-6, 8.70e-6, 1.47e-5, 2.14e-5, 2.91e-5, 3.79e-5, 4.75e-5, 5.85e-5, 6.98e-5],
    "beta": [1.28e-3, 1.76e-3, 1.99e-3, 2.12e-3, 2.26e-3, 2.36e-3, 2.42e-3, 2.51e-3, 2.61e-3, 2.78e-3],
    "Ez": [3.06e-4, 6.19e-4, 7.63e-4, 8.52e-4, 1.03e-3, 1.23e-3, 1.43e-3, 1.69e-3, 1.92e-3, 2.17e-3],
}


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.fixture(scope="module")
def precision_table():
    """Errors of the three storage forms against one FP64 oracle run."""
    base = W.precision_form(W.F32)
    oracle.build()
    o = oracle.Oracle(base.nx, base.ny, base.nz, base.dx, base.dt, base.tau, alpha=base.alpha,
                      sigma_r=base.sigma_r, sigma_z=base.sigma_z, z0=base.z0)
    m = lbm.FIELD_N | lbm.FIELD_UX | lbm.FIELD_UY | lbm.FIELD_UZ | lbm.FIELD_EZ | lbm.RAW_YEE
    forms = {"f32": W.F32, "bf16": W.BF16, "f16": W.F16}
    sims = {k: lbm.Simulation(base.replace(storage=st)) for k, st in forms.items()}
    table = {k: [] for k in forms}
    try:
        for s in STEPS:
            o.step(100)
            mo = o.moments()
            E, _ = o.get_fields()
            for k, sim in sims.items():
                sim.step(100)
                g = sim.fields(m).cpu().numpy().astype(np.float64)
                table[k].append({"step": s, "n": rel(g[0], mo["n"]), "beta": rel(g[1:4], mo["beta"]),
                                 "Ez": rel(g[4], E[2])})
    finally:
        for sim in sims.values():
            sim.close()
        o.close()
    for k, rows in table.items():
        for r in rows:
            print(k, r)
    return table


def test_fp32_storage_meets_1e5_at_step_200(precision_table):
    r = precision_table["f32"][STEPS.index(200)]
    assert r["n"] <= 1e-5 and r["beta"] <= 1e-5 and r["Ez"] <= 1e-5, r


def test_fp16_storage_meets_1e3_every_step(precision_table):
    for r in precision_table["f16"]:
        assert r["n"] <= 1e-3 and r["beta"] <= 1e-3 and r["Ez"] <= 1e-3, r


def test_bf16_storage_misses_the_1e3_bar_measured_table(precision_table):
    """BF16 does not meet the 1e-3 bar (see the module docstring); its
    errors stay within 50 % of the table measured on a GB300."""
    for i, r in enumerate(precision_table["bf16"]):
        for q in ("n", "beta", "Ez"):
            assert r[q] <= 1.5 * BF16_MEASURED[q][i], (q, r, BF16_MEASURED[q][i])


@pytest.mark.parametrize("storage,eps", [(W.F16, 2.0 ** -11), (W.BF16, 2.0 ** -8)])
def test_deviation_codec_roundtrip(storage, eps):
    """Stored values are f - w_i n0 (lattice 0) and f (momentum lattices) in
    the reduced format, round-to-nearest-even: the round trip error of each
    population is within half an ulp of its deviation."""
    w = W.parity_small().replace(nx=9, ny=6, nz=11, boundary=W.PERIODIC, storage=storage)
    f0 = W.random_populations((w.nz, w.ny, w.nx), seed=4)
    wq = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    base = np.zeros_like(f0)
    base[0] = wq[:, None, None, None] * w.n0
    with lbm.Simulation(w) as sim:
        sim.set_state(f0.astype(np.float32))
        f, _, _ = sim.get_state(device=False)
    dev = np.abs(f0 - base)
    err = np.abs(f.numpy().astype(np.float64) - f0)
    # plus FP32 rounding of f and the FP16 subnormal spacing (2^-24) near zero
    assert np.all(err <= eps * dev * 1.0001 + 1e-7 * np.abs(f0) + 6e-8)
