"""GPU 2D-axisymmetric (z, r) form through the pwfa_axi_* C ABI against the
FP64 axisymmetric oracle: element-wise parity on the linear-driver workload
and bit-exact streaming on integer populations."""
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


def make_oracle(w):
    oracle.build()
    return oracle.AxiOracle(w.nz, w.nr, w.dx, w.dt, w.tau, collision=w.collision, couple=w.couple, n0=w.n0,
                            alpha=w.alpha, sigma_r=w.sigma_r, sigma_z=w.sigma_z, z0=w.z0, n_floor=w.n_floor)


@pytest.mark.parametrize("steps", [1, 200])
def test_axisymmetric_parity(steps):
    """n_b/n0 = 0.1, sigma 0.5, 64 x 34 at dx 0.2: every output within rel-L2
    1e-5 of the FP64 oracle after 200 steps."""
    w = W.axisymmetric_parity()
    o = make_oracle(w)
    o.step(steps)
    with lbm.AxiSimulation(w) as sim:
        sim.step(steps)
        assert sim.steps_done() == steps
        g = sim.fields().cpu().numpy().astype(np.float64)
    m = o.moments()
    Ez, Er, Bt = o.get_fields()
    errs = {"n": rel(g[0], m["n"]), "beta_z": rel(g[1], m["beta_z"]), "beta_r": rel(g[2], m["beta_r"]),
            "Ez": rel(g[3], Ez), "Er": rel(g[4], Er), "Bt": rel(g[5], Bt)}
    print(errs)
    assert max(errs.values()) <= 1e-5, errs


def test_axisymmetric_paper_grid_parity():
    """The paper's own grid (2400 x 402 at dz = dr = 0.25 um, Sec. IV) at
    Q = 1 (n_b/n0 = 6.8), the driver started inside the box at z0 = 4
    sigma_z: the launch configuration the benchmark times, 100 steps against
    the FP64 oracle on every output (rel-L2 1e-5). The grid is fine in plasma
    units (a plasma period is ~7600 steps), so this covers the driver's field
    build-up and the first fluid response over the whole grid."""
    w = W.axisymmetric_paper(1.0)
    w = w.replace(z0=4.0 * w.sigma_z)
    o = make_oracle(w)
    o.step(100)
    with lbm.AxiSimulation(w) as sim:
        sim.step(100)
        g = sim.fields().cpu().numpy().astype(np.float64)
    m = o.moments()
    Ez, Er, Bt = o.get_fields()
    errs = {"n": rel(g[0], m["n"]), "beta_z": rel(g[1], m["beta_z"]), "beta_r": rel(g[2], m["beta_r"]),
            "Ez": rel(g[3], Ez), "Er": rel(g[4], Er), "Bt": rel(g[5], Bt)}
    print("paper grid:", errs)
    assert np.abs(Ez).max() > 0 and np.abs(m["beta_z"]).max() > 0
    assert max(errs.values()) <= 1e-5, errs


def test_axisymmetric_streaming_bit_exact():
    """Stream-only lattices, no fields, integer populations: after a step the
    stored source equals the oracle's bit for bit on every interior node and
    on the mirror row of interior columns."""
    w = W.axisymmetric_parity().replace(nz=40, nr=20, collision=W.STREAM_ONLY, couple=0, alpha=0.0)
    N = w.nz * w.nr
    S = (np.arange(27 * N, dtype=np.float64) + 1.0).reshape(3, 9, w.nz, w.nr)
    o = make_oracle(w)
    o.set_source(S)
    o.step(1)
    with lbm.AxiSimulation(w) as sim:
        sim.set_source(S)
        sim.step(1)
        g = sim.get_source().cpu().numpy().astype(np.float64)
    want = o.get_source()
    inner = (slice(None), slice(None), slice(1, w.nz - 1), slice(0, w.nr - 1))
    assert np.array_equal(g[inner], want[inner])
    # boundary nodes hold equilibria (FP32 arithmetic)
    assert rel(g, want) < 1e-6


def test_axisymmetric_uniform_plasma_is_steady():
    w = W.axisymmetric_parity().replace(alpha=0.0, n0=1.3)
    with lbm.AxiSimulation(w) as sim:
        sim.step(50)
        g = sim.fields().cpu().numpy()
    assert np.abs(g[0] - 1.3).max() < 1e-5 and np.abs(g[1:]).max() < 1e-6
