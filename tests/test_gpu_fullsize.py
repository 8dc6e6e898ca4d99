"""Full-size parity on sampled nodes.

The production workload (512x256x256 at dx = 0.05, n_b/n0 = 1, sigma_r =
0.3, sigma_z = 0.5, driver started inside the box) runs on the GPU in the
launch configuration the benchmark times (autotuned fluid block, fused field
step) until the non-linear wake has formed. Its state is then cut into
small patches around sampled nodes: on the driver axis at the driver, in the
bubble and behind it, next to the z walls, and off the axis at the x and y
walls and in a corner. The FP64 oracle takes one step of each patch (an open
box of its own), and the node at the patch centre must equal the GPU's next
step there: all 76 populations, E and B.

One step of the scheme reaches two nodes: a node's new populations are
pulled from post-collision values at distance 1, whose node fields average
edges and faces at distance 1, and E after Ampere reads B(t_{n+1}) at
distance 1, which Faraday formed from E at distance 2. A patch face the
oracle treats as a wall (Eq. 14 boundary nodes, conducting walls, zero
outside) therefore changes nothing at distance 3 from it. Patches that
contain a true wall of the grid keep it where the grid has it.

Driver: patches on the axis span a transverse range symmetric about it (the
oracle puts the axis at the centre of its box) and shift z0 so that the
oracle's driver is where the GPU's is after the prelude. Patches off the
axis lie at r >= 6 c/omega_p, where the driver density exp(-r^2/2 sigma_r^2)
underflows in FP32 and FP64 alike: the oracle runs them without a driver.

Tolerance: one FP32 step against FP64; each compared value within 2e-6 of
the largest magnitude of its group (the node's 76 populations; E and B of
the patch), several times the FP32 rounding of a step's arithmetic. With
populations stored in 16 bits (BF16, FP16) the state the oracle starts from
is the GPU's decoded one, so each new population carries exactly one
rounding of its stored deviation on top: |f_gpu - f| <= u |f - ref| with u
the format's unit roundoff (2^-8, 2^-11) and ref = w_i n0 for lattice 0, 0
for the momentum lattices; E and B stay FP32.
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

PRELUDE = 300
TOL = 2e-6
UNIT_ROUNDOFF = {W.BF16: 2.0 ** -8, W.F16: 2.0 ** -11}
WEIGHTS = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def patch_oracle(w, shape_zyx, k0, driver, steps_done):
    nz, ny, nx = shape_zyx
    oracle.build()
    # the driver centre z0 + t of the GPU after steps_done steps, in the
    # patch's own z coordinate (patch plane 0 = grid plane k0)
    z0 = w.z0 + steps_done * w.dt - k0 * w.dx
    return oracle.Oracle(nx, ny, nz, w.dx, w.dt, w.tau, collision=w.collision, boundary=W.OPEN, couple=w.couple,
                         n0=w.n0, profile=None, profile_rmax=0.0, alpha=w.alpha if driver else 0.0,
                         sigma_r=w.sigma_r, sigma_z=w.sigma_z, z0=z0, n_floor=w.n_floor)


@pytest.mark.parametrize("collision,storage", [(W.REGULARIZED, W.F32), (W.BGK, W.F32), (W.REGULARIZED, W.BF16),
                                               (W.REGULARIZED, W.F16)])
def test_full_size_sampled_nodes_match_oracle(collision, storage):
    w = W.production_timing().replace(collision=collision, storage=storage)
    u = UNIT_ROUNDOFF.get(storage, 0.0)
    ref = np.zeros((4, 19))
    ref[0] = WEIGHTS * w.n0
    nz, ny, nx = w.nz, w.ny, w.nx
    with lbm.Simulation(w) as sim:
        sim.step(PRELUDE)
        sim.autotune(3)
        n_done = sim.steps_done()
        d = sim.diag()
        assert d[7] == 0 and d[5] < 0.9, d  # the wake is there (min n well below 1)
        f0, E0, B0 = sim.get_state()
        sim.step(1)
        f1, E1, B1 = sim.get_state()
        kd = int(round((w.z0 + n_done * w.dt) / w.dx))  # driver centre plane
        ca, cb = nx // 2 - 4, ny // 2 - 4  # 8 columns symmetric about the axis
        # (k0, j0, i0, shape zyx, driver, sampled nodes in patch coordinates)
        axis_nodes = [(3, j, i) for j in (3, 4) for i in (3, 4)]
        patches = [
            (kd - 3, cb, ca, (7, 8, 8), True, axis_nodes),
            (kd - 28, cb, ca, (7, 8, 8), True, axis_nodes),
            (kd - 63, cb, ca, (7, 8, 8), True, axis_nodes),
            (kd + 7, cb, ca, (7, 8, 8), True, axis_nodes),
            (0, cb, ca, (7, 8, 8), True, [(k, 3, 4) for k in (0, 1, 2, 3)]),
            (nz - 7, cb, ca, (7, 8, 8), True, [(k, 4, 3) for k in (3, 4, 5, 6)]),
            (kd - 3, 0, 0, (7, 7, 7), False, [(3, j, i) for j in (0, 1, 3) for i in (0, 2, 3)]),
            (kd - 20, ny // 2 - 3, nx - 7, (7, 7, 7), False, [(3, 3, i) for i in (3, 4, 5, 6)]),
            (kd + 40, ny - 7, nx // 2 - 3, (7, 7, 7), False, [(3, j, 3) for j in (3, 5, 6)]),
        ]
        worst = {"f": 0.0, "E": 0.0, "B": 0.0}
        for k0, j0, i0, shp, driver, nodes in patches:
            pz, py, px = shp
            sl = (slice(k0, k0 + pz), slice(j0, j0 + py), slice(i0, i0 + px))
            fp = f0[(slice(None), slice(None)) + sl].double().cpu().numpy()
            Ep = E0[(slice(None),) + sl].double().cpu().numpy()
            Bp = B0[(slice(None),) + sl].double().cpu().numpy()
            o = patch_oracle(w, shp, k0, driver, n_done)
            o.set_f(fp)
            o.set_fields(Ep, Bp)
            o.step(1)
            fo = o.get_f()
            Eo, Bo = o.get_fields()
            o.close()
            fg = f1[(slice(None), slice(None)) + sl].double().cpu().numpy()
            Eg = E1[(slice(None),) + sl].double().cpu().numpy()
            Bg = B1[(slice(None),) + sl].double().cpu().numpy()
            sE = max(np.abs(Eo).max(), 1e-6)
            sB = max(np.abs(Bo).max(), 1e-6)
            for (k, j, i) in nodes:
                fn_o, fn_g = fo[:, :, k, j, i], fg[:, :, k, j, i]
                # beyond the one rounding of the stored deviation (16-bit forms)
                excess = np.maximum(np.abs(fn_g - fn_o) - 1.01 * u * np.abs(fn_o - ref), 0.0)
                ef = excess.max() / np.abs(fn_o).max()
                eE = np.abs(Eg[:, k, j, i] - Eo[:, k, j, i]).max() / sE
                eB = np.abs(Bg[:, k, j, i] - Bo[:, k, j, i]).max() / sB
                where = (k0 + k, j0 + j, i0 + i)
                assert ef <= TOL, ("f", where, ef)
                assert eE <= TOL, ("E", where, eE, Eg[:, k, j, i], Eo[:, k, j, i])
                assert eB <= TOL, ("B", where, eB, Bg[:, k, j, i], Bo[:, k, j, i])
                worst["f"] = max(worst["f"], ef)
                worst["E"] = max(worst["E"], eE)
                worst["B"] = max(worst["B"], eB)
        print("full-size sampled parity,", storage, collision, "worst scaled error:", worst)
