"""The patch method of the full-size parity test, checked on the oracle alone.

A one-step update reaches two nodes (pull from post-collision values at
distance 1 whose node fields average edges and faces at distance 1; E after
Ampere reads B(t_{n+1}) at distance 1, formed from E at distance 2). So an
open patch cut out of a state, stepped once as a box of its own, must give
the full grid's next step at every node 3 or more nodes from the patch's cut
faces; faces that are walls of the grid stay walls. On the driver axis the
patch is cut symmetric about it (the oracle centres the axis in its box) and
z0 is shifted by the elapsed time and the patch's first plane.
"""
import numpy as np
import pytest

import oracle
from paper_2201_05473_gb300 import workloads as W


def _oracle(nx, ny, nz, w, alpha, z0):
    return oracle.Oracle(nx, ny, nz, w.dx, w.dt, w.tau, collision=w.collision, boundary=W.OPEN, couple=w.couple,
                         n0=w.n0, profile=None, profile_rmax=0.0, alpha=alpha, sigma_r=w.sigma_r,
                         sigma_z=w.sigma_z, z0=z0, n_floor=w.n_floor)


@pytest.mark.parametrize("collision", [W.REGULARIZED, W.BGK])
def test_patch_step_equals_full_step(collision):
    oracle.build()
    w = W.parity_small().replace(nx=20, ny=20, nz=30, alpha=0.8, sigma_r=0.5, sigma_z=0.5, z0=1.5, tau=0.6,
                                 collision=collision)
    full = _oracle(w.nx, w.ny, w.nz, w, w.alpha, w.z0)
    n = 25
    full.step(n)
    f0 = full.get_f()
    E0, B0 = full.get_fields()
    full.step(1)
    f1 = full.get_f()
    E1, B1 = full.get_fields()
    full.close()
    assert np.abs(f0[1:]).max() > 1e-4  # a driven, moving state
    kd = int(round((w.z0 + n * w.dt) / w.dx))
    # (k0, j0, i0, shape, driver, interior nodes to compare); axis patches
    # span x, y in 6..13 (symmetric about 9.5)
    checked = 0
    for k0, j0, i0, shp, drv, nodes in [
        (kd - 3, 6, 6, (7, 8, 8), True, [(3, j, i) for j in (3, 4) for i in (3, 4)]),
        (0, 6, 6, (7, 8, 8), True, [(k, 3, 4) for k in (0, 1, 2, 3)]),
        (w.nz - 7, 6, 6, (7, 8, 8), True, [(k, 4, 3) for k in (3, 4, 5, 6)]),
    ]:
        pz, py, px = shp
        sl = (slice(k0, k0 + pz), slice(j0, j0 + py), slice(i0, i0 + px))
        o = _oracle(px, py, pz, w, w.alpha if drv else 0.0, w.z0 + n * w.dt - k0 * w.dx)
        o.set_f(f0[(slice(None), slice(None)) + sl])
        o.set_fields(E0[(slice(None),) + sl], B0[(slice(None),) + sl])
        o.step(1)
        fo = o.get_f()
        Eo, Bo = o.get_fields()
        o.close()
        for (k, j, i) in nodes:
            g = (k0 + k, j0 + j, i0 + i)
            assert np.allclose(fo[:, :, k, j, i], f1[(slice(None), slice(None)) + g], rtol=1e-12, atol=1e-15), g
            assert np.allclose(Eo[:, k, j, i], E1[(slice(None),) + g], rtol=1e-12, atol=1e-15), g
            assert np.allclose(Bo[:, k, j, i], B1[(slice(None),) + g], rtol=1e-12, atol=1e-15), g
            checked += 1
    assert checked == 12


def test_patch_too_close_to_a_cut_face_differs():
    """The distance rule is not vacuous: a node 1 away from a cut face does
    not reproduce the full step."""
    oracle.build()
    w = W.parity_small().replace(nx=20, ny=20, nz=30, alpha=0.8, sigma_r=0.5, sigma_z=0.5, z0=1.5, tau=0.6)
    full = _oracle(w.nx, w.ny, w.nz, w, w.alpha, w.z0)
    n = 25
    full.step(n)
    f0 = full.get_f()
    E0, B0 = full.get_fields()
    full.step(1)
    f1 = full.get_f()
    full.close()
    kd = int(round((w.z0 + n * w.dt) / w.dx))
    k0, j0, i0 = kd - 3, 6, 6
    sl = (slice(k0, k0 + 7), slice(j0, j0 + 8), slice(i0, i0 + 8))
    o = _oracle(8, 8, 7, w, w.alpha, w.z0 + n * w.dt - k0 * w.dx)
    o.set_f(f0[(slice(None), slice(None)) + sl])
    o.set_fields(E0[(slice(None),) + sl], B0[(slice(None),) + sl])
    o.step(1)
    fo = o.get_f()
    o.close()
    # the populations one node inside the cut x face at the driver plane:
    # they pull post-collision values from the face node, whose node fields
    # average edges outside the patch
    g = (slice(None), slice(None), k0 + 3, j0 + 4, i0 + 1)
    assert not np.allclose(fo[:, :, 3, 4, 1], f1[g], rtol=1e-9, atol=1e-12)
