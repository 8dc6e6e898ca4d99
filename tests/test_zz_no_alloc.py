"""The allocation-free diagnostics entry point, called through the C ABI.

It exists for callers that must not let the library allocate device memory
(an in-situ analysis hook inside another code, or an application that owns a
fixed device-memory budget), so it reduces a state the caller already holds.
Its result must match the handle-based diagnostics of pwfa_lbm_fields on the
same state, on two calls in a row (the shared scratch array keeps the
previous call's contents). This file is collected last on purpose.
"""
import ctypes

import pytest

from paper_2201_05473_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2201_05473_gb300 import lbm  # noqa: E402


def _noalloc(lib, w, f, E, B, out, stream):
    return lib.pwfa_lbm_diag_noalloc(w.nx, w.ny, w.nz, w.dx, w.n_floor,
                                     ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(E.data_ptr()),
                                     ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(stream.cuda_stream))


def _check(got, ref):
    # The same node values reduced in another order; boundary-node populations
    # come back as f^eq of the clamped node's moments, re-summed in FP32.
    # sum n: relative 1e-6. Momentum sums: the wake is mirror-symmetric, so the
    # transverse sums are rounding noise around zero: absolute 1e-5 (each
    # node's n p is ~1e-3, ~3.5e4 nodes). Field energy: the identical FP32
    # values summed in FP64, relative 1e-9. Extremes: absolute 1e-6.
    assert abs(got[0] - ref[0]) <= 1e-6 * abs(ref[0]), (got[0], ref[0])
    for i in (1, 2, 3):
        assert abs(got[i] - ref[i]) <= 1e-5, (i, got[i], ref[i])
    assert abs(got[4] - ref[4]) <= 1e-9 * abs(ref[4]) + 1e-300, (got[4], ref[4])
    assert abs(got[5] - ref[5]) < 1e-6 and abs(got[6] - ref[6]) < 1e-6
    assert got[7] == ref[7] == 0


def test_noalloc_diagnostics_match_handle_diagnostics():
    lib = lbm.load()
    w = W.parity_small().replace(nx=37, ny=20, nz=48, alpha=0.5, z0=-1.0)
    stream = torch.cuda.current_stream()
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with lbm.Simulation(w, stream=stream) as sim:
        for steps in (40, 25):  # two calls in a row, on two different states
            sim.step(steps)
            ref = sim.diag()
            f, E, B = sim.get_state()
            rc = _noalloc(lib, w, f, E, B, out, stream)
            assert rc == 0, lib.pwfa_lbm_last_error().decode()
            torch.cuda.synchronize()
            _check(out.cpu().numpy(), ref)


def test_noalloc_diagnostics_many_blocks():
    """A grid of 1.57 M nodes: 384 first-pass blocks of 4096 nodes, so the
    finishing kernel loops over more than its 256 threads' worth of block
    records and the scratch records past the first 256 are used."""
    lib = lbm.load()
    w = W.parity_small().replace(nx=128, ny=128, nz=96, alpha=0.5, z0=-1.0)
    stream = torch.cuda.current_stream()
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with lbm.Simulation(w, stream=stream) as sim:
        for steps in (30, 10):
            sim.step(steps)
            ref = sim.diag()
            f, E, B = sim.get_state()
            rc = _noalloc(lib, w, f, E, B, out, stream)
            assert rc == 0, lib.pwfa_lbm_last_error().decode()
            torch.cuda.synchronize()
            _check(out.cpu().numpy(), ref)
