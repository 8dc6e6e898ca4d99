"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every function declared in include/*.h, its params
struct matches the header's layout, and invalid parameters are rejected with
PWFA_ERR_PARAM before any device work."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

from paper_2201_05473_gb300 import lbm
from paper_2201_05473_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(pwfa_lbm_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    return lbm.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "pwfa_lbm_create" in names and "pwfa_lbm_step" in names
    out = subprocess.run(["nm", "-D", "--defined-only", lbm.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pwfa_lbm_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


@pytest.mark.parametrize("cname,pytype", [("pwfa_lbm_params", lbm.Params), ("pwfa_axi_params", lbm.AxiParams)])
def test_params_layout_matches_header(tmp_path, cname, pytype):
    """Compile a probe against the header and compare offsets with ctypes."""
    fields = [f[0] for f in pytype._fields_]
    prog = ["#include <stdio.h>", "#include <stddef.h>", '#include "pwfa_lbm.h"', "int main(void){",
            f'printf("%zu\\n", sizeof({cname}));']
    prog += [f'printf("%zu\\n", offsetof({cname}, {f}));' for f in fields]
    prog += ["return 0;}"]
    c = tmp_path / "probe.c"
    c.write_text("\n".join(prog))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert vals[0] == ctypes.sizeof(pytype)
    assert len(vals) == len(fields) + 1
    for f, off in zip(fields, vals[1:]):
        assert getattr(pytype, f).offset == off, f


def _create(lib, **changes):
    w = W.parity_small().replace(**changes)
    p, keep = lbm.params_of(w)
    h = ctypes.c_void_p()
    rc = lib.pwfa_lbm_create(ctypes.byref(p), 1, None, ctypes.byref(h))
    return rc, h, lib.pwfa_lbm_last_error().decode()


@pytest.mark.parametrize("change,needle", [
    (dict(nx=2), "nx, ny, nz"),
    (dict(tau=0.5), "tau"),
    (dict(dx=0.0), "dx"),
    (dict(collision=7), "collision"),
    (dict(storage=9), "storage"),
    (dict(boundary=3), "boundary"),
    (dict(sigma_r=0.0), "sigma"),
    (dict(alpha=-1.0), "alpha"),
    (dict(n0=float("nan")), "n0"),
    (dict(moving_window=2), "moving_window"),
    (dict(moving_window=1, boundary=1), "moving window"),
    (dict(moving_window=1, window_z=float("inf")), "window_z"),
    # maximum sizes: the x-y plane, the z extent and the 32-bit population
    # offsets (19 Np < 2^32: 512 x 512 x 900 nodes is past it)
    (dict(nx=1 << 16, ny=1 << 15), "grid too large"),
    (dict(nz=70000), "grid too large"),
    (dict(nx=512, ny=512, nz=900), "nodes * 19"),
    (dict(driver=5), "unknown driver"),
    (dict(driver=1, moving_window=1), "PIC driver"),
])
def test_invalid_params_rejected(lib, change, needle):
    rc, h, msg = _create(lib, **change)
    assert rc == -1 and not h.value
    assert needle in msg


def test_courant_limit_rejected(lib):
    w = W.parity_small()
    p, keep = lbm.params_of(w)
    p.dt = 0.2 * w.dx / 0.3  # above dx / sqrt(3)
    h = ctypes.c_void_p()
    assert lib.pwfa_lbm_create(ctypes.byref(p), 1, None, ctypes.byref(h)) == -1
    assert "Courant" in lib.pwfa_lbm_last_error().decode()


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.pwfa_lbm_create(None, 1, None, ctypes.byref(h)) == -1
    assert lib.pwfa_lbm_step(None, 1) == -1
    assert lib.pwfa_lbm_destroy(None) == 0
    assert lib.pwfa_lbm_fields(None, 0, 1, None, 0, None) == -1
    assert lib.pwfa_lbm_steps_done(None, 0) == -1
    assert lib.pwfa_lbm_set_field_fusion(None, 1) == -1
    assert lib.pwfa_lbm_set_batching(None, 1) == -1
    assert lib.pwfa_lbm_step_diag(None, 1, None) == -1
    g = (ctypes.c_double * 3)()
    assert lib.pwfa_lbm_adjoint_step(None, 0, None, 10, 0, g, 3) == -1
    assert lib.pwfa_lbm_witness_loss(None, 0, g) == -1


def test_noalloc_argument_checks(lib):
    """pwfa_lbm_diag_noalloc rejects bad arguments with PWFA_ERR_PARAM before
    any CUDA call (the pointers below are never dereferenced)."""
    fake = ctypes.c_void_p(0x1000)

    def call(nx=8, ny=8, nz=8, dx=0.2, n_floor=0.0, f=fake, E=fake, B=fake, out=fake):
        return lib.pwfa_lbm_diag_noalloc(nx, ny, nz, dx, n_floor, f, E, B, out, None)

    assert call(nx=1024, ny=1024, nz=128) == -1  # 134 M nodes, above the fixed scratch
    assert "exceeds" in lib.pwfa_lbm_last_error().decode()
    assert call(nx=0) == -1
    assert call(f=None) == -1
    assert call(dx=0.0) == -1
    assert call(n_floor=-1.0) == -1 and "n_floor" in lib.pwfa_lbm_last_error().decode()
    assert call(n_floor=float("nan")) == -1
