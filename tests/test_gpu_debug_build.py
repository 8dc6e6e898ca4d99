"""The PWFA_DEBUG build of the library on small grids.

The debug build checks every element index the step kernels compute against
its array's extent and records a bad one in the instance's debug word
(without touching memory outside the array); the next public call then fails
with PWFA_ERR_STATE. Here it runs the step paths on 8x8x8 and 16x8x8 grids
(open and periodic, BGK and regularized, the three storage forms, the staged
fluid kernel, the fused field step, the batched path, the moving window, the
PIC driver, recording and the adjoint with its built-in loss, from a
one-segment recording and with the separate transposed field kernels) in a
child process: every call must succeed, and the states must equal those of
the release build.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2201_05473_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def cases():
    base = W.parity_small().replace(nx=8, ny=8, nz=8, z0=0.2, alpha=0.5, tau=0.6)
    long = base.replace(nz=16)
    return [
        ("open_bgk_f32", [base], dict(steps=30)),
        ("open_reg_bf16", [long.replace(collision=W.REGULARIZED, storage=W.BF16)], dict(steps=30, diag=True)),
        ("periodic_bgk_f16", [base.replace(boundary=W.PERIODIC, storage=W.F16)], dict(steps=20)),
        ("fused_fields", [long.replace(collision=W.REGULARIZED)], dict(steps=25, fusion=2)),
        ("batched", [base, long], dict(steps=10)),
        ("window", [long.replace(moving_window=1, window_z=0.2)], dict(steps=20)),
        ("pic", [long.replace(driver=1)], dict(steps=12, particles=400)),
        ("adjoint", [long.replace(profile=np.ones(4), profile_rmax=0.8)], dict(adjoint=12)),
        ("adjoint_one_segment_periodic", [long.replace(boundary=W.PERIODIC, collision=W.REGULARIZED)],
         dict(adjoint=10, ckpt=10)),
        ("adjoint_fusion_off", [long.replace(profile=np.ones(4), profile_rmax=0.8)], dict(adjoint=12, fusion=0)),
        ("fused_fields_periodic", [long.replace(boundary=W.PERIODIC)], dict(steps=25, fusion=2)),
        ("batched_periodic", [base.replace(boundary=W.PERIODIC), long.replace(boundary=W.PERIODIC)],
         dict(steps=10)),
        ("staged_fluid", [long.replace(collision=W.REGULARIZED, storage=W.BF16)], dict(steps=12, variant=1)),
    ]


def run_cases(lbm):
    """Run every case through the binding `lbm`; returns {name: arrays}."""
    out = {}
    for name, works, opt in cases():
        with lbm.Simulation(works) as sim:
            if "fusion" in opt:
                sim.set_field_fusion(opt["fusion"])
            if "variant" in opt:
                for i in range(len(works)):
                    sim.set_fluid_variant(opt["variant"], i)
            if "particles" in opt:
                w = works[0]
                xp, wt = W.bunch_particles(opt["particles"], w.alpha, w.sigma_r, w.sigma_z, w.z0, w.dt, w.nx, w.ny,
                                           w.dx)
                sim.set_particles(xp, wt)
            if "adjoint" in opt:
                g = sim.adjoint_step(None, nsteps=opt["adjoint"], ckpt_every=opt.get("ckpt", 5))
                out[name + "/grad"] = g
            else:
                sim.step(opt["steps"])
            if opt.get("diag"):
                out[name + "/diag"] = sim.step_diag(1)
            for i in range(len(works)):
                f, E, B = sim.get_state(i)
                out[f"{name}/{i}/f"] = f.cpu().numpy()
                out[f"{name}/{i}/E"] = E.cpu().numpy()
                out[f"{name}/{i}/B"] = B.cpu().numpy()
    return out


CHILD = r"""
import sys
sys.path.insert(0, %(root)r)
sys.path.insert(0, %(here)r)
import numpy as np
from paper_2201_05473_gb300 import lbm
lbm.LIB_PATH = %(lib)r
lbm.load(build=False)
import test_gpu_debug_build as T
res = T.run_cases(lbm)
np.savez(%(out)r, **res)
print("DEBUG_OK")
"""


def test_debug_build_small_grids(tmp_path):
    from paper_2201_05473_gb300.build import build
    lib = build(defines=["PWFA_DEBUG"], lib_path=os.path.join(ROOT, "paper_2201_05473_gb300",
                                                              "libpwfa_lbm_debug.so"))
    out = str(tmp_path / "debug.npz")
    cp = subprocess.run([sys.executable, "-c", CHILD % {"root": ROOT, "here": HERE, "lib": lib, "out": out}],
                        capture_output=True, text=True, timeout=900)
    assert cp.returncode == 0 and "DEBUG_OK" in cp.stdout, (cp.stdout[-2000:], cp.stderr[-3000:])
    dbg = dict(np.load(out))
    from paper_2201_05473_gb300 import lbm
    rel = run_cases(lbm)
    assert sorted(dbg) == sorted(rel)
    for k in rel:
        a, b = dbg[k].astype(np.float64), rel[k].astype(np.float64)
        assert np.all(np.isfinite(a)), k
        # the same arithmetic; atomic sums (the adjoint's FP64 driver terms,
        # the PIC deposit's FP32 current) may add in another order
        assert np.allclose(a, b, rtol=1e-6, atol=1e-7), (k, float(np.abs(a - b).max()))
