"""Failure paths on a GPU, made on the host (no GPU fault is provoked).

Allocation failure: with PWFA_FAIL_ALLOC_AT=n the library's n-th device
allocation fails as an out-of-memory cudaMalloc would. Each case runs in a
fresh child process: pwfa_lbm_create and pwfa_lbm_record return
PWFA_ERR_ALLOC, the device memory the failed call had taken is returned
(cudaMemGetInfo back to its level before the call), and the handle that
survives a failed record still steps and records.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import ctypes, json, sys
sys.path.insert(0, %(root)r)
import torch
from paper_2201_05473_gb300 import lbm, workloads as W
lib = lbm.load(build=False)
torch.cuda.init()
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
# 128x128x128 FP32: a 1.4 GB arena, so a leak would show
w = W.parity_small().replace(nx=128, ny=128, nz=128)
p, keep = lbm.params_of(w)
h = ctypes.c_void_p()
out = {"create": lib.pwfa_lbm_create(ctypes.byref(p), 1, None, ctypes.byref(h))}
torch.cuda.synchronize()
out["free_after_create"] = torch.cuda.mem_get_info()[0]
out["free0"] = free0
out["handle"] = bool(h.value)
if h.value:
    out["record"] = lib.pwfa_lbm_record(h, 0, 9, 3)
    out["record_msg"] = lib.pwfa_lbm_last_error().decode()
    torch.cuda.synchronize()
    out["free_after_record"] = torch.cuda.mem_get_info()[0]
    out["step_after"] = lib.pwfa_lbm_step(h, 2)
    out["record_again"] = lib.pwfa_lbm_record(h, 0, 4, 2)
    torch.cuda.synchronize()
    out["destroy"] = lib.pwfa_lbm_destroy(h)
torch.cuda.synchronize()
out["free_end"] = torch.cuda.mem_get_info()[0]
print("RESULT " + json.dumps(out))
"""


def run_child(fail_at):
    env = dict(os.environ)
    if fail_at is None:
        env.pop("PWFA_FAIL_ALLOC_AT", None)
    else:
        env["PWFA_FAIL_ALLOC_AT"] = str(fail_at)
    cp = subprocess.run([sys.executable, "-c", CHILD % {"root": ROOT}], capture_output=True, text=True,
                        timeout=300, env=env)
    assert cp.returncode == 0, cp.stderr[-3000:]
    line = [l for l in cp.stdout.splitlines() if l.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


SLACK = 8 << 20  # cudaMemGetInfo granularity and the runtime's own buffers


def test_allocation_failures_return_err_alloc_and_leak_nothing():
    ok = run_child(None)
    assert ok["create"] == 0 and ok["record"] == 0 and ok["destroy"] == 0
    # create makes two allocations (the instance arena, the diagnostics
    # buffer); record three (checkpoints, segment states, adjoint scratch)
    for n in (1, 2):
        r = run_child(n)
        assert r["create"] == -5 and not r["handle"], r
        assert abs(r["free_after_create"] - r["free0"]) <= SLACK, r
    for n in (3, 4, 5):
        r = run_child(n)
        assert r["create"] == 0 and r["record"] == -5, r
        assert "recording needs" in r["record_msg"]
        # the failed record returned what it had taken
        assert abs(r["free_after_record"] - r["free_after_create"]) <= SLACK, r
        # the handle is still usable
        assert r["step_after"] == 0 and r["record_again"] == 0 and r["destroy"] == 0, r
        assert abs(r["free_end"] - r["free0"]) <= SLACK, r
