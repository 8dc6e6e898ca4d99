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


CHILD_CUDA_ERROR = r"""
import json, sys
sys.path.insert(0, %(root)r)
import torch
from paper_2201_05473_gb300 import lbm, workloads as W
lbm.load(build=False)
w = W.parity_small().replace(nx=16, ny=16, nz=32)
out = {}
s = torch.cuda.Stream()
with torch.cuda.stream(s):
    sim = lbm.Simulation(w, stream=s)
    sim.step(2)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    g.capture_begin()
    try:
        sim.step_diag(1)  # its host read synchronises the capturing stream
        out["code"] = 0
    except lbm.LBMError as e:
        out["code"] = e.code
        out["msg"] = str(e)
    try:
        g.capture_end()
        out["capture_end"] = "ok"
    except Exception as e:
        out["capture_end"] = type(e).__name__
    torch.cuda.synchronize()
    sim.close()
    # the process and the device carry on: a new handle steps and matches a
    # handle that never saw the error
    with lbm.Simulation(w, stream=s) as a:
        a.step(5)
        fa = a.fields(lbm.FIELD_N | lbm.FIELD_EZ | lbm.RAW_YEE)
    with lbm.Simulation(w) as b:
        b.step(5)
        fb = b.fields(lbm.FIELD_N | lbm.FIELD_EZ | lbm.RAW_YEE)
    out["after_equal"] = bool(torch.equal(fa, fb))
print("RESULT " + json.dumps(out))
"""


def test_cuda_error_is_returned_not_raised_on_the_device():
    """A CUDA runtime error made on the host, with no device fault: the
    library's call is made while the caller captures its stream into a
    graph, so the runtime refuses what the call needs (here the first
    diagnostics call's cudaMalloc, which is not an out-of-memory). The call
    returns PWFA_ERR_CUDA, not PWFA_ERR_ALLOC, with the CUDA error named;
    after the caller ends the
    (invalidated) capture, the process and the device carry on (a new handle
    steps and equals one that never saw the error). Child process, like the
    allocation failures."""
    cp = subprocess.run([sys.executable, "-c", CHILD_CUDA_ERROR % {"root": ROOT}], capture_output=True, text=True,
                        timeout=300)
    assert cp.returncode == 0, cp.stderr[-3000:]
    r = json.loads([l for l in cp.stdout.splitlines() if l.startswith("RESULT ")][-1][len("RESULT "):])
    print(r)
    assert r["code"] == -2, r  # PWFA_ERR_CUDA
    assert "captur" in r["msg"].lower(), r  # the CUDA error string names the stream capture
    assert r["after_equal"], r
