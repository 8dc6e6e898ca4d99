#!/usr/bin/env python
"""Throughput of the fused LBM plasma-wakefield step on GB300.

Metric: GLUPS (1e9 node-steps per second; one node-step advances all four
D3Q19 lattices and the Yee fields of one node) and the fraction of the HBM
roofline, on the production workload: 512x256x256 nodes (z, y, x), dx = 0.05
c/omega_p, non-linear driver n_b/n0 = 1, sigma_z = 0.5, sigma_r = 0.3,
regularized collision, FP32. Synthetic inputs: the initial condition is the
paper's cold plasma at rest with a rigid Gaussian driver (no dataset exists).
The timed steps carry the non-linear wake: the driver starts inside the box
(z0 = 4 sigma_z) and an untimed prelude of steps forms the wake first.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 run under torchrun: every rank advances its own replica (the path
has no data exchange between instances), value = all ranks' node-steps /
max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2201_05473_gb300 import workloads as W  # noqa: E402

METRIC = "GLUPS & %HBM peak, fused fwd and adjoint step, FP32 vs BF16-store"
NOMINAL_HBM_GBS = 8000.0
FALLBACK_HBM_GBS = 6800.0
# Algorithmic bytes per node of the fused fluid kernel: the 76 populations
# read and written (FP32 608 B, 16-bit 304 B) and the fields E and B read
# (24 B). The node current it stores (12 B) and the second B level it reads
# (12 B) are not counted: the method need not store J.
FLUID_BYTES = {W.F32: 608 + 24, W.BF16: 304 + 24, W.F16: 304 + 24}
# Algorithmic bytes per node-step of the whole step: populations read+write
# plus E and B read+write.
STEP_BYTES = {W.F32: 608 + 48, W.BF16: 304 + 48, W.F16: 304 + 48}
# Adjoint: per reversed node-step the populations' adjoint read + written
# (608 B), the forward populations read (304 B), forward E and B read (24 B)
# and the fields' adjoints read + written (48 B), plus the forward step
# recomputed from the checkpoint (656 B).
ADJOINT_BYTES = 984 + 656
# What this build's reverse step moves per node instead: the recomputed
# forward step (fluid with its lattice sums 672 B, fused field step 60 B),
# transposed Ampere 48 B, transposed fluid step 696 B (the lattice sums in
# place of the forward populations), fused transposed averages + Faraday
# 72 B; without the recomputation (one-segment recording) the last three.
ADJOINT_BYTES_MOVED = 672 + 60 + 48 + 696 + 72
ADJOINT_BYTES_MOVED_NO_RECOMPUTE = 48 + 696 + 72
# Untimed steps before the warm-up: the driver, started inside the box at
# z0 = 4 sigma_z, forms the non-linear wake (min n ~0.4 after 300 steps).
PRELUDE_STEPS = 300
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "fluid_kernel_traffic.json")
KERNEL_SOURCES = ["paper_2201_05473_gb300/csrc/fluid.cu", "paper_2201_05473_gb300/csrc/fluid_node.cuh",
                  "paper_2201_05473_gb300/csrc/lbm_node.cuh", "paper_2201_05473_gb300/csrc/lbm_device.cuh"]
# the fused field kernel (Ampere with the next step's Faraday): 60 B/node
FIELD_TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ampere_faraday_kernel_traffic.json")
FIELD_SOURCES = ["paper_2201_05473_gb300/csrc/fields.cu", "paper_2201_05473_gb300/csrc/fields_fused.cuh",
                 "paper_2201_05473_gb300/csrc/fields_node.cuh", "paper_2201_05473_gb300/csrc/lbm_device.cuh"]
FIELD_BYTES = 60


def kernel_source_hash(sources=None) -> str:
    h = hashlib.sha256()
    for p in sources or KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            for k in ("hbm_gbs", "hbm_GBs", "hbm"):
                if k in d and isinstance(d[k], (int, float)):
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


def ncu_traffic(nodes, path=TRAFFIC_FILE, sources=None):
    """DRAM bytes per launch (the fluid kernel by default) from the committed
    ncu capture, scaled to the launch's node count, if the capture was taken
    on the current kernel source; else None."""
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except Exception:
        return None
    if d.get("source_sha") != kernel_source_hash(sources):
        return None
    return float(d["bytes_per_node"]) * nodes


class ClockSampler:
    """nvidia-smi clocks/throttle sampling while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        if not getattr(self, "lines", None):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            c = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(c[1]))
                mx.append(float(c[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, c[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate_over_ranks(ms, e2e_s, world, nodes, steps, dist=None, device="cpu"):
    """Whole-job rates of replicas: every rank advanced its own instance of
    `nodes` nodes for `steps` steps; the job time is the max over ranks.
    Returns (GLUPS, e2e GLUPS, max device ms)."""
    import torch
    t = torch.tensor([ms, e2e_s], dtype=torch.float64, device=device)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max, e2e_max = t.tolist()
    value = world * nodes * steps / (ms_max * 1e-3) / 1e9
    e2e = world * nodes * steps / e2e_max / 1e9
    return value, e2e, ms_max


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_config(w, storage: str) -> dict:
    """The keys naming the workload, shared by both arms' JSON lines."""
    return {"workload": w.name, "grid_zyx": [w.nz, w.ny, w.nx], "dx": w.dx, "dt": w.dt, "tau": w.tau,
            "driver": {"nb_over_n0": w.alpha, "sigma_r": w.sigma_r, "sigma_z": w.sigma_z, "z0": w.z0},
            "storage": storage}


def oracle_rate(target_seconds: float, shape=(128, 64, 64)):
    """Node-steps per second of the FP64 oracle, as it stands, on a (z, y, x)
    sub-box of the production workload with the same physics, stepped until
    ~target_seconds of wall time (OpenMP threads: OMP_NUM_THREADS)."""
    import oracle
    oracle.build()
    nz, ny, nx = shape
    w = W.production_timing().replace(nx=nx, ny=ny, nz=nz)
    o = oracle.Oracle(w.nx, w.ny, w.nz, w.dx, w.dt, w.tau, collision=w.collision, alpha=w.alpha,
                      sigma_r=w.sigma_r, sigma_z=w.sigma_z, z0=w.z0)
    o.step(1)
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < target_seconds and steps < 400:
        o.step(1)
        steps += 1
    dt = time.perf_counter() - t0
    o.close()
    return {"rate": w.nodes * steps / dt, "steps": steps, "seconds": dt,
            "box": f"{nz}x{ny}x{nx}"}


def cpu_baseline(target_seconds: float = 12.0):
    """The FP64 oracle on all host cores (a bounded sample of the production
    workload), plus the same oracle on one core in a child process."""
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    r = oracle_rate(target_seconds)
    out = {"value": r["rate"] / 1e9, "unit": "GLUPS", "cores": int(os.environ["OMP_NUM_THREADS"]),
           "kind": "oracle",
           "sample": f"FP64 oracle, {r['box']} sub-box of the 512x256x256 regularized workload, "
                     f"{r['steps']} steps in {r['seconds']:.1f} s"}
    # the 64x32x32 parity workload (200 steps of BGK with the linear driver) in full
    import oracle
    wp = W.parity_small()
    o = oracle.Oracle(wp.nx, wp.ny, wp.nz, wp.dx, wp.dt, wp.tau, collision=wp.collision, alpha=wp.alpha,
                      sigma_r=wp.sigma_r, sigma_z=wp.sigma_z, z0=wp.z0)
    t0 = time.perf_counter()
    o.step(wp.steps)
    tp = time.perf_counter() - t0
    o.close()
    out["parity_workload_full"] = {"value": wp.nodes * wp.steps / tp / 1e9, "unit": "GLUPS",
                                   "cores": int(os.environ["OMP_NUM_THREADS"]),
                                   "sample": f"FP64 oracle, {wp.nz}x{wp.ny}x{wp.nx}, all {wp.steps} steps "
                                             f"in {tp:.2f} s"}
    try:
        code = ("import sys, json; sys.path.insert(0, %r); import bench; "
                "print(json.dumps(bench.oracle_rate(4.0, (64, 32, 32))))" % ROOT)
        cp = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=180,
                            env=dict(os.environ, OMP_NUM_THREADS="1"))
        r1 = json.loads(cp.stdout.strip().splitlines()[-1])
        out["single_core"] = {"value": r1["rate"] / 1e9, "unit": "GLUPS", "cores": 1,
                              "sample": f"FP64 oracle, {r1['box']} sub-box, {r1['steps']} steps in "
                                        f"{r1['seconds']:.1f} s"}
    except Exception as e:  # the all-core figure stands on its own
        out["single_core"] = {"unavailable": str(e)[:200]}
    return out


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, each step a bounded
    sample (64x64x128 sub-box) of the production workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    import oracle
    oracle.build()
    w = W.production_timing().replace(nx=64, ny=64, nz=128)
    o = oracle.Oracle(w.nx, w.ny, w.nz, w.dx, w.dt, w.tau, collision=w.collision, alpha=w.alpha,
                      sigma_r=w.sigma_r, sigma_z=w.sigma_z, z0=w.z0)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    val = w.nodes * args.steps / dt / 1e9
    line = {"metric": METRIC, "value": val, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {**workload_config(W.production_timing(), "f32"),
                       "sample": f"{w.nz}x{w.ny}x{w.nx} sub-box per step", "parallelism": "host cores"},
            "cpu_baseline": {"value": val, "unit": "GLUPS", "cores": int(os.environ["OMP_NUM_THREADS"]),
                             "kind": "oracle", "sample": f"{w.nz}x{w.ny}x{w.nx} sub-box of the "
                                                          f"512x256x256 regularized workload, {args.steps} steps"},
            "e2e": {"value": val, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    from paper_2201_05473_gb300 import lbm

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    lbm.load()
    w = W.production_timing()
    if args.grid:
        nz, ny, nx = (int(v) for v in args.grid.lower().split("x"))
        w = w.replace(nx=nx, ny=ny, nz=nz, name=f"lbm-pwfa {nz}x{ny}x{nx} dx0.05 regularized")
    if args.storage != "f32":
        w = w.replace(storage={"bf16": W.BF16, "f16": W.F16}[args.storage])
    N = w.nodes
    stream = torch.cuda.Stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        sim = lbm.Simulation(w, stream=stream)
        sim.step(args.prelude)
        sim.step(args.warmup)
        if args.launch:
            # fixed shape, no autotuner trial launches (profiling captures)
            sim.set_launch(*(int(v) for v in args.launch.lower().split("x")))
        else:
            sim.autotune(3)
        launch_shape = sim.get_launch()
        fluid_variant = ["direct", "staged"][sim.get_fluid_variant()]
        sim.kernel_times()  # reset counters
        barrier()
        # ---- value: K steps, device-timed with CUDA events on the stream
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(dev) as clk:
            ev0.record(stream)
            sim.step(args.steps)
            ev1.record(stream)
            stream.synchronize()
        barrier()
        ms = ev0.elapsed_time(ev1)
        _, launches = sim.kernel_times()
        # ---- per-kernel roofline: the same K steps with event pairs per kernel
        sim.profile(True)
        sim.step(args.steps)
        kms, kl = sim.kernel_times()
        sim.profile(False)
        # ---- repeatability: five timed runs of 200 steps each (the driver
        # stays in the box), clocks sampled throughout
        repeat = None
        if not args.no_extra:
            per = []
            with ClockSampler(dev) as rclk:
                for _ in range(5):
                    ev0.record(stream)
                    sim.step(200)
                    ev1.record(stream)
                    stream.synchronize()
                    per.append(ev0.elapsed_time(ev1) / 200)
            med = statistics.median(per)
            repeat = {"reps": 5, "steps_each": 200, "median_ms_per_step": med, "min_ms_per_step": min(per),
                      "max_ms_per_step": max(per), "glups_median": N / med / 1e6, "clocks": rclk.summary()}
        diag = sim.diag(check=False)
        sim.close()
        del sim
        torch.cuda.synchronize()
        # ---- e2e through the C ABI with host buffers: create from host
        # params, K steps each followed by a device->host read of the FP64
        # diagnostics, destroy.
        e2e_s = float("nan")
        if not args.no_e2e:
            torch.cuda.empty_cache()
            barrier()
            host_diag = torch.zeros(8, dtype=torch.float64).pin_memory()
            t0 = time.perf_counter()
            sim = lbm.Simulation(w, stream=stream)
            hd = host_diag.numpy()
            for _ in range(args.steps):
                sim.step_diag(1, out=hd)
            sim.close()
            stream.synchronize()
            e2e_s = time.perf_counter() - t0
        # the production run as configured: 2000 steps from the initial
        # condition with the driver entering through the z = 0 wall
        full_run = None
        if not args.no_extra and not args.grid and w.storage == W.F32:
            torch.cuda.empty_cache()
            wf = W.production()
            sim = lbm.Simulation(wf, stream=stream)
            sim.set_launch(*launch_shape)
            barrier()
            with ClockSampler(dev) as fclk:
                ev0.record(stream)
                sim.step(wf.steps)
                ev1.record(stream)
                stream.synchronize()
            fms = ev0.elapsed_time(ev1)
            fd = sim.diag(check=False)
            sim.close()
            full_run = {"workload": wf.name, "steps": wf.steps, "seconds": fms / 1e3,
                        "value": wf.nodes * wf.steps / (fms * 1e-3) / 1e9, "unit": "GLUPS",
                        "pct_hbm_step": wf.nodes * wf.steps / (fms * 1e-3) * STEP_BYTES[W.F32] / (hbm_peak()[0] * 1e9),
                        "min_n_at_end": float(fd[5]), "nonfinite": float(fd[7]), "clocks": fclk.summary()}
        # the same path over 200 steps (the creation spread over more steps)
        e2e_200 = None
        if not args.no_e2e and not args.no_extra:
            torch.cuda.empty_cache()
            barrier()
            t0 = time.perf_counter()
            sim = lbm.Simulation(w, stream=stream)
            hd = host_diag.numpy()
            for _ in range(200):
                sim.step_diag(1, out=hd)
            sim.close()
            stream.synchronize()
            e2e_200 = {"value": world * N * 200 / (time.perf_counter() - t0) / 1e9, "unit": "GLUPS", "steps": 200}
        def time_variant(w2):
            """The production timing of another form of the workload: warm-up,
            autotune, K steps under CUDA events, then K profiled steps."""
            torch.cuda.empty_cache()
            sim = lbm.Simulation(w2, stream=stream)
            sim.step(args.prelude + args.warmup)
            sim.autotune(3)
            sim.kernel_times()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(args.steps)
            e1.record(stream)
            stream.synchronize()
            ms2 = e0.elapsed_time(e1)
            sim.kernel_times()  # reset the counters before the profiled pass
            sim.profile(True)
            sim.step(args.steps)
            k2, l2 = sim.kernel_times()
            sim.profile(False)
            d2 = sim.diag(check=False)
            sim.close()
            return ms2, {k: k2[k] / max(l2[k], 1) for k in k2 if l2[k]}, d2

        glups_main = N * args.steps / (ms * 1e-3) / 1e9
        # ---- reduced-precision storage: same workload, BF16 / FP16 deviations
        storage_lines = {}
        if not args.no_extra and args.only in ("", "storage"):
            for name, st in (("bf16", W.BF16), ("f16", W.F16)):
                ms2, kpl, d2 = time_variant(w.replace(storage=st))
                glups = N * args.steps / (ms2 * 1e-3) / 1e9
                storage_lines[name] = {
                    "value": glups, "unit": "GLUPS", "vs_f32": glups / glups_main,
                    "ms_per_step": ms2 / args.steps, "bytes_per_node_step": STEP_BYTES[st],
                    "pct_hbm_step": glups * 1e9 * STEP_BYTES[st] / (hbm_peak()[0] * 1e9),
                    "fluid_kernel_GBs": FLUID_BYTES[st] * N / (kpl["fluid"] * 1e-3) / 1e9,
                    "kernel_ms_per_step": kpl, "finite": bool(d2[7] == 0)}
        # ---- the same production step with the BGK collision (Eq. 7)
        bgk_line = None
        if not args.no_extra and args.only in ("", "bgk") and w.collision != W.BGK:
            ms2, kpl, d2 = time_variant(w.replace(collision=W.BGK))
            glups = N * args.steps / (ms2 * 1e-3) / 1e9
            bgk_line = {
                "value": glups, "unit": "GLUPS", "vs_regularized": glups / glups_main,
                "ms_per_step": ms2 / args.steps,
                "pct_hbm_step": glups * 1e9 * STEP_BYTES[w.storage] / (hbm_peak()[0] * 1e9),
                "fluid_kernel_GBs": FLUID_BYTES[w.storage] * N / (kpl["fluid"] * 1e-3) / 1e9,
                "kernel_ms_per_step": kpl, "finite": bool(d2[7] == 0)}
        # ---- moving window: the same workload with the box following the
        # driver from the first step (one plane every dx / dt = 5.67 steps)
        window_line = None
        if not args.no_extra and args.only in ("", "window"):
            torch.cuda.empty_cache()
            ww = w.replace(moving_window=1, window_z=w.z0)
            sim = lbm.Simulation(ww, stream=stream)
            sim.step(args.warmup)
            sim.autotune(3)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            p0 = sim.window_planes()
            e0.record(stream)
            sim.step(args.steps)
            e1.record(stream)
            stream.synchronize()
            msw = e0.elapsed_time(e1)
            moved = sim.window_planes() - p0
            sim.kernel_times()
            sim.profile(True)
            sim.step(args.steps)
            kw_, lw_ = sim.kernel_times()
            sim.profile(False)
            dw = sim.diag(check=False)
            sim.close()
            window_line = {"value": N * args.steps / (msw * 1e-3) / 1e9, "unit": "GLUPS",
                           "vs_fixed_box": ms / msw, "planes_moved": moved, "steps": args.steps,
                           "move_kernel_ms": kw_["aux"] / max(lw_["aux"], 1),
                           "fluid_kernel_ms": kw_["fluid"] / max(lw_["fluid"], 1),
                           "note": "box follows the driver; each move: E and B moved by a kernel "
                                   "(24 B/node), populations read one plane up inside the fluid kernel",
                           "finite": bool(dw[7] == 0)}
        # ---- PIC driver (Eq. 1): the production step with the bunch as
        # 2e5 macro-electrons (the paper's particle count, gamma = 5000)
        pic_line = None
        if not args.no_extra and args.only in ("", "pic"):
            torch.cuda.empty_cache()
            wp = w.replace(driver=1)
            npart = 200000
            xp, pwt = W.bunch_particles(npart, wp.alpha, wp.sigma_r, wp.sigma_z, wp.z0, wp.dt, wp.nx, wp.ny, wp.dx)
            sp = lbm.Simulation(wp, stream=stream)
            sp.set_particles(xp, pwt)
            sp.set_launch(*launch_shape)
            sp.step(args.warmup)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sp.step(args.steps)
            e1.record(stream)
            stream.synchronize()
            msp = e0.elapsed_time(e1)
            sp.kernel_times()
            sp.profile(True)
            sp.step(args.steps)
            kp, lp = sp.kernel_times()
            sp.profile(False)
            dp_ = sp.diag(check=False)
            sp.close()
            pic_line = {"value": N * args.steps / (msp * 1e-3) / 1e9, "unit": "GLUPS", "particles": npart,
                        "vs_rigid_driver": ms / msp, "particle_kernel_ms": kp["aux"] / max(lp["aux"], 1),
                        "note": "Boris push + Esirkepov deposit (FP32 atomics) after the fluid kernel",
                        "finite": bool(dp_[7] == 0)}
        # ---- the paper's own geometry: 2D-axisymmetric (z, r), 2400 x 400
        # cells at 0.25 um, Q = 0.1 (context: the paper's LBM routine ran
        # 2.0 M cell-steps/s on a Xeon E5-2695, Table I)
        axi_line = None
        if not args.no_extra and args.only in ("", "axisymmetric"):
            torch.cuda.empty_cache()
            wa_ = W.axisymmetric_paper(0.1)
            sa = lbm.AxiSimulation(wa_, stream=stream)
            sa.step(args.warmup)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sa.step(args.steps)
            e1.record(stream)
            stream.synchronize()
            msa = e0.elapsed_time(e1)
            sa.kernel_times()
            sa.profile(True)
            sa.step(args.steps)
            ka, la = sa.kernel_times()
            sa.profile(False)
            ga = sa.fields()
            finite = bool(torch.isfinite(ga).all().item())
            sa.close()
            rate = wa_.nodes * args.steps / (msa * 1e-3)
            axi_line = {"value": rate / 1e9, "unit": "GLUPS", "grid_zr": [wa_.nz, wa_.nr], "steps": args.steps,
                        "note": "three D2Q9 lattices + cylindrical Yee per node-step",
                        "kernel_ms_per_step": {k: ka[k] / max(la[k], 1) for k in ka if la[k]},
                        "vs_paper_cpu_lbm_routine": rate / 2.0e6, "finite": finite}
        # ---- adjoint: the differentiable form (256x128x128, 500 steps,
        # checkpoints every 23 steps, witness loss)
        adjoint_line = None
        if not args.no_extra and args.only in ("", "adjoint"):
            torch.cuda.empty_cache()
            wa = W.differentiable().replace(profile=__import__("numpy").ones(64), profile_rmax=128 * 0.2 / 2)
            Ta = args.adjoint_steps
            sim = lbm.Simulation(wa, stream=stream)
            barrier()
            t0 = time.perf_counter()
            sim.record(Ta, 0)
            stream.synchronize()
            t_rec = time.perf_counter() - t0
            L = sim.witness_loss()
            sim.kernel_times()
            t0 = time.perf_counter()
            g = sim.adjoint_step(None)  # the built-in witness loss over the recorded run
            t_adj = time.perf_counter() - t0
            _, la = sim.kernel_times()
            # the same sweep with an event pair around every launch
            sim.profile(True)
            sim.adjoint_step(None)
            ka, la2 = sim.kernel_times()
            sim.profile(False)
            sim.close()
            # one segment (ckpt_every = T): the recording leaves every step's
            # lattice sums, E and B in the segment storage (about 40 B per
            # node-step), and the sweep recomputes nothing
            single = None
            torch.cuda.empty_cache()
            try:
                sim = lbm.Simulation(wa, stream=stream)
                t0 = time.perf_counter()
                sim.record(Ta, Ta)
                stream.synchronize()
                t_rec1 = time.perf_counter() - t0
                sim.kernel_times()
                t0 = time.perf_counter()
                g1 = sim.adjoint_step(None)
                t_adj1 = time.perf_counter() - t0
                k1, l1 = sim.kernel_times()
                sim.close()
                g1s = wa.nodes * Ta / t_adj1 / 1e9
                single = {"value": g1s, "unit": "GLUPS", "ckpt_every": Ta,
                          "bytes_per_node_step_moved": ADJOINT_BYTES_MOVED_NO_RECOMPUTE,
                          "pct_hbm_of_bytes_moved": g1s * ADJOINT_BYTES_MOVED_NO_RECOMPUTE / hbm_peak()[0],
                          "record_glups": wa.nodes * Ta / t_rec1 / 1e9,
                          "record_plus_adjoint_glups": wa.nodes * Ta / (t_rec1 + t_adj1) / 1e9,
                          "launches_per_reversed_step": {k: l1[k] / Ta for k in l1 if l1[k]},
                          "grad_alpha_sigr_sigz": [float(v) for v in g1[:3]],
                          "note": "one segment of T steps kept from the recording (checkpoints of the "
                                  "start and end states only); the sweep runs no forward step"}
            except lbm.LBMError as e:
                single = {"unavailable": str(e)}
            adj_glups = wa.nodes * Ta / t_adj / 1e9
            adjoint_line = {"value": adj_glups, "unit": "GLUPS",
                            "note": "reverse sweep incl. the recompute of every segment but the last (which the "
                                    "recording leaves in the segment storage), wall time of pwfa_lbm_adjoint_step "
                                    "(NULL seed: the built-in witness loss); node-steps of the adjoint / time",
                            "bytes_per_node_step": ADJOINT_BYTES,
                            "pct_hbm": adj_glups * 1e9 * ADJOINT_BYTES / (hbm_peak()[0] * 1e9),
                            "bytes_per_node_step_moved": ADJOINT_BYTES_MOVED,
                            "pct_hbm_of_bytes_moved": adj_glups * ADJOINT_BYTES_MOVED / hbm_peak()[0],
                            "record_glups": wa.nodes * Ta / t_rec / 1e9,
                            "record_plus_adjoint_glups": wa.nodes * Ta / (t_rec + t_adj) / 1e9,
                            "grid_zyx": [wa.nz, wa.ny, wa.nx],
                            "steps": Ta, "ckpt_every": int(__import__("math").ceil(Ta ** 0.5)),
                            "witness_loss": L,
                            "kernel_ms_per_reversed_step": {k: ka[k] / Ta for k in ka if la2[k]},
                            "launches_per_reversed_step": {k: la[k] / Ta for k in la if la[k]},
                            "grad_alpha_sigr_sigz": [float(v) for v in g[:3]],
                            "single_segment": single}
        # ---- batched form: 64 instances of uneven size, one launch per phase
        # for all of them, two steps per graph replay, against the same
        # instances stepped one after another; then a scan of 256 small
        # instances, where one instance alone cannot fill the GPU
        batch_line = None
        if not args.no_extra and args.only in ("", "batched"):
            def time_batch(ws, K):
                torch.cuda.empty_cache()
                tot = sum(x.nodes for x in ws)
                sb = lbm.Simulation(ws, stream=stream)
                sb.step(args.warmup + (args.warmup % 2))
                sb.autotune(2)
                sb.step(2)
                sb.kernel_times()
                barrier()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sb.step(K)
                e1.record(stream)
                stream.synchronize()
                msb = e0.elapsed_time(e1)
                _, lb = sb.kernel_times()
                # per-phase device times of the same batched steps
                sb.profile(True)
                sb.step(K)
                kb, lk = sb.kernel_times()
                sb.profile(False)
                sb.set_batching(False)
                sb.step(2)
                e0.record(stream)
                sb.step(K)
                e1.record(stream)
                stream.synchronize()
                msu = e0.elapsed_time(e1)
                db = [sb.diag(i, check=False)[7] for i in range(len(ws))]
                sb.close()
                return {"value": tot * K / (msb * 1e-3) / 1e9, "unit": "GLUPS", "instances": len(ws),
                        "nodes_total": tot, "steps": K, "ms_per_step": msb / K,
                        "launches_per_step": sum(lb.values()) / K,
                        "kernel_ms_per_step": {k: kb[k] / K for k in kb if lk[k]},
                        "unbatched_glups": tot * K / (msu * 1e-3) / 1e9, "speedup_vs_unbatched": msu / msb,
                        "nonfinite_instances": int(sum(1 for v in db if v > 0))}
            Kb = args.steps - args.steps % 2
            ws = W.batched_scan(args.batch_instances, seed=0)
            batch_line = time_batch(ws, Kb)
            batch_line["grids_zyx"] = sorted({(x.nz, x.ny, x.nx) for x in ws})
            batch_line["vs_single_instance_bgk"] = (batch_line["value"] / bgk_line["value"]) if bgk_line else None
            batch_line["small_instances"] = time_batch(W.small_scan(256, seed=0), max(Kb, 20))
            batch_line["small_instances"]["grid_zyx"] = [32, 16, 16]
    value, e2e_val, ms_max = aggregate_over_ranks(ms, e2e_s, world, N, args.steps, dist, "cuda")
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peak, peak_kind = hbm_peak()
    fluid_ms = kms["fluid"] / max(kl["fluid"], 1)
    fluid_bytes = FLUID_BYTES[w.storage] * N
    achieved = fluid_bytes / (fluid_ms * 1e-3) / 1e9
    step_bytes = STEP_BYTES[w.storage]
    step_achieved = value / world * step_bytes  # GB/s of one GPU over the whole step
    line = {
        "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
        "config": {**workload_config(w, args.storage),
                   "prelude_steps": args.prelude,
                   "l2": "inputs larger than L2 (populations %.1f GB)" % (2 * 76 * (4 if w.storage == W.F32 else 2) * N / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "fluid_block": list(launch_shape), "fluid_variant": fluid_variant},
        "pct_hbm_step": {"of_" + peak_kind: value / world * 1e9 * step_bytes / (peak * 1e9),
                         "of_nominal_8000": value / world * 1e9 * step_bytes / (NOMINAL_HBM_GBS * 1e9),
                         "bytes_per_node_step": step_bytes},
        "roofline": {"bound": "hbm", "kernel": "fluid", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "traffic": ncu_traffic(N), "algorithmic_bytes_per_launch": fluid_bytes,
                     "bytes_per_node": FLUID_BYTES[w.storage], "avg_launch_ms": fluid_ms,
                     "step": {"bytes_per_node_step": step_bytes, "achieved": step_achieved,
                              "frac": step_achieved / peak, "ms": ms_max / args.steps}},
        "roofline_fields": ({"bound": "hbm", "kernel": "ampere_faraday",
                             "achieved": FIELD_BYTES * N / (kms["ampere"] / kl["ampere"] * 1e-3) / 1e9,
                             "peak": peak, "unit": "GB/s",
                             "frac": FIELD_BYTES * N / (kms["ampere"] / kl["ampere"] * 1e-3) / 1e9 / peak,
                             "peak_kind": peak_kind,
                             "traffic": ncu_traffic(N, FIELD_TRAFFIC_FILE, FIELD_SOURCES),
                             "algorithmic_bytes_per_launch": FIELD_BYTES * N, "bytes_per_node": FIELD_BYTES,
                             "avg_launch_ms": kms["ampere"] / kl["ampere"]}
                            if kl.get("ampere") and kl.get("faraday", 0) == 0 else None),
        "kernel_ms_per_step": {k: kms[k] / max(kl[k], 1) for k in kms if kl[k]},
        "field_step": ("ampere fused with the next step's faraday (one launch)" if kl.get("faraday", 0) == 0
                       else "separate faraday and ampere launches"),
        "gpu_launches": int(sum(launches.values())),
        "e2e": {"value": e2e_val, "unit": "GLUPS",
                "h2d_bytes_per_step": lbm.ctypes.sizeof(lbm.Params) / args.steps,
                "d2h_bytes_per_step": 64,
                "note": "create from host params, then per step pwfa_lbm_step_diag (step + fused FP64 "
                        "diagnostics, D2H into pinned host memory), destroy",
                "steps_200": e2e_200},
        "storage_forms": storage_lines or None,
        "bgk": bgk_line,
        "adjoint": adjoint_line,
        "batched": batch_line,
        "moving_window": window_line,
        "axisymmetric": axi_line,
        "pic_driver": pic_line,
        "clocks": clk.summary(),
        "repeat": repeat,
        "full_run": full_run,
        "diag_after": {"sum_n": diag[0], "min_n": diag[5], "max_beta": diag[6], "nonfinite": diag[7]},
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def precision_report(args):
    """Precision form: config-1 physics on 256x128x128, populations stored in
    FP32, BF16 and FP16 (deviations), errors of n, beta and E_z against the
    FP64 oracle every 100 steps up to 1000. One JSON line."""
    import numpy as np
    import torch
    from paper_2201_05473_gb300 import lbm
    import oracle
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    oracle.build()
    base = W.precision_form(W.F32)
    steps = args.steps if args.steps != 200 else base.steps
    o = oracle.Oracle(base.nx, base.ny, base.nz, base.dx, base.dt, base.tau, alpha=base.alpha,
                      sigma_r=base.sigma_r, sigma_z=base.sigma_z, z0=base.z0)
    sims = {name: lbm.Simulation(base.replace(storage=st)) for name, st in
            (("f32", W.F32), ("bf16", W.BF16), ("f16", W.F16))}
    m = lbm.FIELD_N | lbm.FIELD_UX | lbm.FIELD_UY | lbm.FIELD_UZ | lbm.FIELD_EZ | lbm.RAW_YEE

    def rel(a, b):
        return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))

    table = {name: [] for name in sims}
    for s0 in range(100, steps + 1, 100):
        o.step(100)
        mo = o.moments()
        E, _ = o.get_fields()
        for name, sim in sims.items():
            sim.step(100)
            g = sim.fields(m).cpu().numpy().astype(np.float64)
            table[name].append({"step": s0, "n": rel(g[0], mo["n"]), "beta": rel(g[1:4], mo["beta"]),
                                "Ez": rel(g[4], E[2])})
    for sim in sims.values():
        sim.close()
    print(json.dumps({"report": "precision", "workload": base.name, "grid_zyx": [base.nz, base.ny, base.nx],
                      "errors_vs_fp64_oracle": table}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--prelude", type=int, default=PRELUDE_STEPS,
                    help="untimed steps before the warm-up that form the wake")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "f16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--grid", default="", help="override the grid as ZxYxX (profiling captures)")
    ap.add_argument("--launch", default="", help="fixed fluid block shape BXxBY instead of the autotuner "
                                                 "(profiling captures)")
    ap.add_argument("--no-extra", action="store_true", help="skip the BF16/FP16 and adjoint lines")
    ap.add_argument("--adjoint-steps", type=int, default=500)
    ap.add_argument("--batch-instances", type=int, default=64,
                    help="instances of the batched parameter scan (fewer: a small case for profiling captures)")
    ap.add_argument("--only", default="", choices=["", "storage", "bgk", "adjoint", "batched", "window", "axisymmetric", "pic"],
                    help="with a small --steps: run the main pass and one extra section (profiling captures)")
    ap.add_argument("--report", default="", choices=["", "precision"],
                    help="precision: error table of BF16/FP16/FP32 storage against the oracle")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.report == "precision":
        precision_report(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
