"""Batched form: many instances of uneven grid sizes advanced by one launch
per phase for all of them (the fluid step, then Ampere fused with the next
step's Faraday), two steps at a time from a captured CUDA graph. Each node
runs the same per-node arithmetic as the single-instance kernels, so the
batched result equals the instance-by-instance one to rounding, and one
instance is checked against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2201_05473_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2201_05473_gb300 import lbm  # noqa: E402

MASK = lbm.FIELD_N | lbm.FIELD_UZ | lbm.FIELD_EZ | lbm.FIELD_BY | lbm.RAW_YEE


def close(fa, fb, i, tol=1e-6):
    """The batched kernels inline the same per-node functions, but are
    compiled into different kernels, so FP32 contraction may round
    differently: agreement to a few ulp per field, relative L2 (tol: 1e-6
    over tens of steps; longer runs let the differences grow)."""
    for c in range(fa.shape[0]):
        a, b = fa[c].double(), fb[c].double()
        den = max(float(b.norm()), 1e-30)
        err = float((a - b).norm()) / den
        print("instance", i, "field", c, "rel diff", err, "max abs", float((a - b).abs().max()))
        assert err <= tol, (i, c, err)


def scan(n, seed=0, scale=1):
    ws = W.batched_scan(n, seed=seed, steps=60)
    # small grids for the test: k in {4..7} -> 64x32x32 ... 112x56x56, ragged tiles
    out = []
    for i, w in enumerate(ws):
        k = 4 + (i % 4)
        out.append(w.replace(nx=8 * k + i % 3, ny=8 * k - i % 2, nz=16 * k))
    return out


@pytest.mark.parametrize("nsteps", [(10,), (7, 6, 1)])
def test_batched_equals_individual(nsteps):
    ws = scan(6)
    with lbm.Simulation(ws) as a, lbm.Simulation(ws) as b:
        b.set_batching(False)
        for n in nsteps:
            a.step(n)
            b.step(n)
        for i in range(len(ws)):
            fa = a.fields(MASK, instance=i)
            fb = b.fields(MASK, instance=i)
            close(fa, fb, i)
            assert a.steps_done(i) == sum(nsteps)


@pytest.mark.parametrize("storage,collision", [(W.BF16, W.REGULARIZED), (W.F16, W.REGULARIZED), (W.BF16, W.BGK),
                                               (W.F16, W.BGK)])
def test_batched_equals_individual_16bit(storage, collision):
    """The batched form with populations stored as 16-bit deviations, with
    the regularized collision (the stored-unit kernels) and with BGK (whose
    batched fluid phase parks lattices 2 and 3 in shared memory): against
    the same instances stepped one by one. A rounding difference of the FP32
    arithmetic between the two compilations can move a stored value by one
    16-bit unit; the fields agree to the bound below (GB300, both
    collisions: n identical, the other fields within 7.8e-9)."""
    ws = [w.replace(storage=storage, collision=collision) for w in scan(4)]
    with lbm.Simulation(ws) as a, lbm.Simulation(ws) as b:
        b.set_batching(False)
        a.step(12)
        b.step(12)
        for i in range(len(ws)):
            fa = a.fields(MASK, instance=i)
            fb = b.fields(MASK, instance=i)
            for c in range(fa.shape[0]):
                x, y = fa[c].double(), fb[c].double()
                err = float((x - y).norm()) / max(float(y.norm()), 1e-30)
                print("16-bit batched", storage, "instance", i, "field", c, "rel diff", err)
                assert err <= 1e-6, (i, c, err)


def test_batched_with_fused_field_steps_between():
    """Per-instance steps with the fused field step (Ampere with the next
    step's Faraday, which swaps the E buffers and leaves the next B computed)
    interleaved with batched pairs, against unbatched steps with separate
    field kernels: the batch table follows the swapped buffers and the
    batched Faraday phase recomputes the look-ahead B."""
    ws = scan(4, seed=5)
    with lbm.Simulation(ws) as a, lbm.Simulation(ws) as b:
        a.set_field_fusion(lbm.Simulation.FUSION_ON)
        b.set_field_fusion(lbm.Simulation.FUSION_OFF)
        b.set_batching(False)
        for n in (3, 4, 1, 2, 5):  # odd counts end on a fused per-instance step
            a.step(n)
            b.step(n)
        for i in range(len(ws)):
            close(a.fields(MASK, instance=i), b.fields(MASK, instance=i), i)
            assert a.steps_done(i) == 15


def test_batched_with_autotuned_shapes_and_state_changes():
    ws = scan(4, seed=3)
    with lbm.Simulation(ws) as a, lbm.Simulation(ws) as b:
        b.set_batching(False)
        a.autotune(2)
        shapes = [a.get_launch(i) for i in range(len(ws))]
        assert all(bx * by == 128 for bx, by in shapes)
        for i, sh in enumerate(shapes):
            b.set_launch(*sh, instance=i)
        a.step(4)
        b.step(4)
        # a state change invalidates the captured table
        f, E, B = a.get_state(instance=2)
        a.set_state(f, E, B, instance=2)
        a.step(6)
        b.step(6)
        for i in range(len(ws)):
            close(a.fields(MASK, instance=i), b.fields(MASK, instance=i), i)


def test_batched_instance_matches_oracle():
    ws = scan(3, seed=5)
    w = ws[1]
    o = oracle.Oracle(w.nx, w.ny, w.nz, w.dx, w.dt, w.tau, alpha=w.alpha, sigma_r=w.sigma_r,
                      sigma_z=w.sigma_z, z0=w.z0)
    with lbm.Simulation(ws) as a:
        a.step(60)
        g = a.fields(lbm.FIELD_N | lbm.FIELD_EZ | lbm.RAW_YEE, instance=1).cpu().numpy().astype(np.float64)
    o.step(60)
    E, _ = o.get_fields()
    n = o.moments()["n"]
    rel = lambda x, y: np.linalg.norm(x - y) / np.linalg.norm(y)
    assert rel(g[0], n) < 1e-5 and rel(g[1], E[2]) < 1e-5


def test_launch_counts_in_batched_mode():
    ws = scan(3)
    with lbm.Simulation(ws) as a:
        a.step(2)
        a.kernel_times()
        a.step(8)
        _, n = a.kernel_times()
        # one launch per phase per step for the whole batch: the fluid step
        # and the fused field step (the driver's step counters advance inside
        # the field launches)
        assert n == {"faraday": 0, "fluid": 8, "ampere": 8, "aux": 0, "adj_fluid": 0, "adj_field": 0}
        a.set_field_fusion(lbm.Simulation.FUSION_OFF)
        a.step(2)
        a.kernel_times()
        a.step(8)
        _, n = a.kernel_times()
        assert n == {"faraday": 8, "fluid": 8, "ampere": 8, "aux": 0, "adj_fluid": 0, "adj_field": 0}


def test_many_small_instances_batched():
    """A scan of 200 small instances (16x16x32 .. 24x24x48): batched and
    unbatched stepping agree, with fused and with separate field steps."""
    ws = [w.replace(nx=16 + 8 * (i % 2), ny=16 + 8 * (i % 2), nz=32 + 16 * (i % 2))
          for i, w in enumerate(W.batched_scan(200, seed=7, steps=20))]
    for fusion in (lbm.Simulation.FUSION_AUTO, lbm.Simulation.FUSION_OFF):
        with lbm.Simulation(ws) as a, lbm.Simulation(ws) as b:
            a.set_field_fusion(fusion)
            b.set_batching(False)
            a.step(12)
            b.step(12)
            for i in (0, 1, 57, 199):
                close(a.fields(MASK, instance=i), b.fields(MASK, instance=i), i)


def test_config4_scan_full_size():
    """The batched form on the 64-instance scan itself (grids 64x32x32 to
    256x128x128, 94 M nodes, n_b/n0 in [0.05, 2]), 500 steps in the
    benchmarked launch configuration: every instance stays finite with
    n > 0, and the smallest, a middle and the largest instance equal the
    same instance stepped alone (a single-instance handle), field by field:
    over 500 non-linear steps the few-ulp differences of the two
    compilations grow to ~1e-6 (GB300: at most 1.3e-6), held to the FP32
    parity bar 1e-5."""
    ws = W.batched_scan(64, seed=0)
    order = sorted(range(len(ws)), key=lambda i: ws[i].nodes)
    pick = [order[0], order[len(order) // 2], order[-1]]
    with lbm.Simulation(ws) as sb:
        sb.autotune(2)
        sb.step(500)
        for i in range(len(ws)):
            d = sb.diag(i)
            assert d[7] == 0 and d[5] > 0, (i, d)
        got = {i: sb.fields(MASK, instance=i) for i in pick}
    for i in pick:
        with lbm.Simulation(ws[i]) as s1:
            s1.step(500)
            close(got[i], s1.fields(MASK), i, tol=1e-5)
