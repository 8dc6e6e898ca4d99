"""Handles on their own CUDA streams: two instances stepped concurrently on
two streams, and one handle moved to another stream with work in flight,
give the states of plain single-stream runs bit for bit."""
import numpy as np
import pytest

from paper_2201_05473_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2201_05473_gb300 import lbm  # noqa: E402


def state(sim):
    f, E, B = sim.get_state()
    return f.cpu().numpy(), E.cpu().numpy(), B.cpu().numpy()


def same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def reference(w, steps):
    with lbm.Simulation(w) as sim:
        sim.step(steps)
        return state(sim)


def test_two_handles_on_two_streams():
    wa = W.parity_small().replace(nx=48, ny=32, nz=96, z0=-1.0, alpha=0.5, collision=W.REGULARIZED)
    wb = W.parity_small().replace(nx=32, ny=32, nz=64, z0=-0.5, alpha=0.3)
    ra, rb = reference(wa, 60), reference(wb, 60)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    with lbm.Simulation(wa, stream=sa) as a, lbm.Simulation(wb, stream=sb) as b:
        for _ in range(6):  # interleaved, no host wait in between
            a.step(10)
            b.step(10)
        assert same(state(a), ra)
        assert same(state(b), rb)


def test_stream_switch_with_work_in_flight():
    w = W.parity_small().replace(nx=48, ny=32, nz=96, z0=-1.0, alpha=0.5, collision=W.REGULARIZED)
    ref = reference(w, 40)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with lbm.Simulation(w, stream=s1) as sim:
        sim.set_field_fusion(lbm.Simulation.FUSION_ON)
        sim.step(20)          # queued on s1
        sim.set_stream(s2)    # s2 waits for s1's work
        sim.step(20)
        assert same(state(sim), ref)


def test_handles_on_concurrent_host_threads():
    """Four host threads, each creating, stepping and destroying its own
    handle on its own stream at the same time (the binding releases the
    interpreter lock in every library call): each result equals a
    single-threaded run bit for bit, and errors are reported per thread."""
    import threading

    works = [W.parity_small().replace(nx=32, ny=32, nz=48 + 16 * i, z0=-1.0 + 0.2 * i, alpha=0.3 + 0.1 * i)
             for i in range(4)]
    refs = [reference(w, 30) for w in works]
    out, errs = [None] * 4, [None] * 4

    def run(i):
        try:
            s = torch.cuda.Stream()
            with lbm.Simulation(works[i], stream=s) as sim:
                for _ in range(3):
                    sim.step(10)
                out[i] = state(sim)
            # a failing call on this thread reports this thread's error
            try:
                with lbm.Simulation(works[i].replace(tau=0.4), stream=s):
                    pass
            except lbm.LBMError as e:
                errs[i] = e.code
        except Exception as e:  # pragma: no cover - surfaced by the asserts below
            errs[i] = repr(e)

    ts = [threading.Thread(target=run, args=(i,)) for i in range(4)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert errs == [-1] * 4, errs  # tau <= 1/2: PWFA_ERR_PARAM on every thread
    for i in range(4):
        assert same(out[i], refs[i]), i
