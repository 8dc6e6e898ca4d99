"""GPU adjoint against the oracle's forward-mode (dual-number) derivatives.

The adjoint gives the full gradient g of L = <seed, E(T)> with respect to
theta = (alpha, sigma_r, sigma_z, profile...); the oracle gives directional
derivatives dL.v for a few directions v in FP64, independently of the
reverse sweep. Bar: relative error <= 1e-4.
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

TOL = 1e-4


def oracle_dirderiv(w, steps, dirs, seed):
    oracle.build()
    E, dE = oracle.tangent_run(steps, dirs, w.nx, w.ny, w.nz, w.dx, w.dt, w.tau, collision=w.collision,
                               boundary=w.boundary, couple=w.couple, n0=w.n0, profile=w.profile,
                               profile_rmax=w.profile_rmax, alpha=w.alpha, sigma_r=w.sigma_r,
                               sigma_z=w.sigma_z, z0=w.z0, n_floor=w.n_floor)
    L = float((seed * E).sum())
    dL = np.array([(seed * dE[k]).sum() for k in range(dirs.shape[0])])
    return L, dL


def directions(np_prof, seed=11):
    rng = np.random.default_rng(seed)
    n = 3 + np_prof
    d = np.zeros((4, n))
    d[0, 0] = d[1, 1] = d[2, 2] = 1.0
    if np_prof:
        d[3, 3:] = rng.standard_normal(np_prof)
    else:
        d[3, :3] = rng.standard_normal(3)
    return d


def run_case(w, steps, ckpt, seed_arr, tol=TOL):
    dirs = directions(0 if w.profile is None else len(w.profile))
    L_o, dL_o = oracle_dirderiv(w, steps, dirs, seed_arr)
    with lbm.Simulation(w) as sim:
        sim.record(steps, ckpt)
        E = sim.fields(lbm.FIELD_EX | lbm.FIELD_EY | lbm.FIELD_EZ | lbm.RAW_YEE).cpu().numpy().astype(np.float64)
        L_g = float((seed_arr * E).sum())
        g = sim.adjoint_step(seed_arr.astype(np.float32))
        assert sim.steps_done() == steps
    dL_g = dirs @ g
    # the loss itself is an FP32 forward value (a local mean of E_z): 1e-4
    assert abs(L_g - L_o) <= 1e-4 * abs(L_o) + 1e-12, (L_g, L_o)
    err = np.abs(dL_g - dL_o) / np.maximum(np.abs(dL_o), 1e-30)
    print("adjoint vs tangent:", dL_g, dL_o, err)
    assert np.all(err <= tol), (dL_g, dL_o, err)
    return g


def random_seed(w, rng):
    s = rng.standard_normal((3, w.nz, w.ny, w.nx))
    return s


@pytest.mark.parametrize("collision", [W.BGK, W.REGULARIZED])
def test_adjoint_periodic_random_functional(collision):
    w = W.parity_small().replace(nx=12, ny=10, nz=16, boundary=W.PERIODIC, collision=collision, alpha=0.4,
                                 sigma_r=0.6, sigma_z=0.5, z0=0.8, tau=0.7)
    rng = np.random.default_rng(2)
    run_case(w, 30, 7, random_seed(w, rng))


@pytest.mark.parametrize("collision", [W.BGK, W.REGULARIZED])
def test_adjoint_open_with_profile(collision):
    prof = np.linspace(1.0, 0.7, 8)
    w = W.parity_small().replace(nx=14, ny=12, nz=24, collision=collision, alpha=0.5, sigma_r=0.5,
                                 sigma_z=0.5, z0=-1.0, tau=0.6, profile=prof, profile_rmax=1.2)
    rng = np.random.default_rng(3)
    run_case(w, 40, 6, random_seed(w, rng))


def test_adjoint_with_vacuum_region():
    """The adjoint through the density floor: a plasma column in vacuum (the
    profile falls to zero inside the box), so the reverse step takes the
    derivative of the floored branch p = A / n_floor at the thin and empty
    nodes; the profile gradient includes the points that are zero."""
    prof = np.array([1.0, 1.0, 0.7, 0.3, 0.0, 0.0, 0.0, 0.0])
    w = W.parity_small().replace(nx=16, ny=16, nz=24, alpha=0.5, sigma_r=0.5, sigma_z=0.5, z0=-1.0, tau=0.6,
                                 profile=prof, profile_rmax=1.6)
    rng = np.random.default_rng(13)
    run_case(w, 40, 7, random_seed(w, rng))


def test_adjoint_witness_loss_config_copy():
    """Differentiable form on its 64x32x32 copy: n_b/n0 = 0.5, 500 steps,
    checkpoints every 23 steps, loss -mean E_z on the witness slab 1.5
    lambda_p behind the driver, 64-point radial profile = 1."""
    w = W.parity_small().replace(alpha=0.5, profile=np.ones(64), profile_rmax=min(32, 32) * 0.2 / 2)
    steps = 500
    k, mask = W.witness_slab(w, steps)
    seed = np.zeros((3, w.nz, w.ny, w.nx))
    seed[2, k][mask] = -1.0 / mask.sum()
    g = run_case(w, steps, 23, seed)
    assert np.all(np.isfinite(g))


def test_autograd_function_matches_adjoint():
    from paper_2201_05473_gb300.autograd import witness_loss
    w = W.parity_small().replace(nx=16, ny=16, nz=40, alpha=0.5, z0=-1.0, profile=np.ones(8),
                                 profile_rmax=1.5)
    steps = 120
    theta = torch.tensor([0.5, 0.5, 0.5], dtype=torch.float64, requires_grad=True)
    prof = torch.ones(8, dtype=torch.float64, requires_grad=True)
    L = witness_loss(theta, prof, w, steps)
    L.backward()
    # same gradient through the raw ABI
    k, mask = W.witness_slab(w, steps)
    seed = np.zeros((3, w.nz, w.ny, w.nx), dtype=np.float32)
    seed[2, k][mask] = -1.0 / mask.sum()
    with lbm.Simulation(w) as sim:
        sim.record(steps)
        g = sim.adjoint_step(seed)
    assert np.allclose(theta.grad.numpy(), g[:3], rtol=1e-6, atol=1e-12)
    assert np.allclose(prof.grad.numpy(), g[3:], rtol=1e-6, atol=1e-12)


def test_adjoint_against_fp32_finite_differences():
    """Sanity check: central differences of the FP32 forward (h = 1e-3) agree
    with the adjoint to ~1e-2 (FP32 noise ~ eps |L| / h)."""
    w = W.parity_small().replace(nx=16, ny=16, nz=40, alpha=0.5, z0=-1.0)
    steps = 120
    k, mask = W.witness_slab(w, steps)

    def loss(alpha):
        with lbm.Simulation(w.replace(alpha=alpha)) as sim:
            sim.step(steps)
            ez = sim.fields(lbm.FIELD_EZ | lbm.RAW_YEE)[0, k].cpu().numpy().astype(np.float64)
        return -ez[mask].mean()

    seed = np.zeros((3, w.nz, w.ny, w.nx), dtype=np.float32)
    seed[2, k][mask] = -1.0 / mask.sum()
    with lbm.Simulation(w) as sim:
        sim.record(steps)
        g = sim.adjoint_step(seed)
    h = 1e-3
    fd = (loss(0.5 + h) - loss(0.5 - h)) / (2 * h)
    assert abs(fd - g[0]) <= 2e-2 * abs(g[0]), (fd, g[0])


def test_adjoint_requires_recording():
    w = W.parity_small().replace(nz=16)
    with lbm.Simulation(w) as sim:
        with pytest.raises(lbm.LBMError):
            sim.adjoint_step(np.zeros((3, w.nz, w.ny, w.nx), dtype=np.float32))


def test_builtin_witness_loss_and_null_seed():
    """The library's built-in objective: pwfa_lbm_witness_loss equals
    -mean(E_z) over the witness slab of the exported fields, and the adjoint
    with a NULL seed (the built-in loss) recording its own forward run
    (nsteps given) equals record + adjoint with the explicit slab seed."""
    w = W.parity_small().replace(nx=16, ny=16, nz=40, alpha=0.5, z0=-1.0, profile=np.ones(8),
                                 profile_rmax=1.5)
    steps = 120
    k, mask = W.witness_slab(w, steps)
    seed = np.zeros((3, w.nz, w.ny, w.nx), dtype=np.float32)
    seed[2, k][mask] = -1.0 / mask.sum()
    with lbm.Simulation(w) as sim:
        sim.record(steps, 11)
        ez = sim.fields(lbm.FIELD_EZ | lbm.RAW_YEE)[0, k].cpu().numpy().astype(np.float64)
        L = sim.witness_loss()
        assert abs(L - (-ez[mask].mean())) <= 1e-12 * max(abs(L), 1e-30) + 1e-15, (L, -ez[mask].mean())
        g_seed = sim.adjoint_step(seed)
    with lbm.Simulation(w) as sim:
        g_null = sim.adjoint_step(None, nsteps=steps, ckpt_every=11)
        assert sim.steps_done() == steps
        # the recording is kept: a second call with nsteps = 0 reuses it
        g_again = sim.adjoint_step(None)
    # the same sweep; the FP64 atomic sums of the driver terms may add in
    # another order
    assert np.allclose(g_null, g_seed, rtol=1e-12, atol=1e-15), (g_null, g_seed)
    assert np.allclose(g_again, g_seed, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("boundary,collision", [(W.OPEN, W.REGULARIZED), (W.OPEN, W.BGK), (W.PERIODIC, W.BGK)])
def test_fused_faces_edges_equal_separate(boundary, collision):
    """The transposed node averages and Faraday (R3, R4) in one z-marching
    kernel against the two separate kernels (field fusion off), on a grid
    spanning several 31 x 7 x 16 tiles with ragged ends: the same
    arithmetic, so the same adjoint state; the gradients then differ only
    by the order of the FP64 atomic sums."""
    prof = np.linspace(1.0, 0.6, 8) if boundary == W.OPEN else None
    w = W.parity_small().replace(nx=70, ny=23, nz=37, boundary=boundary, collision=collision, alpha=0.5,
                                 z0=-1.0, tau=0.6, profile=prof, profile_rmax=3.0)
    seed = random_seed(w, np.random.default_rng(5)).astype(np.float32)
    grads = []
    for mode in (lbm.Simulation.FUSION_ON, lbm.Simulation.FUSION_OFF):
        with lbm.Simulation(w) as sim:
            sim.set_field_fusion(mode)
            sim.record(40, 7)
            grads.append(sim.adjoint_step(seed))
    assert np.all(np.isfinite(grads[0])) and np.any(grads[0] != 0.0)
    assert np.allclose(grads[0], grads[1], rtol=1e-12, atol=1e-15), (grads[0], grads[1])


def test_record_keeps_last_segment_and_single_segment():
    """The recording runs its last segment into the segment slots, so the
    sweep reverses that segment without recomputing it; with one segment
    (ckpt_every >= nsteps) the sweep recomputes nothing. The gradient, and
    the state the instance ends in, must not depend on it: the same as a
    sweep that recomputes every segment (the second call on a recording)
    and as a recording with several segments, up to the order of the FP64
    atomic sums."""
    w = W.parity_small().replace(nx=20, ny=16, nz=40, alpha=0.5, z0=-1.0, tau=0.6, collision=W.REGULARIZED,
                                 profile=np.linspace(1.0, 0.7, 8), profile_rmax=2.0)
    steps = 60
    seed = random_seed(w, np.random.default_rng(9)).astype(np.float32)
    mask = lbm.FIELD_N | lbm.FIELD_EZ | lbm.FIELD_BX
    out = {}
    for ck in (7, steps):
        with lbm.Simulation(w) as sim:
            sim.record(steps, ck)
            after_record = sim.fields(mask).cpu().numpy()
            g_first = sim.adjoint_step(seed)  # last segment taken from the recording
            after_adjoint = sim.fields(mask).cpu().numpy()
            g_again = sim.adjoint_step(seed)  # every segment recomputed
            assert sim.steps_done() == steps
        assert np.array_equal(after_record, after_adjoint)
        assert np.allclose(g_first, g_again, rtol=1e-12, atol=1e-15), (g_first, g_again)
        out[ck] = (after_record, g_first)
    # the recording's end state does not depend on where its checkpoints are
    assert np.array_equal(out[7][0], out[steps][0])
    assert np.allclose(out[7][1], out[steps][1], rtol=1e-12, atol=1e-15), (out[7][1], out[steps][1])
    # and equals plain stepping
    with lbm.Simulation(w) as sim:
        sim.step(steps)
        assert np.array_equal(sim.fields(mask).cpu().numpy(), out[7][0])


def test_adjoint_with_16bit_storage():
    """The adjoint of a run whose populations are stored as BF16 / FP16
    deviations: the recomputed forward steps are the 16-bit ones, the reverse
    arithmetic is FP32 (the storage rounding is passed through as the
    identity). The gradients of the built-in witness loss, with the profile
    entries, follow the FP32-storage gradients closely: FP16 closer than
    BF16, both within the guards below (about three times the GB300
    measurement: FP16 3.6e-6, BF16 1.9e-5 relative L2 over the gradient)."""
    w = W.parity_small().replace(nx=24, ny=24, nz=48, alpha=0.5, z0=-1.0, tau=0.6, profile=np.ones(8),
                                 profile_rmax=2.0)
    steps = 120
    g = {}
    for st in (W.F32, W.F16, W.BF16):
        with lbm.Simulation(w.replace(storage=st)) as sim:
            g[st] = sim.adjoint_step(None, nsteps=steps, ckpt_every=11)
    err = {st: float(np.linalg.norm(g[st] - g[W.F32]) / np.linalg.norm(g[W.F32])) for st in (W.F16, W.BF16)}
    print("16-bit storage adjoint vs FP32 storage (rel-L2 over the gradient):", err)
    assert np.all(np.isfinite(g[W.BF16])) and np.all(np.isfinite(g[W.F16]))
    assert err[W.F16] < err[W.BF16]
    assert err[W.F16] < 1e-5 and err[W.BF16] < 6e-5, err


def test_adjoint_full_size_against_finite_differences():
    """The differentiable form at its full size (256x128x128, n_b/n0 = 0.5,
    500 steps, checkpoints every ceil(sqrt(500)) = 23, the built-in witness
    loss, a 64-point profile): the adjoint's derivatives with respect to
    (n_b/n0, sigma_r, sigma_z) and along a random profile direction against
    central differences of the FP32 forward with h = 1e-3 (relative for the
    driver parameters). FP32 forward noise ~ eps |L| / h makes this a check
    to 1e-2."""
    prof = np.ones(64)
    w = W.differentiable().replace(profile=prof, profile_rmax=128 * 0.2 / 2)
    steps = 500

    def loss(**kw):
        with lbm.Simulation(w.replace(**kw)) as sim:
            sim.step(steps)
            return sim.witness_loss()

    with lbm.Simulation(w) as sim:
        g = sim.adjoint_step(None, nsteps=steps)
    rng = np.random.default_rng(21)
    d = rng.standard_normal(64)
    checks = []
    for i, name in enumerate(("alpha", "sigma_r", "sigma_z")):
        v = getattr(w, name)
        h = 1e-3 * v
        fd = (loss(**{name: v + h}) - loss(**{name: v - h})) / (2 * h)
        checks.append((name, fd, g[i]))
    h = 1e-3
    fd = (loss(profile=prof + h * d) - loss(profile=prof - h * d)) / (2 * h)
    checks.append(("profile", fd, float(d @ g[3:])))
    print("full-size adjoint vs central differences:", checks)
    for name, fd, ad in checks:
        assert abs(fd - ad) <= 1e-2 * abs(ad), (name, fd, ad)
