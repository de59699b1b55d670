"""fv_adjoint against the FP64 oracle.

The loss is the gauge loss L = sum_n dt_n sum_g (m_g^n - T_g^n)^2 of the
gradient workload (dam break over the obstacle; target record from the seeded
perturbed initial state with column 0.95 m and obstacle 0.25 m).  Its
derivative with respect to the initial state, with dt_n and the levels K^n
held at their forward values, is checked against central differences of the
oracle's loss with the oracle's own dt_n and K^n held fixed (orc_run_record),
along seeded directions and for single entries.

The checks start from a generic state (the dam break with all four fields
perturbed, cases.generic): at the unperturbed dam break, alpha is exactly 1 or
exactly eps and the fluctuations are exactly 0 over whole regions, so stencil
extrema tie exactly and the frozen-branch map has kinks at the point itself
(one-sided derivatives differ; the adjoint returns one of its generalised
gradients).  Limiter switches lie about 1e-7 (relative) from a generic state,
so the differences use a step of 1e-9.

The FP32 gradient is the derivative along the FP32 trajectory.  The
frozen-branch map switches limiter branches densely, so its exact gradient is
itself rough in the state: moving this initial state by 5e-6 (relative, the
FP32 rounding level) changes the FP64 gradient by 2 % (alpha rho) and 11 %
(alpha) in L1.  The FP32 gradient can follow the FP64 one only to that level;
the float arithmetic of the reverse sweep itself is pinned on the host
(test_adjoint_host.py, float along the oracle trajectory: 1e-5).  The FP32
checks here use a target far from the trajectory (T = m_g^0 + 500 kg/m^3), so
that the FP32 forward error of the residuals m - T does not add to that.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1806_04960_gb300 import cases

pytestmark = pytest.mark.gpu

NX, NY, NSTEPS, CFL = 64, 32, 80, 0.45
H = 1e-9  # relative step of the central differences


@pytest.fixture(scope="module")
def fv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_04960_gb300 import build
    build.build()
    from paper_1806_04960_gb300 import fv as mod
    return mod


@pytest.fixture(scope="module")
def problem():
    c = cases.generic(cases.c5(NX, NY, steps=NSTEPS, cfl=CFL), 7)
    gauges = cases.c5_gauges(c)
    tc = cases.c5_target(NX, NY, cfl=CFL)
    _, _, _, target = O.run_record(tc, NSTEPS, gauges, cfl=CFL)
    _, dt, K, m = O.run_record(c, NSTEPS, gauges, cfl=CFL)
    loss = float(np.sum(dt * np.sum((m - target) ** 2, axis=1)))
    far = np.repeat(c.q[0].ravel()[gauges][None, :] + 500.0, NSTEPS, axis=0)
    return dict(case=c, gauges=gauges, target=target, dt=dt, K=K, m=m, loss=loss, far=far)


def oracle_loss(pb, q, target):
    c = pb["case"]
    _, _, _, m = O.run_record(c, NSTEPS, pb["gauges"], q=q, cfl=CFL, dt_fix=pb["dt"], K_fix=pb["K"])
    return float(np.sum(pb["dt"] * np.sum((m - target) ** 2, axis=1)))


def oracle_dir_deriv(pb, d, h, target=None):
    q = pb["case"].q
    t = pb["target"] if target is None else target
    return (oracle_loss(pb, q + h * d, t) - oracle_loss(pb, q - h * d, t)) / (2 * h)


def gpu_grad(fv, pb, prec, every=0, target=None):
    c = pb["case"]
    s = fv.Solver(c, prec)
    s.set_state(c.q)
    g, info, series = s.adjoint(NSTEPS, pb["gauges"], pb["target"] if target is None else target,
                                cfl=CFL, checkpoint_every=every, want_series=True)
    s.close()
    return g, info, series


@pytest.fixture(scope="module")
def fd_dirs(problem):
    d = cases.c5_directions(problem["case"], count=32)[:16]
    return d, np.array([oracle_dir_deriv(problem, dk, H) for dk in d])


@pytest.fixture(scope="module")
def fd_dirs_far(problem):
    d = cases.c5_directions(problem["case"], count=32)[16:32]
    return d, np.array([oracle_dir_deriv(problem, dk, H, problem["far"]) for dk in d])


def test_fp64_forward_record_matches_oracle(fv, problem):
    g, info, series = gpu_grad(fv, problem, fv.FV_FP64)
    assert np.max(np.abs(series - problem["m"]) / np.abs(problem["m"])) < 1e-10
    assert abs(info.loss - problem["loss"]) <= 1e-9 * problem["loss"]
    assert info.checkpoints == int(np.ceil(NSTEPS / np.ceil(np.sqrt(NSTEPS))))
    assert np.all(g[:, problem["case"].solid == 1] == 0.0)


def test_fp64_gradient_directions_match_oracle_differences(fv, problem, fd_dirs):
    g, _, _ = gpu_grad(fv, problem, fv.FV_FP64)
    d, fd = fd_dirs
    dd = np.array([np.sum(g * dk) for dk in d])
    assert np.all(np.abs(dd - fd) < 1e-5 * np.max(np.abs(fd))), (dd, fd)


def test_fp64_gradient_far_target_matches_oracle_differences(fv, problem, fd_dirs_far):
    g, _, _ = gpu_grad(fv, problem, fv.FV_FP64, target=problem["far"])
    d, fd = fd_dirs_far
    dd = np.array([np.sum(g * dk) for dk in d])
    assert np.all(np.abs(dd - fd) < 1e-5 * np.max(np.abs(fd))), (dd, fd)


def test_fp32_gradient_directions_match_oracle_differences(fv, problem, fd_dirs_far):
    g, info, series = gpu_grad(fv, problem, fv.FV_FP32_DEV, target=problem["far"])
    assert np.max(np.abs(series - problem["m"]) / np.abs(problem["m"])) < 1e-4
    d, fd = fd_dirs_far
    dd = np.array([np.sum(g * dk) for dk in d])
    assert np.all(np.abs(dd - fd) < 5e-2 * np.max(np.abs(fd))), (dd, fd)


def test_fp32_gradient_follows_fp64_gradient(fv, problem):
    g64, _, _ = gpu_grad(fv, problem, fv.FV_FP64, target=problem["far"])
    g32, _, _ = gpu_grad(fv, problem, fv.FV_FP32_DEV, target=problem["far"])
    for v, tol in ((0, 5e-2), (1, 5e-2), (2, 5e-2), (3, 0.25)):
        assert np.sum(np.abs(g32[v] - g64[v])) / np.sum(np.abs(g64[v])) < tol, v


def test_fp64_gradient_entries_match_oracle_differences(fv, problem):
    """Single entries (alpha rho and alpha of liquid cells: in a gas cell a
    step that the loss resolves is a relative change of 1e-6, beyond the
    nearest limiter switch) by differences of the oracle's loss along the unit
    vector."""
    c = problem["case"]
    g, _, _ = gpu_grad(fv, problem, fv.FV_FP64)
    rng = np.random.Generator(np.random.PCG64(11))
    liquid = np.flatnonzero(((c.solid == 0) & (c.q[3] > 0.5)).ravel())
    picks = []
    for cell in rng.choice(liquid, size=3, replace=False):
        for v in (0, 3):
            picks.append((v, int(cell)))
    for v, cell in picks:
        e = np.zeros_like(c.q)
        e.reshape(4, -1)[v, cell] = 1.0
        h = H * (c.rho0 if v == 0 else 1.0)   # field scale: a gas cell's own value is too small
        fd = oracle_dir_deriv(problem, e, h)
        got = g.reshape(4, -1)[v, cell]
        assert abs(got - fd) <= 1e-4 * max(abs(fd), 1e-3 * np.max(np.abs(g[v]))), (v, cell, got, fd)


@pytest.mark.parametrize("prec", ["FV_FP64", "FV_FP32_DEV"])
def test_gradient_independent_of_checkpoint_spacing(fv, problem, prec):
    p = getattr(fv, prec)
    ref, info0, _ = gpu_grad(fv, problem, p, every=0)
    for every in (1, 7, NSTEPS):
        g, info, _ = gpu_grad(fv, problem, p, every=every)
        assert np.array_equal(g, ref)
        assert info.loss == info0.loss
        assert info.checkpoints == -(-NSTEPS // every)
        assert info.recomputed_steps == NSTEPS - info.checkpoints


def test_autograd_function(fv, problem):
    import torch
    c = problem["case"]
    s = fv.Solver(c, fv.FV_FP64)
    q0 = torch.tensor(c.q, device="cuda", dtype=torch.float64, requires_grad=True)
    L = fv.gauge_loss_function().apply(q0, s, NSTEPS, CFL, problem["gauges"], problem["target"])
    (3.0 * L).backward()
    g, _, _ = gpu_grad(fv, problem, fv.FV_FP64)
    assert abs(L.item() - problem["loss"]) <= 1e-9 * problem["loss"]
    assert np.array_equal(q0.grad.cpu().numpy(), 3.0 * g)
    s.close()


def test_adjoint_rejects_bad_arguments(fv, problem):
    c = problem["case"]
    s = fv.Solver(c, fv.FV_FP64)
    s.set_state(c.q)
    solid_cell = int(np.flatnonzero(c.solid.ravel())[0])
    with pytest.raises(fv.FvError) as ei:
        s.adjoint(4, [solid_cell], np.zeros(4), cfl=CFL)
    assert ei.value.status == fv.FV_EINVAL
    with pytest.raises(fv.FvError):
        s.adjoint(4, [c.nx * c.ny], np.zeros(4), cfl=CFL)
    with pytest.raises(fv.FvError):
        s.adjoint(4, [0], np.full(4, np.nan), cfl=CFL)
    with pytest.raises(fv.FvError):
        s.adjoint(0, [0], np.zeros(0), cfl=CFL)
    s.close()


def test_full_grid_gradient_on_conditioned_horizon(fv):
    """The 512 x 256 workload over 200 steps (t = 0.016 s).  Beyond about
    step 600 the bed toe of the dam-break wave amplifies perturbations (the
    frozen-branch map multiplies a 1e-13 perturbation by ~10 per 20 steps
    there) and gradients reach 1e25 and more.  With 131k cells the limiter
    switches lie within 1e-9 of the state, so the differences use 1e-11 (they
    agree with 1e-10 and 1e-12 to 2e-5).  FP64 against the oracle's
    differences with the target record (1e-4), FP32 with the far target (to
    the roughness floor of the gradient, see above)."""
    n, h = 200, 1e-11
    c = cases.generic(cases.c5(512, 256, cfl=CFL), 7)
    gauges = cases.c5_gauges(c)
    _, _, _, target = O.run_record(cases.c5_target(512, 256, cfl=CFL), n, gauges, cfl=CFL)
    _, dt, K, _ = O.run_record(c, n, gauges, cfl=CFL)
    far = np.repeat(c.q[0].ravel()[gauges][None, :] + 500.0, n, axis=0)

    def loss(q, t):
        _, _, _, m = O.run_record(c, n, gauges, q=q, cfl=CFL, dt_fix=dt, K_fix=K)
        return float(np.sum(dt * np.sum((m - t) ** 2, axis=1)))

    d = cases.c5_directions(c, count=1, seed=33)[0]
    for prec, t, tol in ((fv.FV_FP64, target, 1e-4), (fv.FV_FP32_DEV, far, 5e-2)):
        s = fv.Solver(c, prec)
        s.set_state(c.q)
        g, info, _ = s.adjoint(n, gauges, t, cfl=CFL)
        s.close()
        assert np.all(np.isfinite(g))
        fd = (loss(c.q + h * d, t) - loss(c.q - h * d, t)) / (2 * h)
        assert abs(np.sum(g * d) - fd) <= tol * abs(fd), (prec, np.sum(g * d), fd)


def test_frozen_map_matches_oracle_and_its_differences_match_the_adjoint(fv, problem):
    """fv_step_frozen, the map fv_adjoint differentiates: with the free run's
    dt and levels (recorded through the C ABI) its gauge record equals the
    oracle's (<= 1e-10) in FP64, and central differences of its loss along
    seeded directions equal the adjoint's directional derivatives (the same
    bound as against the oracle's differences)."""
    c, gauges, target = problem["case"], problem["gauges"], problem["target"]
    s = fv.Solver(c, fv.FV_FP64)
    s.set_state(c.q)
    dts, Ks = s.record_free_run(NSTEPS, CFL)
    s.close()
    assert np.array_equal(Ks, problem["K"])
    # the GPU's own free run: its dt follows its state, 1e-14 apart from the oracle's
    assert np.all(np.abs(dts - problem["dt"]) <= 1e-12 * problem["dt"])

    def loss(q):
        s = fv.Solver(c, fv.FV_FP64)
        s.set_state(q)
        m = s.step_frozen(dts, Ks, gauges)
        s.close()
        return float(np.sum(dts * np.sum((m - target) ** 2, axis=1))), m

    l0, m0 = loss(c.q)
    assert np.max(np.abs(m0 - problem["m"]) / np.abs(problem["m"])) < 1e-10
    assert abs(l0 - problem["loss"]) <= 1e-9 * problem["loss"]
    g, _, _ = gpu_grad(fv, problem, fv.FV_FP64)
    d = cases.c5_directions(c, count=32)[:8]
    dd = np.array([np.sum(g * dk) for dk in d])
    fd = np.array([(loss(c.q + H * dk)[0] - loss(c.q - H * dk)[0]) / (2 * H) for dk in d])
    assert np.all(np.abs(dd - fd) < 1e-5 * np.max(np.abs(fd))), (dd, fd)


def test_frozen_map_arguments(fv, problem):
    c = problem["case"]
    s = fv.Solver(c, fv.FV_FP64)
    s.set_state(c.q)
    with pytest.raises(fv.FvError):
        s.step_frozen(np.array([1e-4]), np.full((1, c.nx), c.ny + 1))    # level above the grid
    with pytest.raises(fv.FvError):
        s.step_frozen(np.array([np.nan]), np.zeros((1, c.nx)))             # dt not finite
    s.close()
