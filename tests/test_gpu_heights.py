"""fv_adjoint's obstacle-height derivative against the FP64 oracle.

The paper removes whole cells for an obstacle; its height gets a derivative
through the partial cells of reading R-h (raising obstacle k by theta dy
leaves each of its top fluid cells the capacity 1 - theta).  fv_adjoint
returns dL/dh_k at theta = 0+ with dt_n and the levels held at their forward
values; the oracle's partial cells give the same map, whose one-sided
differences in theta (Richardson-extrapolated, dt_n and K^n fixed) are the
reference.  Workload: water over a 0.2 m obstacle in a 2 x 1 m box (48 x 24),
60 steps from a generic state (no exact ties in the limiter), 5 gauges.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1806_04960_gb300 import cases

pytestmark = pytest.mark.gpu

NSTEPS, CFL = 60, 0.45


@pytest.fixture(scope="module")
def fv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_04960_gb300 import build
    build.build()
    from paper_1806_04960_gb300 import fv as mod
    return mod


def _gauges(c):
    g = np.array([c.nx * 5 + 10, c.nx * 8 + 20, c.nx * 10 + 24, c.nx * 3 + 30, c.nx * 10 + 35],
                 dtype=np.int64)
    assert np.all(c.solid.ravel()[g] == 0)
    return g


def _problem(c):
    g = _gauges(c)
    _, dt, K, m = O.run_record(c, NSTEPS, g, cfl=CFL)
    _, _, _, target = O.run_record(cases.generic(cases.heights(c.nx, c.ny), 8), NSTEPS, g, cfl=CFL)
    far = np.repeat(c.q[0].ravel()[g][None, :] + 500.0, NSTEPS, axis=0)
    return dict(case=c, gauges=g, dt=dt, K=K, m=m, target=target, far=far,
                hid=cases.height_ids(c))


@pytest.fixture(scope="module")
def one():
    return _problem(cases.generic(cases.heights(), 7))


@pytest.fixture(scope="module")
def two():
    rects = [cases.H_RECT, (0.92, 1.05, 0.0, 0.3)]
    c0 = cases.dambreak(48, 24, lx=2.0, ly=1.0, x_col=1.2, h_col=0.6, rects=rects, k0=4.36e5,
                        cfl=CFL, steps=NSTEPS)
    return _problem(cases.generic(c0, 7))


def oracle_dL_dh(pb, k, target):
    """Richardson-extrapolated one-sided difference of the oracle's loss in
    theta_k (dt_n and K^n fixed), per metre of height."""
    c = pb["case"]

    def loss(theta):
        cap = np.ones((c.ny, c.nx))
        cap[pb["hid"] == k] = 1.0 - theta
        _, _, _, m = O.run_record(c, NSTEPS, pb["gauges"], cfl=CFL, dt_fix=pb["dt"],
                                  K_fix=pb["K"], cap=cap)
        return float(np.sum(pb["dt"] * np.sum((m - target) ** 2, axis=1)))

    L0, e = loss(0.0), 1e-5
    d1 = (loss(e) - L0) / e
    d2 = (loss(2 * e) - L0) / (2 * e)
    return (2 * d1 - d2) / c.dy


def gpu(fv, pb, prec, target, every=0):
    c = pb["case"]
    s = fv.Solver(c, prec)
    s.set_state(c.q)
    out = s.adjoint_heights(NSTEPS, pb["gauges"], target, pb["hid"], cfl=CFL,
                            checkpoint_every=every)
    s.close()
    return out


def test_fp64_height_derivative_matches_oracle(fv, one):
    grad, dh, info, _ = gpu(fv, one, fv.FV_FP64, one["target"])
    ref = oracle_dL_dh(one, 0, one["target"])
    assert dh.shape == (1,)
    assert abs(dh[0] - ref) < 1e-5 * abs(ref), (dh, ref)
    assert abs(ref) > 1e-3 * info.loss / one["case"].dy    # a derivative that matters


def test_fp64_two_obstacles_match_oracle(fv, two):
    _, dh, _, _ = gpu(fv, two, fv.FV_FP64, two["target"])
    for k in (0, 1):
        ref = oracle_dL_dh(two, k, two["target"])
        assert abs(dh[k] - ref) < 1e-5 * abs(ref), (k, dh, ref)


def test_fp32_height_derivative_matches_oracle(fv, one):
    """FP32 deviation form along its own trajectory, target far from it (so
    the float forward error does not enter through the residuals)."""
    _, dh, _, _ = gpu(fv, one, fv.FV_FP32_DEV, one["far"])
    ref = oracle_dL_dh(one, 0, one["far"])
    assert abs(dh[0] - ref) < 2e-2 * abs(ref), (dh, ref)


def test_heights_leave_the_state_gradient_and_loss_unchanged(fv, one):
    c = one["case"]
    for prec in (fv.FV_FP64, fv.FV_FP32_DEV):
        grad, dh, info, _ = gpu(fv, one, prec, one["target"])
        s = fv.Solver(c, prec)
        s.set_state(c.q)
        g0, info0, _ = s.adjoint(NSTEPS, one["gauges"], one["target"], cfl=CFL)
        s.close()
        assert np.array_equal(grad, g0)
        assert info.loss == info0.loss


def test_height_derivative_independent_of_checkpoints(fv, one):
    for prec in (fv.FV_FP64, fv.FV_FP32_DEV):
        a = gpu(fv, one, prec, one["target"], every=0)[1]
        b = gpu(fv, one, prec, one["target"], every=7)[1]
        assert np.array_equal(a, b)


def test_lake_at_rest_has_no_height_derivative(fv):
    """A lake at rest over the obstacle stays at rest for every theta, so dL/dh
    vanishes whatever the target, to roundoff (about 1e-21 of the loss scale
    in the deviation form)."""
    c = cases.dambreak(48, 24, lx=2.0, ly=1.0, rects=[cases.H_RECT], k0=4.36e5,
                       lake_level=15 / 24, cfl=CFL, steps=NSTEPS)
    g = _gauges(c)
    far = np.repeat(c.q[0].ravel()[g][None, :] + 500.0, NSTEPS, axis=0)
    hid = cases.height_ids(c)
    for prec, tol in ((fv.FV_FP32_DEV, 1e-12), (fv.FV_FP64, 1e-9)):
        s = fv.Solver(c, prec)
        s.set_state(c.q)
        _, dh, info, _ = s.adjoint_heights(NSTEPS, g, far, hid, cfl=CFL)
        s.close()
        scale = info.loss / c.dy
        assert abs(dh[0]) <= tol * scale, (prec, dh, scale)


def test_bad_height_maps_are_rejected(fv, one):
    c = one["case"]
    s = fv.Solver(c, fv.FV_FP64)
    s.set_state(c.q)
    bad = one["hid"].copy()
    bad[10, 3] = 0                                   # a fluid cell with fluid below
    with pytest.raises(RuntimeError):
        s.adjoint_heights(4, one["gauges"], one["target"][:4], bad, cfl=CFL)
    bad = one["hid"].copy()
    bad[bad == 0] = 5
    with pytest.raises(RuntimeError):
        fv.fv_adjoint(s.h, 4, CFL, one["gauges"], one["target"][:4], np.empty_like(c.q),
                      height_id=bad, nheights=2)
    s.close()
