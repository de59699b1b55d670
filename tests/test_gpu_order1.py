"""GPU parity of the first-order scheme (Sections 3.2-3.3; fv_set_order(h, 1))
against the oracle's first-order mode (orc_run_record with order 1).

Tolerances as for the second-order path: FP64 relative L-infinity per
component <= 1e-10 with identical dt and levels; FP32 deviation form relative
L1 <= 1e-4 (alpha rho, alpha) and 1e-3 (momenta); rest states at roundoff.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1806_04960_gb300 import cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1806_04960_gb300 import build
    build.build()
    from paper_1806_04960_gb300 import fv as mod
    return mod


def rel_linf(a, b):
    return np.array([np.abs(a[v] - b[v]).max() / max(np.abs(b[v]).max(), 1e-300) for v in range(4)])


def rel_l1(a, b):
    return np.array([np.abs(a[v] - b[v]).sum() / max(np.abs(b[v]).sum(), 1e-300) for v in range(4)])


def gpu_o1(fv, case, nsteps, prec, cfl, q=None):
    s = fv.Solver(case, prec)
    s.set_order(1)
    s.set_state(case.q if q is None else q)
    t = s.step(nsteps, cfl, want_time=True)
    out = s.get_state()
    K = s.levels()
    d = s.diag()
    s.close()
    return out, t, K, d


@pytest.mark.parametrize("cfl,n", [(0.45, 200), (0.9, 200)])
def test_fp64_first_order_dambreak_matches_oracle(fv, cfl, n):
    c = cases.c1()
    qo, dts, Ks, _ = O.run_record(c, n, [0], cfl=cfl, order=1)
    qg, tg, K, d = gpu_o1(fv, c, n, fv.FV_FP64, cfl)
    assert np.all(rel_linf(qg, qo) <= 1e-10), rel_linf(qg, qo)
    assert abs(tg - dts.sum()) <= 1e-12 * dts.sum()
    _, Kn = O.dt_levels(c, qo, cfl=cfl)
    assert np.array_equal(K, Kn)
    assert d.status == 0 and d.steps == n


@pytest.mark.parametrize("nx,ny,sides", [(45, 13, (0, 0, 0, 0)), (1, 20, (0, 0, 0, 0)),
                                          (33, 1, (0, 0, 0, 0)), (100, 37, (1, 1, 0, 1))])
def test_fp64_first_order_ragged_and_transmissive(fv, nx, ny, sides):
    c = cases.perturbed(cases.dambreak(nx, ny, lx=4.0 * nx / 64, ly=2.0 * ny / 32, sides=sides), 3)
    qo, dts, _, _ = O.run_record(c, 40, [0], cfl=0.45, order=1)
    qg, tg, _, _ = gpu_o1(fv, c, 40, fv.FV_FP64, 0.45)
    assert np.all(rel_linf(qg, qo) <= 1e-10), rel_linf(qg, qo)


@pytest.mark.parametrize("prec", ["FV_FP64", "FV_FP32_DEV"])
def test_first_order_lakes_at_rest(fv, prec):
    p = getattr(fv, prec)
    tol = 1e-12 if prec == "FV_FP64" else 1e-9
    for c in (cases.c1_lake(), cases.lake_box(60, obstacle=True), cases.c2_lake(256, 128)):
        q, _, _, d = gpu_o1(fv, c, 100, p, 0.9)
        fl = c.solid == 0
        assert d.status == 0
        assert np.abs(q[1]).max() <= tol * c.rho0 and np.abs(q[2]).max() <= tol * c.rho0
        assert np.abs(q[0] - c.q[0])[fl].max() <= tol * c.rho0
        # FP32 holds alpha as float (eps = 1e-3 is not a float)
        a0 = c.q[3] if prec == "FV_FP64" else c.q[3].astype(np.float32).astype(np.float64)
        assert np.array_equal(q[3], a0)


def test_fp32_first_order_dambreak_follows_oracle(fv):
    c = cases.c1()
    qo, _, _, _ = O.run_record(c, 200, [0], cfl=0.45, order=1)
    qg, _, _, d = gpu_o1(fv, c, 200, fv.FV_FP32_DEV, 0.45)
    e = rel_l1(qg, qo)
    assert d.status == 0
    assert e[0] <= 1e-4 and e[3] <= 1e-4 and e[1] <= 1e-3 and e[2] <= 1e-3, e


def test_first_order_mass_conserved(fv):
    c = cases.c1()
    s = fv.Solver(c, fv.FV_FP64)
    s.set_order(1)
    s.set_state(c.q)
    m0 = s.diag().mass
    s.step(300, 0.9)
    assert abs(s.diag().mass - m0) <= 1e-13 * m0
    s.close()


def test_order_switch_and_errors(fv):
    """Orders can be switched between calls; a step of order 1 then 2 equals
    the oracle's; invalid orders and the first-order adjoint are rejected."""
    c = cases.perturbed(cases.c1(64, 32), 5)
    q1, _, _, _ = O.run_record(c, 10, [0], cfl=0.45, order=1)
    q2, _, _, _ = O.run_record(c, 10, [0], q=q1, cfl=0.45, order=2)
    s = fv.Solver(c, fv.FV_FP64)
    s.set_state(c.q)
    s.set_order(1)
    s.step(10, 0.45)
    s.set_order(2)
    s.step(10, 0.45)
    assert np.all(rel_linf(s.get_state(), q2) <= 1e-10)
    with pytest.raises(fv.FvError) as ei:
        s.set_order(3)
    assert ei.value.status == fv.FV_EINVAL
    s.set_order(1)
    with pytest.raises(fv.FvError):
        s.adjoint(4, [int(np.flatnonzero(c.solid.ravel() == 0)[0])], np.zeros(4), cfl=0.45)
    s.close()
