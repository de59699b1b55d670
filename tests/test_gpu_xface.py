"""GPU parity of the conservative Osher-Romberg x faces (fv_set_xface(h,
FV_XFACE_OR), Eq. (OR_cons)) against the oracle's Osher-Romberg x solver, at
second and first order; same tolerances as the Gauss-Legendre paths."""
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


def gpu(fv, case, nsteps, prec, cfl, order):
    s = fv.Solver(case, prec)
    s.set_order(order)
    s.set_xface(fv.FV_XFACE_OR)
    s.set_state(case.q)
    s.step(nsteps, cfl)
    q = s.get_state()
    d = s.diag()
    s.close()
    return q, d


@pytest.mark.parametrize("order", [2, 1])
def test_fp64_osher_romberg_x_matches_oracle(fv, order):
    c = cases.c1()
    qo, _, _, _ = O.run_record(c, 200, [0], cfl=0.45, order=order, xsolver=1)
    qg, d = gpu(fv, c, 200, fv.FV_FP64, 0.45, order)
    assert d.status == 0
    assert np.all(rel_linf(qg, qo) <= 1e-10), rel_linf(qg, qo)
    # a different scheme from the Gauss-Legendre x faces
    qgl, _, _, _ = O.run_record(c, 200, [0], cfl=0.45, order=order)
    assert rel_l1(qg, qgl)[1] > 1e-6


def test_fp64_osher_romberg_x_ragged_transmissive(fv):
    c = cases.perturbed(cases.dambreak(45, 13, lx=2.8125, ly=0.8125, sides=(1, 1, 0, 1)), 9)
    qo, _, _, _ = O.run_record(c, 40, [0], cfl=0.45, xsolver=1)
    qg, _ = gpu(fv, c, 40, fv.FV_FP64, 0.45, 2)
    assert np.all(rel_linf(qg, qo) <= 1e-10), rel_linf(qg, qo)


def test_fp32_osher_romberg_x_follows_oracle_and_lakes_rest(fv):
    c = cases.c1()
    qo, _, _, _ = O.run_record(c, 200, [0], cfl=0.45, xsolver=1)
    qg, d = gpu(fv, c, 200, fv.FV_FP32_DEV, 0.45, 2)
    e = rel_l1(qg, qo)
    assert d.status == 0 and e[0] <= 1e-4 and e[3] <= 1e-4 and e[1] <= 1e-3 and e[2] <= 1e-3, e
    for prec, tol in ((fv.FV_FP64, 1e-12), (fv.FV_FP32_DEV, 1e-9)):
        for order in (2, 1):
            lake = cases.c1_lake()
            q, d = gpu(fv, lake, 100, prec, 0.9, order)
            assert np.abs(q[1]).max() <= tol * lake.rho0 and np.abs(q[2]).max() <= tol * lake.rho0


def test_xface_errors(fv):
    c = cases.c1(32, 16)
    s = fv.Solver(c, fv.FV_FP64)
    s.set_state(c.q)
    with pytest.raises(fv.FvError):
        s.set_xface(2)
    s.set_xface(fv.FV_XFACE_OR)
    with pytest.raises(fv.FvError):
        s.adjoint(4, [int(np.flatnonzero(c.solid.ravel() == 0)[0])], np.zeros(4), cfl=0.45)
    s.close()
