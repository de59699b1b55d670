"""The allocation-free entry point fv_step_static against the handle-based path.

fv_step_static exists for callers that cannot allocate device memory (an
application that owns all GPU memory through its own pool, or a latency-
critical loop that cannot afford cudaMalloc's implicit synchronisation); its
scratch lives in one static device array.  This file is collected last so that
a run stopping at the first failure has already run every other test; it also
passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

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


def static_step(fv, case, q_in, q_out, solid, stream):
    grid = fv.fv_grid(case.nx, case.ny, case.x0, case.y0, case.dx, case.dy)
    eos = fv.fv_eos(case.rho0, case.k0, case.gamma, case.g, case.eps)
    side = (C.c_int32 * 4)(*case.sides)
    dt = C.c_double(0.0)
    st = fv._lib.fv_step_static(C.byref(grid), C.byref(eos), side, C.c_void_p(solid.data_ptr()),
                                C.c_void_p(q_in.data_ptr()), C.c_void_p(q_out.data_ptr()),
                                float(case.cfl), C.c_void_p(stream), C.byref(dt))
    assert st == fv.FV_OK, fv.fv_last_error()
    return dt.value


@pytest.mark.parametrize("make", [lambda: cases.c1(), lambda: cases.perturbed(cases.dambreak(45, 13, lx=1.4, ly=0.4, x_col=0.5), 7)])
def test_static_step_matches_handle_path_two_calls(fv, make):
    import torch
    c = make()
    stream = torch.cuda.current_stream().cuda_stream
    dev = torch.device("cuda")
    solid = torch.from_numpy(np.ascontiguousarray(c.solid, dtype=np.uint8)).to(dev)
    q0 = torch.from_numpy(c.q).to(dev)
    q1 = torch.empty_like(q0)
    q2 = torch.empty_like(q0)
    dt1 = static_step(fv, c, q0, q1, solid, stream)
    dt2 = static_step(fv, c, q1, q2, solid, stream)
    torch.cuda.synchronize()
    s = fv.Solver(c, fv.FV_FP64)
    s.set_state(c.q)
    d0 = s.diag().dt_next
    s.step(1, c.cfl)
    ref1 = s.get_state()
    s.step(1, c.cfl)
    ref2 = s.get_state()
    s.close()
    assert abs(dt1 - d0) <= 1e-14 * d0
    assert np.all(rel_linf(q1.cpu().numpy(), ref1) <= 1e-10)
    assert np.all(rel_linf(q2.cpu().numpy(), ref2) <= 1e-10)
    assert dt2 > 0.0


def test_static_step_rejects_oversized_grid(fv):
    import torch
    c = cases.c1()
    grid = fv.fv_grid(fv_max := 8193, 4, 0.0, 0.0, 0.1, 0.1)
    eos = fv.fv_eos(c.rho0, c.k0, 1.0, c.g, c.eps)
    side = (C.c_int32 * 4)(0, 0, 0, 0)
    x = torch.zeros(4, device="cuda", dtype=torch.float64)
    st = fv._lib.fv_step_static(C.byref(grid), C.byref(eos), side, C.c_void_p(x.data_ptr()),
                                C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr() + 8), 0.5,
                                None, None)
    assert st == fv.FV_EINVAL and "8192" in fv.fv_last_error()
