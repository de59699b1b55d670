"""The allocation-free entry point fv_step_static against the handle-based path.

fv_step_static exists for callers that cannot allocate device memory (an
application that owns all GPU memory through its own pool, or a latency-
critical loop that cannot afford cudaMalloc's implicit synchronisation); its
scratch lives in one static device array.  Both paths run the same kernels on
the same table, so their results are compared bit for bit.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process.
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


def static_step(fv, case, q_in, q_out, solid, stream, want_dt=True):
    """One fv_step_static call through the C ABI; returns (status, dt)."""
    grid = fv.fv_grid(case.nx, case.ny, case.x0, case.y0, case.dx, case.dy)
    eos = fv.fv_eos(case.rho0, case.k0, case.gamma, case.g, case.eps)
    side = (C.c_int32 * 4)(*case.sides)
    dt = C.c_double(0.0)
    st = fv._lib.fv_step_static(C.byref(grid), C.byref(eos), side, C.c_void_p(solid.data_ptr()),
                                C.c_void_p(q_in.data_ptr()), C.c_void_p(q_out.data_ptr()),
                                float(case.cfl), C.c_void_p(stream),
                                C.byref(dt) if want_dt else None)
    return st, dt.value


def device_inputs(case):
    import torch
    dev = torch.device("cuda")
    solid = torch.from_numpy(np.ascontiguousarray(case.solid, dtype=np.uint8)).to(dev)
    q0 = torch.from_numpy(np.ascontiguousarray(case.q)).to(dev)
    return solid, q0


def handle_steps(fv, case, n):
    """States after 1..n steps of the handle path, and the first step's dt."""
    s = fv.Solver(case, fv.FV_FP64)
    s.set_state(case.q)
    d0 = s.diag().dt_next
    out = []
    for _ in range(n):
        s.step(1, case.cfl)
        out.append(s.get_state())
    s.close()
    return out, d0


@pytest.mark.parametrize("make", [lambda: cases.c1(),
                                  lambda: cases.perturbed(cases.dambreak(45, 13, lx=1.4, ly=0.4,
                                                                         x_col=0.5), 7)])
def test_static_step_matches_handle_path_two_calls(fv, make):
    import torch
    c = make()
    stream = torch.cuda.current_stream().cuda_stream
    solid, q0 = device_inputs(c)
    q1 = torch.empty_like(q0)
    q2 = torch.empty_like(q0)
    st1, dt1 = static_step(fv, c, q0, q1, solid, stream)
    st2, dt2 = static_step(fv, c, q1, q2, solid, stream)
    torch.cuda.synchronize()
    assert st1 == fv.FV_OK and st2 == fv.FV_OK, fv.fv_last_error()
    (ref1, ref2), d0 = handle_steps(fv, c, 2)
    assert dt1 == d0
    assert np.array_equal(q1.cpu().numpy(), ref1)
    assert np.array_equal(q2.cpu().numpy(), ref2)
    assert dt2 > 0.0


def test_small_grid_after_large_grid_asynchronous(fv):
    """The array keeps the previous call's contents (column sums, levels,
    equilibrium table beyond the new grid's rows): a call on the 4096 x 2048
    benchmark grid followed by two calls on a ragged 45 x 13 grid with
    transmissive sides, without dt_out (asynchronous: no check, no sync until
    the caller synchronises the stream), gives the handle path's bits."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    big = cases.c2()
    sb, qb0 = device_inputs(big)
    qb1 = torch.empty_like(qb0)
    st, _ = static_step(fv, big, qb0, qb1, sb, stream)
    assert st == fv.FV_OK, fv.fv_last_error()
    del sb, qb0, qb1
    c = cases.perturbed(cases.dambreak(45, 13, lx=1.4, ly=0.4, x_col=0.5, h_col=0.3,
                                       sides=(1, 1, 0, 1)), 7)
    solid, q0 = device_inputs(c)
    q1 = torch.empty_like(q0)
    q2 = torch.empty_like(q0)
    assert static_step(fv, c, q0, q1, solid, stream, want_dt=False)[0] == fv.FV_OK
    assert static_step(fv, c, q1, q2, solid, stream, want_dt=False)[0] == fv.FV_OK
    torch.cuda.current_stream().synchronize()
    (ref1, ref2), _ = handle_steps(fv, c, 2)
    assert np.array_equal(q1.cpu().numpy(), ref1)
    assert np.array_equal(q2.cpu().numpy(), ref2)


def test_static_step_allocates_no_device_memory(fv):
    """After one warm call (which looks up the array's address and loads the
    kernels), a call leaves the device's free memory unchanged."""
    import torch
    c = cases.c1()
    stream = torch.cuda.current_stream().cuda_stream
    solid, q0 = device_inputs(c)
    q1 = torch.empty_like(q0)
    assert static_step(fv, c, q0, q1, solid, stream)[0] == fv.FV_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert static_step(fv, c, q0, q1, solid, stream)[0] == fv.FV_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_static_step_reports_a_bad_input_state(fv):
    """With dt_out a non-admissible q_in is FV_EINVAL and named as the input."""
    import torch
    c = cases.c1()
    stream = torch.cuda.current_stream().cuda_stream
    q = c.q.copy()
    q[3][5, 5] = -0.1
    solid, _ = device_inputs(c)
    q0 = torch.from_numpy(q).cuda()
    q1 = torch.empty_like(q0)
    st, _ = static_step(fv, c, q0, q1, solid, stream)
    assert st == fv.FV_EINVAL and "q_in" in fv.fv_last_error()


def test_static_step_rejects_oversized_grid(fv):
    import torch
    c = cases.c1()
    grid = fv.fv_grid(8193, 4, 0.0, 0.0, 0.1, 0.1)
    eos = fv.fv_eos(c.rho0, c.k0, 1.0, c.g, c.eps)
    side = (C.c_int32 * 4)(0, 0, 0, 0)
    x = torch.zeros(4, device="cuda", dtype=torch.float64)
    st = fv._lib.fv_step_static(C.byref(grid), C.byref(eos), side, C.c_void_p(x.data_ptr()),
                                C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr() + 8), 0.5,
                                None, None)
    assert st == fv.FV_EINVAL and "8192" in fv.fv_last_error()
