"""x-strip decomposition on one GPU (fv_set_partition / fv_part_*, driven by
decomp.StripSolver): a grid advanced as 2-4 strips with halo and rate
exchanges equals one handle on the whole grid bit for bit, in FP64 and in the
FP32 deviation form, on walled and transmissive, even and ragged grids, and
on the benchmark's 4096 x 2048 grid."""
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


def whole_grid(fv, case, prec, steps, cfl):
    s = fv.Solver(case, prec)
    s.set_state(case.q)
    s.step(steps, cfl)
    q, d = s.get_state(), s.diag()
    s.close()
    return q, d


def strips(case, prec, parts, steps, cfl):
    from paper_1806_04960_gb300 import decomp
    s = decomp.StripSolver(case, prec, parts)
    s.set_state(case.q)
    s.step(steps, cfl)
    q = s.get_state()
    t, n, status, ts = s.diag()
    s.close()
    return q, t, n, status, ts


def ragged():
    return cases.perturbed(cases.dambreak(45, 13, lx=1.4, ly=0.4, x_col=0.5, h_col=0.3,
                                          sides=(1, 1, 0, 1)), 7)


@pytest.mark.parametrize("prec", ["FV_FP64", "FV_FP32_DEV"])
@pytest.mark.parametrize("make,parts,steps,cfl", [
    (lambda: cases.c1(), 2, 60, 0.45),
    (lambda: cases.c1(), 3, 60, 0.9),
    (lambda: cases.perturbed(cases.c1(), 5), 4, 40, 0.45),
    (ragged, 3, 8, 0.45),
])
def test_strips_equal_the_whole_grid(fv, prec, make, parts, steps, cfl):
    c = make()
    p = getattr(fv, prec)
    ref, d = whole_grid(fv, c, p, steps, cfl)
    got, t, n, status, ts = strips(c, p, parts, steps, cfl)
    assert status == 0 and d.status == 0
    assert n == steps and all(x == t for x in ts)
    assert t == d.t
    assert np.array_equal(got, ref)


def test_strips_on_the_benchmark_grid(fv):
    """4096 x 2048 with its 8 obstacles, FP32, 2 strips: 5 steps bit for bit."""
    c = cases.c2()
    ref, d = whole_grid(fv, c, fv.FV_FP32_DEV, 5, c.cfl)
    got, t, _, status, _ = strips(c, fv.FV_FP32_DEV, 2, 5, c.cfl)
    assert status == 0 and t == d.t
    assert np.array_equal(got, ref)


def test_partition_arguments(fv):
    import torch
    c = cases.c1()
    s = fv.Solver(c, fv.FV_FP64)
    with pytest.raises(fv.FvError):
        fv.fv_set_partition(s.h, 1, 100)          # own_lo must be 0 or 2
    with pytest.raises(fv.FvError):
        fv.fv_set_partition(s.h, 2, c.nx - 1)     # E halo must be 0 or 2 columns
    fv.fv_set_partition(s.h, 2, c.nx)
    s.set_state(c.q)
    with pytest.raises(fv.FvError):
        s.step(2, 0.45)                           # one step per call
    buf = torch.empty(fv.fv_part_halo_bytes(s.h), dtype=torch.uint8, device="cuda")
    with pytest.raises(fv.FvError):
        fv.fv_part_pack(s.h, 1, buf)              # no strip to the E
    fv.fv_part_pack(s.h, 0, buf)
    assert fv.fv_part_halo_bytes(s.h) == 8 * c.ny * 8 + 16
    s.close()
