"""A grid past 32-bit plane offsets: the 8-obstacle dam break at 32768 x 16448
cells (539 M cells; the four state planes hold 2.16e9 elements, so the alpha
entries of the top 256 rows lie past element 2^31 of the state; 17 GB per FP64
state on the device and about 55 GB of host arrays).  One step in each
precision against the oracle at sampled cells: random fluid cells, cells
whose alpha entry lies past element 2^31, cells next to the obstacles, on strip
column edges and on the water column's edge."""
import numpy as np
import pytest

from paper_1806_04960_gb300 import cases
from oracle import oracle as O

pytestmark = pytest.mark.gpu

NX, NY = 32768, 16448


HOST_BYTES = 80 * 2 ** 30      # the case, two states and the generator's temporaries
DEVICE_BYTES = 60 * 2 ** 30    # the FP32 handle's state, staging and scratch, or the FP64 one's


@pytest.fixture(scope="module")
def fv():
    import os
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    if avail < HOST_BYTES:
        pytest.skip(f"needs {HOST_BYTES >> 30} GiB of free host memory, {avail >> 30} available")
    free, _ = torch.cuda.mem_get_info()
    if free < DEVICE_BYTES:
        pytest.skip(f"needs {DEVICE_BYTES >> 30} GiB of free device memory, {free >> 30} available")
    from paper_1806_04960_gb300 import build
    build.build()
    from paper_1806_04960_gb300 import fv as mod
    return mod


@pytest.fixture(scope="module")
def case():
    return cases.c2(NX, NY)


def picks(c):
    n = NX * NY
    assert 4 * n > 2 ** 31
    rng = np.random.Generator(np.random.PCG64(2 ** 31))
    fluid = c.solid.ravel() == 0
    out = [rng.integers(0, n, 4000)]
    first_past = 2 ** 31 - 3 * n            # alpha plane entries past element 2^31
    out.append(rng.integers(first_past, n, 1000))
    sol = np.flatnonzero(c.solid.ravel())
    nb = np.concatenate([sol - 1, sol + 1, sol - NX, sol + NX])
    out.append(rng.choice(nb[(nb >= 0) & (nb < n)], 500))
    jj = rng.integers(0, NY, 500)
    out.append(jj * NX + rng.choice(np.concatenate([np.arange(31, NX, 32), np.arange(0, NX, 32)]), 500))
    col = int(np.ceil(1.0 / c.dx))          # the water column's right edge, x = 1
    jj = rng.integers(0, NY // 2, 500)
    out.append(jj * NX + col - 1 + rng.integers(0, 2, 500))
    cells = np.unique(np.concatenate(out))
    return cells[fluid[cells]]


# (relative to the component's largest sampled value, absolute) per component
TOL = {"FV_FP64": [(1e-12, 0.0), (1e-12, 1e-11), (1e-12, 1e-11), (1e-12, 0.0)],
       "FV_FP32_DEV": [(1e-6, 0.0), (1e-4, 0.0), (1e-4, 0.0), (1e-6, 0.0)]}


@pytest.mark.parametrize("prec", ["FV_FP64", "FV_FP32_DEV"])
def test_one_step_past_32_bit_plane_offsets(fv, case, prec):
    """The oracle steps from the state the GPU holds (FP32: rounded to the
    deviation form and widened back) at the sampled cells.  The relative bounds
    are those of the 4096 x 2048 sampled steps.  After one step from rest the
    momenta are tiny (largest sampled |alpha rho v| about 3e-5), while the
    water column at rest keeps FP64 momenta of roundoff size (measured 1.4e-12
    where the oracle's are exactly 0, 1e-16 of alpha rho c): FP64 momenta also
    pass within 1e-11 absolute."""
    tol = TOL[prec]
    c = case
    s = fv.Solver(c, getattr(fv, prec))
    s.set_state(c.q)
    q0 = s.get_state() if prec == "FV_FP32_DEV" else c.q
    s.step(1, c.cfl)
    d = s.diag()
    q1 = s.get_state()
    s.close()
    assert d.status == 0 and d.steps == 1
    cells = picks(c)
    ref, dt = O.step_cells(c, q0, cells)
    got = q1.reshape(4, -1)[:, cells].T
    del q1
    assert abs(d.t - dt) <= (1e-13 if prec == "FV_FP64" else 1e-6) * dt
    for v in range(4):
        rtol, atol = tol[v]
        scale = np.abs(ref[:, v]).max()
        excess = np.abs(got[:, v] - ref[:, v]) - rtol * (scale if scale > 0 else 1.0) - atol
        assert excess.max() <= 0.0, (prec, v, np.abs(got[:, v] - ref[:, v]).max(), scale)
