"""Pins of the oracle's partial cells (reading R-h, an extension of the paper).

The paper removes whole cells for obstacles, so an obstacle's height has no
derivative in its scheme.  Reading R-h gives the fluid cell on top of an
obstacle a capacity c = 1 - theta when the obstacle reaches theta dy into it.
These tests pin that extension to what it must satisfy independently of its
own formulas:
  * c = 1 everywhere is the paper's scheme, bit for bit;
  * the mass sum_i c_i (alpha rho)_i dx dy is conserved in a closed box (this
    fails if the x faces' open parts do not match on both sides or if the y
    terms are not divided by c), while the unweighted sum is not;
  * a lake at rest over a raised obstacle stays at rest (no spurious force
    from the partial cells' wall parts or the split interior integral);
  * the loss is smooth in theta at theta = 0+ (one-sided differences are
    linear in the step), so its right derivative exists.
"""
import numpy as np

from oracle import oracle as O
from paper_1806_04960_gb300 import cases

NSTEPS, CFL = 40, 0.45


def _caps(c, theta):
    cap = np.ones((c.ny, c.nx))
    cap[cases.height_ids(c) >= 0] = 1.0 - theta
    return cap


def _gauges(c):
    return np.array([c.nx * 5 + 10, c.nx * 8 + 20, c.nx * 6 + 24, c.nx * 3 + 28, c.nx * 10 + 35],
                    dtype=np.int64)


def test_height_cells_sit_on_the_obstacle():
    c = cases.heights()
    hid = cases.height_ids(c)
    cells = np.argwhere(hid >= 0)
    assert len(cells) == 5
    for j, i in cells:
        assert c.solid[j - 1, i] == 1 and c.solid[j, i] == 0
        assert abs(j * c.dy - 0.2) < c.dy   # the obstacle's top face, snapped to the grid


def test_unit_capacity_is_the_paper_scheme():
    c = cases.generic(cases.heights(), 7)
    g = _gauges(c)
    q0, dt0, K0, m0 = O.run_record(c, 20, g, cfl=CFL)
    q1, dt1, K1, m1 = O.run_record(c, 20, g, cfl=CFL, cap=np.ones((c.ny, c.nx)))
    assert np.array_equal(q0, q1) and np.array_equal(m0, m1) and np.array_equal(dt0, dt1)
    assert np.array_equal(K0, K1)


def test_partial_cells_conserve_weighted_mass():
    c = cases.generic(cases.heights(), 7)
    cap = _caps(c, 0.35)
    fluid = c.solid == 0
    g = _gauges(c)
    q, _, _, _ = O.run_record(c, NSTEPS, g, cfl=CFL, cap=cap)
    m0 = np.sum((cap * c.q[0])[fluid])
    m1 = np.sum((cap * q[0])[fluid])
    assert abs(m1 - m0) <= 1e-13 * m0 * NSTEPS
    # the unweighted sum moves: the partial cells' own mass changes are larger
    u0, u1 = np.sum(c.q[0][fluid]), np.sum(q[0][fluid])
    assert abs(u1 - u0) > 1e-9 * u0


def test_partial_cells_keep_lake_at_rest():
    c = cases.dambreak(48, 24, lx=2.0, ly=1.0, rects=[cases.H_RECT], k0=4.36e5, lake_level=15 / 24,
                       cfl=CFL)
    cap = _caps(c, 0.5)
    q, _, _, _ = O.run_record(c, 100, _gauges(c), cfl=CFL, cap=cap)
    fluid = c.solid == 0
    mom = np.max(np.abs(q[1:3][:, fluid]))
    assert mom < 1e-9, mom
    assert np.max(np.abs(q[0][fluid] - c.q[0][fluid]) / c.q[0][fluid]) < 1e-12


def test_loss_is_smooth_in_theta_from_above():
    c = cases.generic(cases.heights(), 7)
    g = _gauges(c)
    _, dt, K, m = O.run_record(c, 60, g, cfl=CFL)
    tgt = m * (1.0 + 1e-3)

    def loss(theta):
        _, _, _, mm = O.run_record(c, 60, g, cfl=CFL, dt_fix=dt, K_fix=K, cap=_caps(c, theta))
        return float(np.sum(dt * np.sum((mm - tgt) ** 2, axis=1)))

    L0 = loss(0.0)

    def richardson(e):
        # one-sided differences d(e) = L' + e L''/2 + O(e^2); 2 d(e) - d(2e) = L' + O(e^2)
        d1, d2 = (loss(e) - L0) / e, (loss(2 * e) - L0) / (2 * e)
        return 2.0 * d1 - d2, d1

    r5, d5 = richardson(1e-5)
    r6, _ = richardson(1e-6)
    assert abs(r5 - r6) < 1e-5 * abs(r5)
    assert abs(d5 - r5) > 10.0 * abs(r5 - r6)   # the step's own error is the linear term
    assert abs(r5) > 1e-2 * L0
