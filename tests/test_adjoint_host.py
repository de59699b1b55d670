"""Reverse-mode building blocks of fv_adjoint against central finite differences.

Each per-face and per-cell function of the kernels (x face, y face, the
Section 3.4 reconstruction, the interior integral) is evaluated on the host
through fv_host_adj_check; its reverse derivative d<lout, out>/d in, with every
branch held as at the input, must equal the central difference quotient of
the forward function.  Inputs are chosen away from the branch boundaries, so
the finite difference sees one smooth piece; each branch of the
reconstruction (limiter active, limiter ramp, order switch, first-order
fallback) is exercised and identified from the outputs.
"""
import math

import numpy as np
import pytest

from paper_1806_04960_gb300 import fv

MODEL = [1000.0, 4.36e5, 1.0, 9.81, 1e-3]
DX = 1.0 / 32.0
KAPPA = 9.81 * 1000.0 / 4.36e5
# dx, dy, dt, rho^E at the centre, the south face and the north face (0.3 m below the level)
K = np.array([DX, DX, 2e-4, 1000 * np.exp(KAPPA * 0.3), 1000 * np.exp(KAPPA * (0.3 + DX / 2)),
              1000 * np.exp(KAPPA * (0.3 - DX / 2))])
FSCALE = np.array([5.0, 300.0, 300.0, 0.05])


def central_fd(which, k, x, lout, rel, scale):
    g = np.zeros_like(x)
    for i in range(x.size):
        h = rel * max(abs(x[i]), scale[i])
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        g[i] = (lout @ fv.fv_host_adj_check(which, MODEL, k, xp)
                - lout @ fv.fv_host_adj_check(which, MODEL, k, xm)) / (2 * h)
    return g


def rel_err(g, lin):
    return np.max(np.abs(g - lin)) / np.max(np.abs(lin))


def face_state(rng):
    q = np.array([rng.uniform(100, 1100), rng.normal() * 300, rng.normal() * 300, 0.0])
    q[3] = q[0] / rng.uniform(900, 1100)
    return q


def supersonic_pair(rng):
    """Two face states whose velocities are both supersonic in x and in y
    (1.3 c .. 2 c, one sign per direction), so every path node is too: the
    general branch of |A1| and sign(A2) rather than their subsonic closed
    forms."""
    c = math.sqrt(MODEL[1] / MODEL[0])
    sx, sy = rng.choice([-1.0, 1.0], 2)
    out = []
    for _ in range(2):
        m = rng.uniform(300, 1100)
        q = np.array([m, sx * m * c * rng.uniform(1.3, 2.0), sy * m * c * rng.uniform(1.3, 2.0),
                      m / rng.uniform(900, 1100)])
        out.append(q)
    return np.concatenate(out)


@pytest.mark.parametrize("speed", ["subsonic", "supersonic"])
@pytest.mark.parametrize("which", [0, 1])
def test_face_adjoints_match_central_differences(which, speed):
    rng = np.random.default_rng(100 + which + (10 if speed == "supersonic" else 0))
    for _ in range(6):
        if speed == "subsonic":
            x = np.concatenate([face_state(rng), face_state(rng)])
        else:
            x = supersonic_pair(rng)
        lout = rng.normal(size=8)
        _, lin = fv.fv_host_adj_check(which, MODEL, None, x, lout)
        g = central_fd(which, None, x, lout, 1e-6, np.ones(8))
        assert rel_err(g, lin) < 1e-8


def test_face_adjoint_sign_of_zero_velocity_is_zero():
    """At rest (u = v = 0 on the whole path) |u| and sign(v) have no derivative;
    the reverse pass takes sign(0) = 0, the value the symmetric quotient gives."""
    q = np.array([1000.0, 0.0, 0.0, 1.0])
    x = np.concatenate([q, q])
    lout = np.arange(1.0, 9.0)
    for which in (0, 1):
        _, lin = fv.fv_host_adj_check(which, MODEL, None, x, lout)
        g = central_fd(which, None, x, lout, 1e-6, np.ones(8))
        assert np.max(np.abs(g - lin)) <= 1e-7 * np.max(np.abs(lin))


def recon_input(rng, aE, big=1.0, spread=1.0, margin=0.02):
    sc = FSCALE * np.array([big, spread, spread, spread])
    Qf = np.array([rng.normal() * sc[0], rng.normal() * sc[1], rng.normal() * sc[2], 0.0])
    nb = [rng.normal(size=4) * sc for _ in range(8)]
    cand = np.array([Qf] + nb)
    # strict bounds: min/max of the stencil pushed outward, so no two limiter
    # candidates tie (in the kernels the bound follows its extremal cell)
    mx = cand.max(axis=0) + np.abs(rng.normal(size=4)) * sc * margin
    mn = cand.min(axis=0) - np.abs(rng.normal(size=4)) * sc * margin
    return np.concatenate([Qf] + nb[:4] + [mx, mn, [aE]])


RSCALE = np.concatenate([np.tile([5.0, 300.0, 300.0, 1.0], 7), [1.0]])


def check_recon(x, rng, rel=1e-7, tol=5e-6):
    lout = rng.normal(size=22)
    out, lin = fv.fv_host_adj_check(2, MODEL, K, x, lout)
    g = central_fd(2, K, x, lout, rel, RSCALE)
    assert rel_err(g, lin) < tol
    return out


def test_recon_adjoint_limiter_active():
    rng = np.random.default_rng(7)
    for _ in range(6):
        x = recon_input(rng, aE=rng.uniform(0.3, 1.0))
        out = check_recon(x, rng)
        base, faceW = out[16:20], out[0:4]
        assert np.any(faceW != base)                     # second order
        psi_g = (out[4:8] - base) / (0.5 * DX)          # psi * gx
        gx = (x[8:12] - x[4:8]) / (2 * DX)
        assert 0.0 < np.max(np.abs(psi_g)) < np.max(np.abs(gx))  # psi < 1


def test_recon_adjoint_limiter_ramp():
    """Face increments between eta and 2 eta: the limiter factor is on its ramp."""
    rng = np.random.default_rng(8)
    eta_m = 1000.0 * 2.0 ** -20
    for _ in range(4):
        x = np.zeros(29)
        # only alpha rho varies: |d| = |fE - fW| / 4 within (eta, 2 eta)
        x[4] = -rng.uniform(1.2, 1.8) * 2 * eta_m
        x[8] = rng.uniform(1.2, 1.8) * 2 * eta_m
        x[12], x[16] = 0.3 * eta_m, -0.2 * eta_m
        x[20], x[24] = 0.6 * eta_m, -0.5 * eta_m    # tight bounds: the printed factor is < 1
        x[28] = 0.9
        check_recon(x, rng, rel=1e-6, tol=5e-6)


def test_recon_adjoint_order_switch():
    """alpha <= 10 eps: Psi = 0 and no predictor; the states are the cell's."""
    rng = np.random.default_rng(9)
    for _ in range(3):
        x = recon_input(rng, aE=0.005)
        out = check_recon(x, rng)
        assert np.all(out[0:4] == x[0:4]) and np.all(out[20:22] == 0.0)


def test_recon_adjoint_first_order_fallback():
    """A non-admissible reconstructed state: every output state is Qf."""
    rng = np.random.default_rng(10)
    for _ in range(3):
        x = recon_input(rng, aE=0.02, big=20.0)
        x[4], x[8] = -40.0, 40.0     # alpha rho slope large enough to make a face negative
        x[20], x[24] = 60.0, -60.0
        out = check_recon(x, rng)
        for s in range(5):
            assert np.all(out[4 * s:4 * s + 4] == x[0:4])


def test_interior_adjoint_matches_central_differences():
    rng = np.random.default_rng(11)
    for _ in range(6):
        f = [rng.normal(size=4) * FSCALE for _ in range(5)]
        x = np.concatenate(f + [[rng.uniform(0.3, 1.0), rng.normal() * 0.1, rng.normal() * 0.1]])
        lout = rng.normal(size=8)
        _, lin = fv.fv_host_adj_check(3, MODEL, K, x, lout)
        g = central_fd(3, K, x, lout, 1e-7, np.concatenate([np.tile(FSCALE, 5), [1, 1, 1]]))
        assert rel_err(g, lin) < 1e-7


def test_host_reverse_sweep_matches_oracle_differences():
    """The reverse sweep of fv_adjoint, run on the host with the kernels' own
    per-cell and per-face code (fv_host_adjoint_step) along the oracle's
    trajectory, against central differences of the oracle's gauge loss with the
    oracle's dt and levels held fixed.  Generic state (no exact ties), so the
    frozen-branch map is differentiable there.  Then the float instantiation
    (the FP32 path's arithmetic) along the same trajectory against double."""
    import ctypes as C
    from oracle import oracle as O
    from paper_1806_04960_gb300 import cases
    L = fv._lib
    L.fv_host_adjoint_step.argtypes = [C.POINTER(fv.fv_grid), C.POINTER(fv.fv_eos),
                                       C.POINTER(C.c_int32), C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_double, C.c_void_p, C.c_void_p, C.c_int]
    c = cases.generic(cases.c5(32, 16, cfl=0.45), 7)
    grid = fv.fv_grid(c.nx, c.ny, c.x0, c.y0, c.dx, c.dy)
    eos = fv.fv_eos(c.rho0, c.k0, c.gamma, c.g, c.eps)
    side = (C.c_int32 * 4)(*c.sides)
    solid = np.ascontiguousarray(c.solid, dtype=np.uint8)

    def reverse_step(q, K, dt, lam, prec=fv.FV_FP64):
        q = np.ascontiguousarray(q)
        K = np.ascontiguousarray(K, dtype=np.int32)
        lam = np.ascontiguousarray(lam)
        out = np.zeros_like(lam)
        assert L.fv_host_adjoint_step(C.byref(grid), C.byref(eos), side, solid.ctypes.data,
                                      q.ctypes.data, K.ctypes.data, float(dt), lam.ctypes.data,
                                      out.ctypes.data, prec) == 0
        return out

    nsteps = 24
    gauges = cases.c5_gauges(c, count=8)
    _, _, _, target = O.run_record(cases.c5_target(32, 16), nsteps, gauges, cfl=0.45)
    states, dts, Ks, ms = [c.q], [], [], []
    for _ in range(nsteps):
        q1, dt, K, m = O.run_record(c, 1, gauges, q=states[-1], cfl=0.45)
        states.append(q1)
        dts.append(dt[0])
        Ks.append(K[0])
        ms.append(m[0])
    dts, Ks, ms = np.array(dts), np.array(Ks), np.array(ms)
    lam = np.zeros_like(c.q)
    for n in range(nsteps, 0, -1):
        lam.reshape(4, -1)[0, gauges] += 2.0 * dts[n - 1] * (ms[n - 1] - target[n - 1])
        lam = reverse_step(states[n - 1], Ks[n - 1], dts[n - 1], lam)

    def loss(q):
        _, _, _, m = O.run_record(c, nsteps, gauges, q=q, cfl=0.45, dt_fix=dts, K_fix=Ks)
        return float(np.sum(dts * np.sum((m - target) ** 2, axis=1)))

    for d in cases.c5_directions(c, count=4):
        fd = (loss(c.q + 1e-9 * d) - loss(c.q - 1e-9 * d)) / 2e-9
        assert abs(np.sum(lam * d) - fd) <= 1e-5 * abs(fd)
    assert np.all(lam[:, c.solid == 1] == 0.0)

    # the same sweep in the float arithmetic of the FP32 path (state rounded to
    # the float deviation form), along the same trajectory, against double
    far = np.repeat(c.q[0].ravel()[gauges][None, :] + 500.0, nsteps, axis=0)
    sweeps = {}
    for prec in (fv.FV_FP64, fv.FV_FP32_DEV):
        lam = np.zeros_like(c.q)
        for n in range(nsteps, 0, -1):
            lam.reshape(4, -1)[0, gauges] += 2.0 * dts[n - 1] * (ms[n - 1] - far[n - 1])
            lam = reverse_step(states[n - 1], Ks[n - 1], dts[n - 1], lam, prec)
        sweeps[prec] = lam
    for v, tol in ((0, 1e-5), (1, 1e-5), (2, 1e-5), (3, 1e-3)):
        a, b = sweeps[fv.FV_FP32_DEV][v], sweeps[fv.FV_FP64][v]
        assert np.sum(np.abs(a - b)) / np.sum(np.abs(b)) < tol, v


def test_host_first_order_y_face_matches_oracle():
    """The kernels' first-order y face (yface_o1, host instantiation) against
    the oracle's (reading R-o1): random fluctuations, volume fractions,
    heights, including the level face."""
    from oracle import oracle as O
    rng = np.random.default_rng(31)
    kap = MODEL[3] * MODEL[0] / MODEL[1]
    for k in range(12):
        dy = 1.0 / 32
        ya = -0.5 * dy if k == 0 else rng.uniform(-0.6, 0.6)
        aEa, aEb = (1.0, 1e-3) if k == 0 else (rng.uniform(0.2, 1.0), rng.uniform(0.2, 1.0))
        fa = np.array([rng.normal() * 5, rng.normal() * 300, rng.normal() * 300, 0.0])
        fb = np.array([rng.normal() * 5, rng.normal() * 300, rng.normal() * 300, 0.0])
        if k % 3 == 1:
            fa[3], fb[3] = rng.normal() * 0.01, rng.normal() * 0.01
        pE_face = MODEL[1] * (math.exp(-kap * (ya + 0.5 * dy)) - 1.0)
        got = fv.fv_host_yface_o1(fa, aEa, fb, aEb, ya, dy, MODEL)
        ref = O.dfluct_y_o1(fa, aEa, fb, aEb, ya, dy, pE_face, rho0=MODEL[0], k0=MODEL[1],
                            g=MODEL[3])
        for a, b in zip(got, ref):
            assert np.allclose(a, b, rtol=1e-11, atol=1e-9 * np.abs(b).max()), (k, a, b)


def test_host_osher_romberg_x_face_matches_oracle():
    """The kernels' xface_or (host instantiation) against the oracle's
    conservative Osher-Romberg x face (Eq. (OR_cons), reading R-orx)."""
    from oracle import oracle as O
    rng = np.random.default_rng(41)
    for _ in range(12):
        qm, qp = face_state(rng), face_state(rng)
        got = fv.fv_host_xface_or(qm, qp, MODEL)
        ref = O.dfluct_x_or(qm, qp, rho0=MODEL[0], k0=MODEL[1], g=MODEL[3])
        for a, b in zip(got, ref):
            assert np.allclose(a, b, rtol=1e-11, atol=1e-9 * np.abs(b).max())


def _host_height_step(c, q, K, dt, lam, hid, prec):
    import ctypes as C
    grid = fv.fv_grid(c.nx, c.ny, c.x0, c.y0, c.dx, c.dy)
    eos = fv.fv_eos(c.rho0, c.k0, c.gamma, c.g, c.eps)
    side = (C.c_int32 * 4)(*c.sides)
    solid = np.ascontiguousarray(c.solid, dtype=np.uint8)
    q = np.ascontiguousarray(q)
    K = np.ascontiguousarray(K, dtype=np.int32)
    lam = np.ascontiguousarray(lam)
    hid = np.ascontiguousarray(hid, dtype=np.int32)
    nh = int(hid.max()) + 1
    out = np.zeros(nh)
    assert fv._lib.fv_host_height_step(C.byref(grid), C.byref(eos), side, solid.ctypes.data,
                                       q.ctypes.data, K.ctypes.data, float(dt), lam.ctypes.data,
                                       hid.ctypes.data, nh, out.ctypes.data, prec) == 0
    return out


def test_host_height_step_matches_oracle_differences():
    """The obstacle-height part of one reverse step (fv_host_height_step, the
    kernel's per-cell code on the host) against the one-sided difference in
    theta of lam . Q^{n+1} from the oracle's partial cells (reading R-h), with
    the step's dt and levels held fixed; Richardson-extrapolated, so the
    difference's own error is O(e^2).  Two obstacles of different heights
    side by side, so that a top cell's neighbour is another obstacle's top
    cell.  Then the float instantiation (FP32 deviation form, lam mapped to
    its storage form) against double."""
    from oracle import oracle as O
    from paper_1806_04960_gb300 import cases
    rects = [cases.H_RECT, (0.92, 1.05, 0.0, 0.3)]
    c0 = cases.dambreak(48, 24, lx=2.0, ly=1.0, x_col=1.2, h_col=0.6, rects=rects, k0=4.36e5,
                        cfl=0.45)
    c = cases.generic(c0, 7)
    hid = cases.height_ids(c)
    assert set(np.unique(hid)) == {-1, 0, 1}
    g = np.array([5], dtype=np.int64)
    q, _, _, _ = O.run_record(c, 6, g, cfl=0.45)     # a state with the water moving
    dt, K = O.dt_levels(c, q=q, cfl=0.45)
    rng = np.random.Generator(np.random.PCG64(41))
    lam = rng.standard_normal(q.shape) * (c.solid == 0)

    def lam_q1(theta, k):
        cap = np.ones((c.ny, c.nx))
        cap[hid == k] = 1.0 - theta
        q1, _, _, _ = O.run_record(c, 1, g, q=q, cfl=0.45, dt_fix=[dt], K_fix=[K], cap=cap)
        return float(np.sum(lam * q1))

    host = _host_height_step(c, q, K, dt, lam, hid, fv.FV_FP64)
    for k in (0, 1):
        base = lam_q1(0.0, k)
        e = 1e-5
        d1 = (lam_q1(e, k) - base) / e
        d2 = (lam_q1(2 * e, k) - base) / (2 * e)
        ref = 2 * d1 - d2
        assert abs(host[k] - ref) < 1e-6 * abs(ref), (k, host[k], ref)
    # float (deviation form): lam on the storage form (m - a rho^E, mu, mv, a)
    rhoE = c.rho0 * np.exp(-c.g * c.rho0 / c.k0 *
                           ((np.arange(c.ny)[:, None] + 0.5) - K[None, :]) * c.dy)
    lam_s = lam.copy()
    lam_s[3] += rhoE * lam[0]
    host32 = _host_height_step(c, q, K, dt, lam_s, hid, fv.FV_FP32_DEV)
    assert np.all(np.abs(host32 - host) < 1e-3 * np.abs(host)), (host32, host)


def test_host_height_step_rejects_bad_maps():
    """The height map is validated as in fv_adjoint: an id outside [-1,
    nheights) or on a cell that is not a fluid cell resting on a solid one."""
    from paper_1806_04960_gb300 import cases
    c = cases.heights()
    hid = cases.height_ids(c)
    lam = np.ones_like(c.q)
    K = np.full(c.nx, 14, dtype=np.int32)
    import ctypes as C
    grid = fv.fv_grid(c.nx, c.ny, c.x0, c.y0, c.dx, c.dy)
    eos = fv.fv_eos(c.rho0, c.k0, c.gamma, c.g, c.eps)
    side = (C.c_int32 * 4)(*c.sides)
    solid = np.ascontiguousarray(c.solid, dtype=np.uint8)
    out = np.zeros(4)

    def call(h, nh):
        h = np.ascontiguousarray(h, dtype=np.int32)
        return fv._lib.fv_host_height_step(C.byref(grid), C.byref(eos), side, solid.ctypes.data,
                                           c.q.ctypes.data, K.ctypes.data, 1e-4, lam.ctypes.data,
                                           h.ctypes.data, nh, out.ctypes.data, fv.FV_FP64)
    assert call(hid, 1) == 0
    bad = hid.copy(); bad[10, 3] = 0          # fluid below
    assert call(bad, 1) == 1
    bad = hid.copy(); bad[0, 20] = 0          # a solid cell
    assert call(bad, 1) == 1
    bad = hid.copy(); bad[bad == 0] = 1       # id >= nheights
    assert call(bad, 1) == 1
    bad = hid.copy(); bad[0, 0] = -2          # id < -1
    assert call(bad, 1) == 1
    assert call(hid, 0) == 1
