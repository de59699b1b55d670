"""ctypes wrapper and build step for the FP64 CPU oracle (fv_oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
timed CPU baseline.  The product library never imports or calls it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fv_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)
_U8 = C.POINTER(C.c_uint8)


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (plain g++, OpenMP over rows).

    -ffp-contract=off keeps the arithmetic identical on x86-64 and AArch64."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            L.orc_run.argtypes = [_I32, _D, _D, _I32, _U8, _D, _D, C.c_int, C.c_double, _D, _D, _I32]
            L.orc_run.restype = C.c_int
            L.orc_dt_levels.argtypes = [_I32, _D, _D, _I32, _U8, _D, C.c_double, _D, _I32]
            L.orc_dt_levels.restype = C.c_int
            L.orc_step_cells.argtypes = [_I32, _D, _D, _I32, _U8, _D, C.c_double, _I64, C.c_int,
                                         _D, _D]
            L.orc_step_cells.restype = C.c_int
            L.orc_run_record.argtypes = [_I32, _D, _D, _I32, _U8, _D, _D, C.c_int, C.c_double,
                                         _D, _I32, _D, _I32, _I64, C.c_int, _D, C.c_int, _D]
            L.orc_dfluct_x_or.argtypes = [_D, _D, _D, _D, _D]
            L.orc_sign_A1_apply.argtypes = [_D, _D, _D, _D]
            L.orc_dfluct_y_o1.argtypes = [_D, _D, C.c_double, _D, C.c_double, C.c_double,
                                          C.c_double, C.c_double, _D, _D]
            L.orc_run_record.restype = C.c_int
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_max_threads.restype = C.c_int
            L.orc_flux.argtypes = [_D, _D, _D, _D]
            L.orc_cell_rec.argtypes = [_I32, _D, _D, _I32, _U8, _D, C.c_double, C.c_int, C.c_int, _D]
            L.orc_cell_rec.restype = C.c_int
            L.orc_jacobians.argtypes = [_D, _D, _D, _D]
            L.orc_eigen.argtypes = [_D, _D, C.c_int, _D, _D, _D]
            L.orc_abs_A1_apply.argtypes = [_D, _D, _D, _D]
            L.orc_sign_A2_apply.argtypes = [_D, _D, _D, _D]
            L.orc_dfluct_x.argtypes = [_D, _D, _D, _D, _D]
            L.orc_dfluct_y.argtypes = [_D, _D, C.c_double, _D, C.c_double, C.c_double, _D, _D]
            _lib = L
    return _lib


def _p(a, t=_D):
    return a.ctypes.data_as(t)


def _case_args(case):
    gi = np.array([case.nx, case.ny], dtype=np.int32)
    gd = np.array([case.x0, case.y0, case.dx, case.dy], dtype=np.float64)
    eos = np.array([case.rho0, case.k0, case.gamma, case.g, case.eps], dtype=np.float64)
    sides = np.array(case.sides, dtype=np.int32)
    solid = np.ascontiguousarray(case.solid, dtype=np.uint8)
    return gi, gd, eos, sides, solid


class OracleError(RuntimeError):
    pass


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().orc_max_threads())


def run(case, nsteps: int, q=None, cfl: float | None = None):
    """Advance ``nsteps`` steps.  Returns (q_out (4,ny,nx), t, dt history, K of last step)."""
    L = lib()
    gi, gd, eos, sides, solid = _case_args(case)
    qin = np.ascontiguousarray(case.q if q is None else q, dtype=np.float64)
    qout = np.empty_like(qin)
    t = np.zeros(1)
    dts = np.zeros(max(nsteps, 1))
    K = np.zeros(case.nx, dtype=np.int32)
    rc = L.orc_run(_p(gi, _I32), _p(gd), _p(eos), _p(sides, _I32), _p(solid, _U8), _p(qin),
                   _p(qout), int(nsteps), float(case.cfl if cfl is None else cfl), _p(t), _p(dts),
                   _p(K, _I32))
    if rc == 1:
        raise OracleError("invalid input")
    if rc == 2:
        raise OracleError("non-admissible state (non-finite, alpha <= 0 or alpha*rho <= 0)")
    return qout, float(t[0]), dts[:nsteps], K


def run_record(case, nsteps: int, gauges, q=None, cfl: float | None = None, dt_fix=None,
               K_fix=None, order: int = 2, xsolver: int = 0, cap=None, roe: bool = False,
               bj_printed: bool = False, no_pos: bool = False, aE_mode: int = 0):
    """Advance ``nsteps`` steps of the scheme of ``order`` (2: Eq. (Scheme);
    1: the first-order scheme of Sections 3.2-3.3) with x faces by
    ``xsolver`` (0: Gauss-Legendre Osher; 1: conservative Osher-Romberg,
    Eq. (OR_cons)), recording each step's dt,
    levels and the alpha rho at the flat gauge cells after it.  With
    ``dt_fix`` (nsteps) and ``K_fix`` (nsteps, nx) the steps use those instead
    of their own.  ``cap`` (ny, nx), second order only: the fluid capacities
    of reading R-h (a partial cell on top of an obstacle; 1 = a whole cell).
    ``roe`` (second order, Gauss-Legendre x faces): the printed sqrt(rho)-
    weighted Roe averages of Eqs. (b_4^x), (b_4^y) in place of reading R-vel;
    ``bj_printed``: the printed Barth-Jespersen factor (no ramp, reading R-bj);
    ``no_pos``: no first-order fallback of reading R-pos; ``aE_mode`` 1 / 2:
    alpha^E = 1 / two-layer (1 below the level, eps above) instead of reading
    R-eq.  These switches exist for experiments and tests of the readings.
    Returns (q_out, dt (nsteps), K (nsteps, nx), m (nsteps, ngauges))."""
    L = lib()
    gi, gd, eos, sides, solid = _case_args(case)
    qin = np.ascontiguousarray(case.q if q is None else q, dtype=np.float64)
    qout = np.empty_like(qin)
    g = np.ascontiguousarray(gauges, dtype=np.int64)
    n = max(nsteps, 1)
    dts = np.zeros(n)
    Ks = np.zeros((n, case.nx), dtype=np.int32)
    ms = np.zeros((n, max(g.size, 1)))
    if (dt_fix is None) != (K_fix is None):
        raise ValueError("give both dt_fix and K_fix or neither")
    dfix = None if dt_fix is None else np.ascontiguousarray(dt_fix, dtype=np.float64)
    kfix = None if K_fix is None else np.ascontiguousarray(K_fix, dtype=np.int32)
    cp = None if cap is None else np.ascontiguousarray(cap, dtype=np.float64)
    if cp is not None and cp.shape != (case.ny, case.nx):
        raise ValueError("cap must be (ny, nx)")
    rc = L.orc_run_record(_p(gi, _I32), _p(gd), _p(eos), _p(sides, _I32), _p(solid, _U8),
                          _p(qin), _p(qout), int(nsteps), float(case.cfl if cfl is None else cfl),
                          None if dfix is None else _p(dfix),
                          None if kfix is None else _p(kfix, _I32), _p(dts), _p(Ks, _I32),
                          _p(g, _I64), int(g.size), _p(ms), (int(order) | (int(xsolver) << 4) | (int(bool(roe)) << 5)
                           | (int(bool(bj_printed)) << 6) | (int(bool(no_pos)) << 7)
                           | (int(aE_mode) << 8)),
                          None if cp is None else _p(cp))
    if rc == 1:
        raise OracleError("invalid input")
    if rc == 2:
        raise OracleError("non-admissible state (non-finite, alpha <= 0 or alpha*rho <= 0)")
    return qout, dts[:nsteps], Ks[:nsteps], ms[:nsteps, :g.size]


def dt_levels(case, q=None, cfl: float | None = None):
    L = lib()
    gi, gd, eos, sides, solid = _case_args(case)
    qin = np.ascontiguousarray(case.q if q is None else q, dtype=np.float64)
    dt = np.zeros(1)
    K = np.zeros(case.nx, dtype=np.int32)
    rc = L.orc_dt_levels(_p(gi, _I32), _p(gd), _p(eos), _p(sides, _I32), _p(solid, _U8), _p(qin),
                         float(case.cfl if cfl is None else cfl), _p(dt), _p(K, _I32))
    if rc:
        raise OracleError("invalid input")
    return float(dt[0]), K


def step_cells(case, q, cells, cfl: float | None = None):
    """One step of state ``q`` evaluated only at flat cell indices ``cells``
    (j*nx + i).  Returns (values (len(cells), 4), dt)."""
    L = lib()
    gi, gd, eos, sides, solid = _case_args(case)
    qin = np.ascontiguousarray(q, dtype=np.float64)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    out = np.zeros((len(cells), 4))
    dt = np.zeros(1)
    rc = L.orc_step_cells(_p(gi, _I32), _p(gd), _p(eos), _p(sides, _I32), _p(solid, _U8), _p(qin),
                          float(case.cfl if cfl is None else cfl), _p(cells, _I64), len(cells),
                          _p(out), _p(dt))
    if rc == 1:
        raise OracleError("invalid input")
    return out, float(dt[0])


def cell_rec(case, q, i: int, j: int, cfl: float | None = None) -> dict:
    """Reconstructed face, centre and slope data of fluid cell (i, j)."""
    L = lib()
    gi, gd, eos, sides, solid = _case_args(case)
    qin = np.ascontiguousarray(q, dtype=np.float64)
    out = np.zeros(27)
    rc = L.orc_cell_rec(_p(gi, _I32), _p(gd), _p(eos), _p(sides, _I32), _p(solid, _U8), _p(qin),
                        float(case.cfl if cfl is None else cfl), int(i), int(j), _p(out))
    if rc:
        raise OracleError("invalid input or non-fluid cell")
    return dict(qW=out[0:4], qE=out[4:8], fS=out[8:12], fN=out[12:16], qc=out[16:20],
                aE=out[20], rhoES=out[21], rhoEN=out[22], rhoEc=out[23], dax=out[24],
                day=out[25], dt=out[26])


# ---- pieces for the pin tests -------------------------------------------------

def _model(rho0=1000.0, k0=4.36e5, gamma=1.0, g=9.81, eps=1e-3):
    return np.array([rho0, k0, gamma, g, eps], dtype=np.float64)


def flux(q, **m):
    f, g = np.zeros(5), np.zeros(5)
    lib().orc_flux(_p(_model(**m)), _p(np.ascontiguousarray(q, dtype=np.float64)), _p(f), _p(g))
    return f, g


def jacobians(q, **m):
    A1, A2 = np.zeros(25), np.zeros(25)
    lib().orc_jacobians(_p(_model(**m)), _p(np.ascontiguousarray(q, dtype=np.float64)), _p(A1), _p(A2))
    return A1.reshape(5, 5), A2.reshape(5, 5)


def eigen(q, direction: int, **m):
    R, L, Ri = np.zeros(25), np.zeros(5), np.zeros(25)
    lib().orc_eigen(_p(_model(**m)), _p(np.ascontiguousarray(q, dtype=np.float64)), int(direction), _p(R),
                    _p(L), _p(Ri))
    return R.reshape(5, 5), L, Ri.reshape(5, 5)


def abs_A1_apply(q, x, **m):
    out = np.zeros(5)
    lib().orc_abs_A1_apply(_p(_model(**m)), _p(np.ascontiguousarray(q, dtype=np.float64)),
                           _p(np.ascontiguousarray(x, dtype=np.float64)), _p(out))
    return out


def sign_A2_apply(q, x, **m):
    out = np.zeros(5)
    lib().orc_sign_A2_apply(_p(_model(**m)), _p(np.ascontiguousarray(q, dtype=np.float64)),
                            _p(np.ascontiguousarray(x, dtype=np.float64)), _p(out))
    return out


def dfluct_x(qm, qp, **m):
    Dm, Dp = np.zeros(4), np.zeros(4)
    lib().orc_dfluct_x(_p(_model(**m)), _p(np.ascontiguousarray(qm, dtype=np.float64)),
                       _p(np.ascontiguousarray(qp, dtype=np.float64)), _p(Dm), _p(Dp))
    return Dm, Dp


def dfluct_x_or(qm, qp, **m):
    """x-face fluctuations with the conservative Osher-Romberg viscosity."""
    Dm, Dp = np.zeros(4), np.zeros(4)
    lib().orc_dfluct_x_or(_p(_model(**m)), _p(np.ascontiguousarray(qm, dtype=np.float64)),
                          _p(np.ascontiguousarray(qp, dtype=np.float64)), _p(Dm), _p(Dp))
    return Dm, Dp


def sign_A1_apply(q, x, **m):
    out = np.zeros(5)
    lib().orc_sign_A1_apply(_p(_model(**m)), _p(np.ascontiguousarray(q, dtype=np.float64)),
                            _p(np.ascontiguousarray(x, dtype=np.float64)), _p(out))
    return out


def dfluct_y_o1(fa, aEa, fb, aEb, ya, dy, pE_face, **m):
    """First-order y-face fluctuations between two cell centres (reading R-o1)."""
    Dm, Dp = np.zeros(4), np.zeros(4)
    lib().orc_dfluct_y_o1(_p(_model(**m)), _p(np.ascontiguousarray(fa, dtype=np.float64)),
                          float(aEa), _p(np.ascontiguousarray(fb, dtype=np.float64)), float(aEb),
                          float(ya), float(dy), float(pE_face), _p(Dm), _p(Dp))
    return Dm, Dp


def dfluct_y(fm, aEm, fp, aEp, rhoE, **m):
    Dm, Dp = np.zeros(4), np.zeros(4)
    lib().orc_dfluct_y(_p(_model(**m)), _p(np.ascontiguousarray(fm, dtype=np.float64)), float(aEm),
                       _p(np.ascontiguousarray(fp, dtype=np.float64)), float(aEp), float(rhoE), _p(Dm),
                       _p(Dp))
    return Dm, Dp
