"""CPU checks of the C ABI library: it loads, exports every function the
headers declare, and its host-compiled face solvers agree with the oracle."""
import os
import re
import ctypes

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fvmod():
    from paper_1806_04960_gb300 import build
    build.build()
    from paper_1806_04960_gb300 import fv
    return fv


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        txt = open(os.path.join(inc, f)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(fv_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol(fvmod):
    lib = ctypes.CDLL(fvmod.LIB_PATH)
    decl = declared_functions()
    assert {"fv_create", "fv_set_state", "fv_step", "fv_get_state", "fv_destroy"} <= decl
    for name in decl:
        assert hasattr(lib, name), name
    assert set(fvmod.ABI_SYMBOLS) == decl


def test_version_and_error_strings(fvmod):
    assert "sm_103a" in fvmod.fv_version()
    assert isinstance(fvmod.fv_last_error(), str)


def test_host_face_solvers_match_oracle(fvmod):
    from oracle import oracle as O
    from test_oracle_pins import random_states
    model = np.array([1000.0, 4.36e5, 1.0, 9.81, 1e-3])
    worst_x = worst_y = 0.0
    for qa, qb in zip(random_states(100, 1, alpha_lo=0.001, vmax=20),
                      random_states(100, 2, alpha_lo=0.001, vmax=20)):
        Dm, Dp = fvmod.fv_host_xface(qa, qb, model)
        Om, Op = O.dfluct_x(qa, qb)
        scale = np.abs(np.concatenate([Om, Op])).max()
        worst_x = max(worst_x, np.abs(np.concatenate([Dm - Om, Dp - Op])).max() / scale)
        rhoE = 1000.3
        fa = qa - np.array([qa[3] * rhoE, 0, 0, qa[3]])
        fb = qb - np.array([qb[3] * rhoE, 0, 0, qb[3]])
        Dm, Dp = fvmod.fv_host_yface(qa, qb, model)
        Om, Op = O.dfluct_y(fa, qa[3], fb, qb[3], rhoE)
        scale = np.abs(np.concatenate([Om, Op])).max()
        worst_y = max(worst_y, np.abs(np.concatenate([Dm - Om, Dp - Op])).max() / scale)
    assert worst_x < 1e-12 and worst_y < 1e-12, (worst_x, worst_y)


def test_host_face_solvers_vanish_for_equal_states(fvmod):
    from test_oracle_pins import random_states
    model = np.array([1000.0, 4.36e5, 1.0, 9.81, 1e-3])
    for q in random_states(20, 5):
        for fun in (fvmod.fv_host_xface, fvmod.fv_host_yface):
            Dm, Dp = fun(q, q, model)
            assert np.all(Dm == 0) and np.all(Dp == 0)


def test_host_face_null_pointer_is_einval(fvmod):
    lib = ctypes.CDLL(fvmod.LIB_PATH)
    lib.fv_host_xface.restype = ctypes.c_int
    assert lib.fv_host_xface(None, None, None, None, None) == 1


def test_cell_operation_counts(fvmod):
    """The algorithmic counts of one cell-update that the benchmark's roofline
    uses: a first-order cell (the order switch) needs a strict subset of a
    second-order cell's work (no slopes, limiter or predictor), and with gamma
    = 1 (c constant) neither takes a square root."""
    so = fvmod.fv_host_cell_ops()
    fo = fvmod.fv_host_cell_ops(first_order=True)
    assert so["sqrt"] == 0 and fo["sqrt"] == 0
    assert 0 < fo["flops"] < so["flops"]
    for k in ("add", "mul", "div", "cmp"):
        assert 0 < fo[k] < so[k], k
    assert so["flops"] == so["add"] + so["mul"] + so["div"] + so["sqrt"]
    lib = ctypes.CDLL(fvmod.LIB_PATH)
    lib.fv_host_cell_ops_first_order.restype = ctypes.c_int
    assert lib.fv_host_cell_ops_first_order(None) == 1
