"""The FP32 face solvers in the paired form the FP32 step kernels run (two
quadrature nodes or Romberg terms per float2 operation) against the scalar
float form and the double solver, evaluated on the host (fv_host_face_f32):
the same arithmetic in float rounding.

Bounds, relative to the largest |D-|, |D+| of the double solver on the
float-rounded states: paired vs scalar float 2e-6 (measured 5e-7 over 300
seeded pairs), each vs double 5e-6 (measured 1.2e-6).  Equal states and a
column at rest give exact zeros in both forms, the property that keeps the
FP32 lakes at rest exact.
"""
import numpy as np
import pytest

from test_oracle_pins import random_states

MODEL = np.array([1000.0, 4.36e5, 1.0, 9.81, 1e-3])


@pytest.fixture(scope="module")
def fvmod():
    from paper_1806_04960_gb300 import build
    build.build()
    from paper_1806_04960_gb300 import fv
    return fv


def f32(q):
    return np.asarray(q, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("which", [0, 1])
def test_paired_form_matches_scalar_and_double(fvmod, which):
    ref = fvmod.fv_host_xface if which == 0 else fvmod.fv_host_yface
    worst_ps = worst_pd = worst_sd = 0.0
    for qa, qb in zip(random_states(300, 1, alpha_lo=0.001, vmax=20),
                      random_states(300, 2, alpha_lo=0.001, vmax=20)):
        Pm, Pp = fvmod.fv_host_face_f32(which, qa, qb, MODEL, True)
        Sm, Sp = fvmod.fv_host_face_f32(which, qa, qb, MODEL, False)
        Dm, Dp = ref(f32(qa), f32(qb), MODEL)
        scale = np.abs(np.concatenate([Dm, Dp])).max()
        worst_ps = max(worst_ps, np.abs(np.concatenate([Pm - Sm, Pp - Sp])).max() / scale)
        worst_pd = max(worst_pd, np.abs(np.concatenate([Pm - Dm, Pp - Dp])).max() / scale)
        worst_sd = max(worst_sd, np.abs(np.concatenate([Sm - Dm, Sp - Dp])).max() / scale)
    assert worst_ps < 2e-6, worst_ps
    assert worst_pd < 5e-6 and worst_sd < 5e-6, (worst_pd, worst_sd)


@pytest.mark.parametrize("paired", [True, False])
def test_equal_states_and_rest_give_exact_zeros(fvmod, paired):
    for q in random_states(20, 5):
        for which in (0, 1):
            Dm, Dp = fvmod.fv_host_face_f32(which, q, q, MODEL, paired)
            assert np.all(Dm == 0) and np.all(Dp == 0)
    # a column at rest: u = v = 0 and a jump of alpha p that vanishes
    # (d(alpha rho) = rho0 d(alpha), exact in float)
    for m, a in ((812.5, 0.8125), (1000.0, 1.0), (3.0, 0.00390625)):
        da = 2.0 ** -6
        qa = np.array([m, 0.0, 0.0, a])
        qb = np.array([m + 1000.0 * da, 0.0, 0.0, a + da])
        Dm, Dp = fvmod.fv_host_face_f32(1, qa, qb, MODEL, paired)
        assert np.all(Dm == 0) and np.all(Dp == 0), (Dm, Dp)


def test_bad_arguments(fvmod):
    with pytest.raises(fvmod.FvError):
        fvmod.fv_host_face_f32(2, np.ones(4), np.ones(4), MODEL)
