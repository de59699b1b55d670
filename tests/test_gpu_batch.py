"""Batched ensemble (fv_batch_*) against the single-domain path and the oracle.

Each domain of an ensemble runs the same per-tile arithmetic with its own dt;
the batched and single-domain kernels are separate instantiations whose
roundoff may differ, so the comparison is at CFL 0.45 (where roundoff is not
amplified) with the parity tolerances: 1e-12 relative (FP64), 1e-5 (FP32)."""
import numpy as np
import pytest

from paper_1806_04960_gb300 import cases
from oracle import oracle as O

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


def small_ensemble():
    doms = cases.weir_domains(count=5, seed=77, nmin=40, nmax=150)
    doms.append(cases.c1())
    doms.append(cases.perturbed(cases.dambreak(33, 17, lx=1.0, ly=0.5, x_col=0.3), 5))
    return doms


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_equals_single_domain_runs(fv, prec):
    doms = small_ensemble()
    b = fv.Batch(doms, prec)
    for k, c in enumerate(doms):
        b.set_state(k, c.q)
    b.step(7, 0.45)
    b.step(6, 0.45)
    tol = 1e-12 if prec == 0 else 1e-5
    for k, c in enumerate(doms):
        s = fv.Solver(c, prec)
        s.set_state(c.q)
        s.step(13, 0.45)
        ref = s.get_state()
        dref = s.diag()
        s.close()
        got = b.get_state(k)
        dg = b.diag(k)
        for v in range(4):
            scale = np.abs(ref[v]).max() or 1.0
            assert np.abs(got[v] - ref[v]).max() <= tol * scale, (k, v)
        assert abs(dg.t - dref.t) <= tol * dref.t and dg.steps == 13 and dg.status == 0
    ts = {b.diag(k).t for k in range(len(doms))}
    assert len(ts) > 1          # per-domain dt
    b.close()


def test_batch_domain_matches_oracle(fv):
    doms = small_ensemble()
    b = fv.Batch(doms, fv.FV_FP64)
    for k, c in enumerate(doms):
        b.set_state(k, c.q)
    b.step(20, 0.45)
    for k in (0, 5):
        qo, to, _, _ = O.run(doms[k], 20, cfl=0.45)
        got = b.get_state(k)
        for v in range(4):
            scale = np.abs(qo[v]).max() or 1.0
            assert np.abs(got[v] - qo[v]).max() <= 1e-10 * scale
        assert abs(b.diag(k).t - to) <= 1e-12 * to
    b.close()


def test_batch_rejects_bad_input(fv):
    doms = small_ensemble()[:2]
    b = fv.Batch(doms, fv.FV_FP64)
    b.set_state(0, doms[0].q)
    with pytest.raises(fv.FvError):
        b.step(1, 0.9)            # domain 1 has no state
    with pytest.raises(fv.FvError):
        b.set_state(5, doms[0].q)
    b.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_tune_keeps_state_and_results(fv, prec):
    """fv_batch_tune leaves every domain's state, time and levels as they were,
    and the tuned batch steps to the same bits as an untuned one (the work
    list changes the speed only)."""
    doms = small_ensemble()
    a, b = fv.Batch(doms, prec), fv.Batch(doms, prec)
    for k, c in enumerate(doms):
        a.set_state(k, c.q)
        b.set_state(k, c.q)
    a.step(3, 0.45)
    b.step(3, 0.45)
    before = [a.get_state(k) for k in range(len(doms))]
    t_before = [a.diag(k).t for k in range(len(doms))]
    rows, order, pers = a.tune(0.45)
    assert rows in (32, 48, 64, 96, 128, 160, 192, 256) and order in (0, 1) and pers in (0, 1)
    for k in range(len(doms)):
        assert np.array_equal(a.get_state(k), before[k])
        assert a.diag(k).t == t_before[k] and a.diag(k).steps == 3
    a.step(5, 0.45)
    b.step(5, 0.45)
    for k in range(len(doms)):
        assert np.array_equal(a.get_state(k), b.get_state(k)), k
        assert a.diag(k).t == b.diag(k).t
    a.close()
    b.close()


def test_batch_tune_needs_states(fv):
    doms = small_ensemble()
    b = fv.Batch(doms, 1)
    b.set_state(0, doms[0].q)
    with pytest.raises(fv.FvError):
        b.tune(0.45)
    for k, c in enumerate(doms):
        b.set_state(k, c.q)
    with pytest.raises(fv.FvError):
        b.tune(1.5)
    b.close()


def test_batch_full_size_sampled_step(fv):
    """The benchmark's ensemble at full size (256 weir domains, 77.8 M cells,
    FP32) in the launch configuration it times (work list from
    fv_batch_tune): 5 ensemble steps, tune, one more step; for 8 seeded
    domains the oracle recomputes that step at sampled cells (random, next to
    the weir, on strip column and block row edges) from the GPU's state, with
    the domain's own dt.  Bounds as for the single-domain FP32 full-size
    check: 1e-6 (alpha rho, alpha), 1e-4 (momenta) of each component's
    largest value."""
    doms = cases.weir_domains()
    b = fv.Batch(doms, fv.FV_FP32_DEV)
    for k, c in enumerate(doms):
        b.set_state(k, c.q)
    b.step(5, 0.9)
    b.tune(0.9)
    rng = np.random.Generator(np.random.PCG64(4961))
    ks = rng.choice(len(doms), 8, replace=False)
    before = {int(k): b.get_state(int(k)) for k in ks}
    b.step(1, 0.9)
    after = {int(k): b.get_state(int(k)) for k in ks}
    b.close()
    tol = [1e-6, 1e-4, 1e-4, 1e-6]
    for k in ks:
        k = int(k)
        c = doms[k]
        fl = c.solid.ravel() == 0
        fluid = np.flatnonzero(fl)
        picks = [rng.choice(fluid, min(400, fluid.size), replace=False)]
        sol = c.solid.astype(bool)
        near = np.zeros_like(sol)
        near[:, 1:] |= sol[:, :-1]
        near[:, :-1] |= sol[:, 1:]
        near[1:, :] |= sol[:-1, :]
        near &= ~sol
        picks.append(np.flatnonzero(near.ravel()))
        cols = np.concatenate([np.arange(31, c.nx, 32), np.arange(0, c.nx, 32)])
        rows = np.concatenate([np.arange(7, c.ny, 8), np.arange(0, c.ny, 8)])
        jj, ii = np.meshgrid(rows, cols, indexing="ij")
        cand = (jj * c.nx + ii).ravel()
        cand = cand[fl[cand]]
        picks.append(rng.choice(cand, min(300, cand.size), replace=False))
        cells = np.unique(np.concatenate(picks))
        ref, _ = O.step_cells(c, before[k], cells, cfl=0.9)
        got = after[k].reshape(4, -1)[:, cells].T
        for v in range(4):
            scale = np.abs(ref[:, v]).max()
            err = np.abs(got[:, v] - ref[:, v]).max() / (scale if scale > 0 else 1.0)
            assert err <= tol[v], (k, v, err)


def test_batch_launch_forms_give_the_same_bits(fv):
    """Every strip height, work order and launch form (fv_batch_set_launch)
    steps the ensemble to the same bits: the per-cell arithmetic does not
    depend on which CTA takes a strip."""
    doms = small_ensemble()
    ref = None
    for rows, order, pers in ((128, 0, 1), (128, 0, 0), (32, 1, 0), (256, 1, 1), (48, 0, 0)):
        b = fv.Batch(doms, 1)
        b.set_launch(rows, order, pers)
        for k, c in enumerate(doms):
            b.set_state(k, c.q)
        b.step(6, 0.45)
        got = [b.get_state(k) for k in range(len(doms))]
        b.close()
        if ref is None:
            ref = got
        else:
            for k in range(len(doms)):
                assert np.array_equal(got[k], ref[k]), (rows, order, pers, k)
    b = fv.Batch(doms, 1)
    for bad in ((0, 0, 1), (12, 0, 1), (32, 2, 1), (32, 0, 2)):
        with pytest.raises(fv.FvError):
            b.set_launch(*bad)
    b.close()
