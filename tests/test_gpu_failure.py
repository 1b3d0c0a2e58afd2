"""Failure paths, the final-time API and resume, through the C-ABI.

Every failure is made on the host (a NaN written into the state, an iteration
cap too small to converge, a wait limit too short to finish); nothing here
faults or stalls the GPU.  The contract under test (include/hbpc.h): a failed
hbpc_step leaves the state at the last completed step, and a state read out
and written into a new context continues bit for bit like an uninterrupted run.
"""
import numpy as np
import pytest
import torch

from oracle import dgsem, exact, hbpc as ohbpc, laws, newton
from paper_2109_04804_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    import __graft_entry__ as g
    g.build()
    from paper_2109_04804_gb300 import hbpc
    assert torch.cuda.is_available()
    return hbpc


def advection(hb, **kw):
    args = dict(law=hb.LAW_ADVECTION, a=(1.0, 1.0), q=6, kmax=1, dt=0.02, tol_newton_rel=1e-13,
                tol_newton_abs=1e-13, tol_gmres_rel=1e-9, gmres_restart=60)
    args.update(kw)
    return hb.Context(2, (6, 5), (0, 0), (1, 1), 4, **args)


def euler(hb, **kw):
    args = dict(law=hb.LAW_EULER, flux=hb.FLUX_RUSANOV, q=4, kmax=1, dt=0.03, tol_newton_rel=1e-12,
                tol_newton_abs=1e-13, tol_gmres_rel=1e-6, gmres_restart=60, pc=hb.PC_BJEXT)
    args.update(kw)
    return hb.Context(2, (5, 4), (-1, -1), (1, 1), 3, **args)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_nan_in_state_gives_nonfinite_and_keeps_state(hb, prec):
    ctx = euler(hb, precision=hb.PREC_FP64 if prec == "fp64" else hb.PREC_MIXED)
    w = inputs.density_wave(ctx.node_coords())
    w[3, 2, 1, 1] = np.nan
    ctx.set_state(w)
    before = ctx.get_state()
    with pytest.raises(hb.HBPCError) as ei:
        ctx.step(1)
    assert ei.value.status == hb.ERR_NONFINITE
    after = ctx.get_state()
    assert after.tobytes() == before.tobytes()
    assert ctx.stats()["steps"] == 0
    ctx.close()


@pytest.mark.parametrize("cap", ["newton", "gmres"])
def test_iteration_cap_gives_no_convergence_and_keeps_state(hb, cap):
    if cap == "newton":      # one Newton iteration cannot meet 1e-12 on the Euler stage
        ctx = euler(hb, newton_max_iter=1)
        w0 = inputs.density_wave(ctx.node_coords())
    else:                    # one GMRES iteration per Newton step, three Newton steps
        ctx = advection(hb, gmres_max_iter=1, newton_max_iter=3)
        w0 = inputs.sine_product(ctx.node_coords())
    ctx.set_state(w0)
    with pytest.raises(hb.HBPCError) as ei:
        ctx.step(1)
    assert ei.value.status == hb.ERR_NO_CONVERGENCE
    assert ctx.get_state().tobytes() == w0.tobytes()
    assert ctx.stats()["steps"] == 0
    ctx.close()


def test_failure_after_completed_steps_keeps_the_last_one(hb):
    """Two steps succeed, then the state is poisoned by a NaN in a copy: the
    failed third step leaves exactly the state it was given."""
    ctx = advection(hb)
    ctx.set_state(inputs.sine_product(ctx.node_coords()))
    ctx.step(2)
    w2 = ctx.get_state()
    bad = w2.copy()
    bad[0, 0, 0, 0] = np.inf
    ctx.set_state(bad)
    with pytest.raises(hb.HBPCError) as ei:
        ctx.step(1)
    assert ei.value.status == hb.ERR_NONFINITE
    assert ctx.get_state().tobytes() == bad.tobytes()
    assert ctx.stats()["steps"] == 2
    ctx.close()


@pytest.mark.parametrize("make", ["advection", "euler_mixed"])
def test_resume_is_bit_identical(hb, make):
    """get_state after k steps -> a new context -> set_state, set_time -> the
    remaining steps give the same bits as one uninterrupted run."""
    mk = (lambda: advection(hb)) if make == "advection" else (lambda: euler(hb, precision=hb.PREC_MIXED))
    a = mk()
    w0 = (inputs.sine_product if make == "advection" else inputs.density_wave)(a.node_coords())
    a.set_state(w0)
    a.step(3)
    full = a.get_state()
    a.close()
    b = mk()
    b.set_state(w0)
    b.step(1)
    ckpt = b.get_state()
    t_ckpt = b.stats()["t"]
    b.close()
    c = mk()
    c.set_state(ckpt)
    c.set_time(t_ckpt)
    c.step(2)
    assert c.get_state().tobytes() == full.tobytes()
    assert abs(c.stats()["t"] - 3 * 0.02 * (1 if make == "advection" else 1.5)) < 1e-15
    c.close()


def test_advance_to_lands_on_t_end(hb):
    """Two whole steps of dt and a last step of dt / 2 reach t_end = 2.5 dt;
    the result equals the exact per-Fourier-mode HBPC(6,1) result of those
    three steps."""
    dt = 0.02
    ctx = advection(hb, dt=dt)
    w0 = inputs.sine_product(ctx.node_coords())
    ctx.set_state(w0)
    ctx.advance_to(2.5 * dt)
    w = ctx.get_state()
    st = ctx.stats()
    assert st["steps"] == 3 and st["t"] == 2.5 * dt
    disc = dgsem.Disc(dgsem.Mesh(2, (6, 5), (0, 0), (1, 1)), 4, laws.Physics(laws.ADVECTION, 2, a=(1.0, 1.0)))
    ref = exact.fourier_hbpc(disc, inputs.sine_product(disc.node_coords()), dt, 6, 1, 2)
    ref = exact.fourier_hbpc(disc, ref, 0.5 * dt, 6, 1, 1)
    assert np.linalg.norm(w - ref) / np.linalg.norm(ref) <= 1e-11
    # already there: nothing to do; before the current time: rejected
    ctx.advance_to(2.5 * dt)
    assert ctx.stats()["steps"] == 3
    with pytest.raises(hb.HBPCError) as ei:
        ctx.advance_to(dt)
    assert ei.value.status == hb.ERR_INVALID_ARG
    ctx.close()


def test_run_to_solver_t_end_matches_oracle(hb):
    """hbpc_run advances to the solver's T_end (Algorithm 1): Euler, 2 whole
    steps and a remainder of 0.4 dt, against the oracle's HBPC(4,1)."""
    dt = 0.03
    t_end = 2.4 * dt
    ctx = euler(hb, dt=dt, t_end=t_end, pc=hb.PC_NONE, tol_newton_rel=1e-13, tol_gmres_rel=1e-8)
    w0 = inputs.density_wave(ctx.node_coords())
    ctx.set_state(w0)
    ctx.run()
    w = ctx.get_state()
    assert ctx.stats()["t"] == t_end
    ph = laws.Physics(laws.EULER, 2, flux="rusanov")
    disc = dgsem.Disc(dgsem.Mesh(2, (5, 4), (-1, -1), (1, 1)), 3, ph)
    opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-13, gmres_tol=1e-8, restart=60, jv="fd")
    ref = inputs.density_wave(disc.node_coords())
    for h in (dt, dt, 0.4 * dt):
        ref = ohbpc.dg_stepper(disc, h, 4, 1, opts)(ref)
    assert np.linalg.norm(w - ref) / np.linalg.norm(ref) <= 1e-11
    ctx.close()
    nt = euler(hb)
    with pytest.raises(hb.HBPCError) as ei:      # no final time given
        nt.run()
    assert ei.value.status == hb.ERR_INVALID_ARG
    nt.close()


def test_wait_limit_gives_timeout(hb):
    """A wait limit far shorter than a step: the call returns
    HBPC_ERR_TIMEOUT while the device keeps working; destroying the context
    waits for it, and a new context works normally."""
    ctx = hb.Context(2, (64, 64), (0, 0), (1, 1), 5, law=hb.LAW_ADVECTION, a=(1.0, 1.0), q=8, kmax=4,
                     dt=1.0 / 96, tol_newton_rel=1e-12, tol_newton_abs=1e-12, tol_gmres_rel=1e-5,
                     pc=hb.PC_BJEXT, precision=hb.PREC_MIXED)
    ctx.set_state(inputs.sine_product(ctx.node_coords()))
    ctx.set_wait_limit(1e-6)
    with pytest.raises(hb.HBPCError) as ei:
        ctx.step(1)
    assert ei.value.status == hb.ERR_TIMEOUT
    ctx.close()
    torch.cuda.synchronize()
    c2 = advection(hb)
    c2.set_wait_limit(60.0)
    c2.set_state(inputs.sine_product(c2.node_coords()))
    c2.step(1)
    assert np.isfinite(c2.get_state()).all()
    c2.close()
