"""Corrector batching (the outlook of Sec. 6): the s - 1 corrector stages of one
sweep of Algorithm 1 depend only on the previous level, so they are solved as
one batched Newton-GMRES.  The result must be the same HBPC step: against the
exact per-Fourier-mode HBPC result (linear advection) and the oracle's
Newton-GMRES steps (Euler, viscous Burgers), at the parity tolerance of the
sequential path (1e-11 relative L2, Newton tolerance 1e-13)."""
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("pc", ["bjext", "none"])
@pytest.mark.parametrize("q,kmax", [(8, 4), (6, 2)])
def test_advection_batched_correctors_vs_exact(hb, prec, pc, q, kmax):
    dt = 0.01
    n = (6, 5)
    ctx = hb.Context(2, n, (0, 0), (1, 1), 5, law=hb.LAW_ADVECTION, a=(1.0, 1.0), q=q, kmax=kmax, dt=dt,
                     tol_newton_rel=1e-13, tol_newton_abs=1e-13, tol_gmres_rel=1e-9, gmres_restart=100,
                     pc=hb.PC_BJEXT if pc == "bjext" else hb.PC_NONE,
                     precision=hb.PREC_FP64 if prec == "fp64" else hb.PREC_MIXED)
    ctx.set_corrector_batch(True)
    w0 = inputs.sine_product(ctx.node_coords())
    ctx.set_state(w0)
    ctx.step(3)
    w = ctx.get_state()
    st = ctx.stats()
    disc = dgsem.Disc(dgsem.Mesh(2, n, (0, 0), (1, 1)), 5, laws.Physics(laws.ADVECTION, 2, a=(1.0, 1.0)))
    ref = exact.fourier_hbpc(disc, inputs.sine_product(disc.node_coords()), dt, q, kmax, 3)
    assert rel(w, ref) <= 1e-11
    # one batched solve per sweep: (s - 1) predictor solves + kmax batched ones per step
    s = q // 2
    assert st["newton_solves"] == 3 * ((s - 1) + kmax)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_euler_batched_correctors_vs_oracle(hb, prec):
    dt = 0.04
    n = (4, 3)
    ctx = hb.Context(2, n, (-1, -1), (1, 1), 3, law=hb.LAW_EULER, flux=hb.FLUX_RUSANOV, q=6, kmax=2, dt=dt,
                     tol_newton_rel=1e-13, tol_newton_abs=1e-13, tol_gmres_rel=1e-8, gmres_restart=100,
                     pc=hb.PC_BJEXT, precision=hb.PREC_FP64 if prec == "fp64" else hb.PREC_MIXED)
    ctx.set_corrector_batch(True)
    ctx.set_state(inputs.density_wave(ctx.node_coords()))
    ctx.step(2)
    w = ctx.get_state()
    ph = laws.Physics(laws.EULER, 2, flux="rusanov")
    disc = dgsem.Disc(dgsem.Mesh(2, n, (-1, -1), (1, 1)), 3, ph)
    opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-13, gmres_tol=1e-8, restart=100, jv="fd")
    adv = ohbpc.dg_stepper(disc, dt, 6, 2, opts)
    ref = inputs.density_wave(disc.node_coords())
    for _ in range(2):
        ref = adv(ref)
    assert rel(w, ref) <= 1e-11
    ctx.close()


def test_viscous_burgers_batched_matches_sequential(hb):
    """The batched and the sequential correctors give the same step."""
    out = []
    for batched in (False, True):
        ctx = hb.Context(2, (5, 4), (0, 0), (1, 1), 4, law=hb.LAW_BURGERS, nu=0.01, q=6, kmax=2, dt=0.01,
                         tol_newton_rel=1e-13, tol_newton_abs=1e-14, tol_gmres_rel=1e-9, gmres_restart=100,
                         pc=hb.PC_BJEXT)
        if batched:
            ctx.set_corrector_batch(True)
        ctx.set_state(0.5 + 0.2 * inputs.burgers_fourier(ctx.node_coords(), seed=3, n_modes=3, kmax=2))
        ctx.step(2)
        out.append(ctx.get_state())
        ctx.close()
    assert rel(out[1], out[0]) <= 1e-11


def test_corrector_batch_switches(hb):
    ctx = hb.Context(2, (3, 3), (0, 0), (1, 1), 3, law=hb.LAW_ADVECTION, a=(1.0, 1.0), q=6, kmax=1, dt=0.01,
                     tol_newton_rel=1e-13, tol_newton_abs=1e-13, tol_gmres_rel=1e-9, pc=hb.PC_BJEXT)
    ctx.set_corrector_batch(True)
    ctx.set_corrector_batch(True)      # already on: nothing to do
    with pytest.raises(hb.HBPCError) as ei:
        ctx.set_pc(hb.PC_LEARNED)
    assert ei.value.status == hb.ERR_UNSUPPORTED
    ctx.set_corrector_batch(False)
    ctx.set_state(inputs.sine_product(ctx.node_coords()))
    ctx.step(1)
    assert ctx.stats()["newton_solves"] == 2 + 2
    ctx.close()
    ns = hb.Context(2, (3, 3), (0, 0), (1, 1), 3, law=hb.LAW_NAVIER_STOKES, mu=0.01, q=4, kmax=1, dt=0.01)
    with pytest.raises(hb.HBPCError) as ei:
        ns.set_corrector_batch(True)
    assert ei.value.status == hb.ERR_UNSUPPORTED
    ns.close()
