"""The Schur form of the Newton systems (Sec. 3.2.4, Eq. 19) on the GPU: the
same roots as the extended form, against the exact per-Fourier-mode HBPC
result (linear advection), the oracle's Schur Newton (one stage) and the
oracle's HBPC steps (Euler), at the parity tolerance of the extended path."""
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
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("pc", ["bjext", "none"])
def test_advection_schur_steps_vs_exact(hb, pc):
    dt, n, q, kmax = 0.005, (6, 5), 6, 2
    ctx = hb.Context(2, n, (0, 0), (1, 1), 4, law=hb.LAW_ADVECTION, a=(1.0, 1.0), q=q, kmax=kmax, dt=dt,
                     tol_newton_rel=1e-13, tol_newton_abs=1e-13, tol_gmres_rel=1e-9, gmres_restart=100,
                     pc=hb.PC_BJEXT if pc == "bjext" else hb.PC_NONE)
    ctx.set_schur(True)
    ctx.set_state(inputs.sine_product(ctx.node_coords()))
    ctx.step(3)
    w = ctx.get_state()
    disc = dgsem.Disc(dgsem.Mesh(2, n, (0, 0), (1, 1)), 4, laws.Physics(laws.ADVECTION, 2, a=(1.0, 1.0)))
    ref = exact.fourier_hbpc(disc, inputs.sine_product(disc.node_coords()), dt, q, kmax, 3)
    assert rel(w, ref) <= 1e-11
    ctx.close()


@pytest.mark.parametrize("flux", ["lf", "rusanov"])
def test_euler_schur_stage_solve_vs_oracle(hb, flux):
    """One implicit stage (Eq. 7-9) by the Schur form: the oracle's Schur Newton
    reaches the same root."""
    dt, n, N = 0.03, (4, 3), 3
    a1, a2 = 0.5, 1.0 / 6.0
    ctx = hb.Context(2, n, (-1, -1), (1, 1), N, law=hb.LAW_EULER, flux=1 if flux == "rusanov" else 0, dt=dt,
                     tol_newton_rel=1e-13, tol_newton_abs=1e-14, tol_gmres_rel=1e-9, gmres_restart=100,
                     pc=hb.PC_BJEXT)
    ctx.set_schur(True)
    ph = laws.Physics(laws.EULER, 2, flux=flux)
    disc = dgsem.Disc(dgsem.Mesh(2, n, (-1, -1), (1, 1)), N, ph)
    rng = np.random.default_rng(9)
    W0 = inputs.density_wave(disc.node_coords()) * (1.0 + 0.02 * rng.standard_normal(disc.shape))
    b = W0 + 0.01 * rng.standard_normal(disc.shape)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    Wg = torch.empty(disc.ndof, dtype=torch.float64, device="cuda")
    Sg = torch.empty_like(Wg)
    ctx.newton_solve(dev(b), a1, a2, dev(W0), Wg, Sg)
    opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-14, gmres_tol=1e-9, restart=100, jv="fd", pc="bjext")
    Wo, So, st = newton.schur_newton_solve(disc, b, a1, a2, dt, W0, opts)
    assert st.converged
    assert rel(Wg.cpu().numpy(), Wo) <= 1e-11
    assert rel(Sg.cpu().numpy(), So) <= 1e-10
    ctx.close()


def test_euler_schur_steps_vs_oracle(hb):
    dt, n = 0.02, (4, 3)
    ctx = hb.Context(2, n, (-1, -1), (1, 1), 3, law=hb.LAW_EULER, flux=hb.FLUX_RUSANOV, q=4, kmax=1, dt=dt,
                     tol_newton_rel=1e-13, tol_newton_abs=1e-13, tol_gmres_rel=1e-8, gmres_restart=100,
                     pc=hb.PC_BJEXT)
    ctx.set_schur(True)
    ctx.set_state(inputs.density_wave(ctx.node_coords()))
    ctx.step(2)
    w = ctx.get_state()
    ph = laws.Physics(laws.EULER, 2, flux="rusanov")
    disc = dgsem.Disc(dgsem.Mesh(2, n, (-1, -1), (1, 1)), 3, ph)
    opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-13, gmres_tol=1e-8, restart=100, jv="fd")
    adv = ohbpc.dg_stepper(disc, dt, 4, 1, opts)
    ref = inputs.density_wave(disc.node_coords())
    for _ in range(2):
        ref = adv(ref)
    assert rel(w, ref) <= 1e-11
    ctx.close()


def test_schur_restarted_gmres(hb):
    """A restart length far below the iterations needed: the Schur restart
    residual rhs - J_Schur dW keeps GMRES on course."""
    dt, n = 0.01, (5, 4)
    ctx = hb.Context(2, n, (0, 0), (1, 1), 3, law=hb.LAW_ADVECTION, a=(1.0, 1.0), q=4, kmax=0, dt=dt,
                     tol_newton_rel=1e-13, tol_newton_abs=1e-13, tol_gmres_rel=1e-10, gmres_restart=5,
                     pc=hb.PC_NONE)
    ctx.set_schur(True)
    ctx.set_state(inputs.sine_product(ctx.node_coords()))
    ctx.step(2)
    w = ctx.get_state()
    assert ctx.stats()["gmres_its"] > 10
    disc = dgsem.Disc(dgsem.Mesh(2, n, (0, 0), (1, 1)), 3, laws.Physics(laws.ADVECTION, 2, a=(1.0, 1.0)))
    ref = exact.fourier_hbpc(disc, inputs.sine_product(disc.node_coords()), dt, 4, 0, 2)
    assert rel(w, ref) <= 1e-11
    ctx.close()


def test_schur_rejections(hb):
    mixed = hb.Context(2, (3, 3), (0, 0), (1, 1), 3, precision=hb.PREC_MIXED)
    with pytest.raises(hb.HBPCError) as ei:
        mixed.set_schur(True)
    assert ei.value.status == hb.ERR_UNSUPPORTED
    mixed.close()
    c = hb.Context(2, (3, 3), (0, 0), (1, 1), 3, q=6, kmax=1)
    c.set_schur(True)
    with pytest.raises(hb.HBPCError) as ei:
        c.set_corrector_batch(True)
    assert ei.value.status == hb.ERR_UNSUPPORTED
    c.set_schur(False)
    c.set_corrector_batch(True)
    c.close()
