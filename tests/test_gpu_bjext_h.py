"""BJ^H_ext on the GPU (Sec. 3.2.3): the element Hessian blocks assembled by
the dual-number form of the Jacobian assembly, S = I - c1 J + c2 (H + J^2),
its inverse and the BJ^H_ext apply, against the oracle's complex-step blocks
and closed-form inverse blocks.  Tolerances as for BJ_ext: the same FP64
quantities summed in another order and inverted by Gauss-Jordan instead of LU,
1e-11 relative; FP32 blocks in the mixed mode, 1e-4.  Newton and HBPC results
do not depend on the preconditioner beyond the solver tolerances (1e-11)."""
import numpy as np
import pytest
import torch

from oracle import dgsem, laws, newton
from oracle.basis import GAUSS, LOBATTO
from paper_2109_04804_gb300 import inputs
from tests.test_gpu_parity import FAM, FLUX, LAWS, dev, euler_field, host, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    import __graft_entry__ as g
    g.build()
    from paper_2109_04804_gb300 import hbpc
    assert torch.cuda.is_available()
    return hbpc


def pair(hb, law, dim, N, n, family=LOBATTO, flux="lf", nu=0.0, **solver):
    lo, hi, a = (-1, -1, -1), (1, 1, 1), (1.0, -0.6, 0.35)
    ctx = hb.Context(dim, n, lo, hi, N, law=LAWS[law], flux=FLUX[flux], a=a, eps=1.0, nu=nu,
                     nodes=FAM[family], **solver)
    ph = laws.Physics(law, dim, a=a, eps=1.0, flux=flux, nu=nu)
    disc = dgsem.Disc(dgsem.Mesh(dim, n, lo, hi), N, ph, family)
    return ctx, disc


def stage_point(disc, seed):
    """(W, sigma): sigma = R1(W) plus a perturbation, as inside a Newton
    iteration (the Hessian blocks depend on sigma)."""
    rng = np.random.default_rng(seed)
    if disc.ph.law == laws.EULER:
        W = euler_field(disc, seed, amp=0.02)
    else:
        W = 0.5 + 0.2 * rng.standard_normal(disc.shape)
    S = dgsem.R1(disc, W)
    S = S + 0.1 * np.abs(S).max() * rng.standard_normal(disc.shape)
    return W, S, rng


APPLY_CASES = [
    # law, dim, N, n, family, flux, nu
    (laws.EULER, 2, 4, (7, 5), LOBATTO, "rusanov", 0.0),
    (laws.EULER, 2, 3, (5, 4), GAUSS, "lf", 0.0),
    (laws.EULER, 1, 3, (37,), LOBATTO, "lf", 0.0),
    (laws.EULER, 3, 2, (3, 4, 2), LOBATTO, "rusanov", 0.0),
    (laws.BURGERS, 2, 3, (7, 5), LOBATTO, "rusanov", 0.02),
    (laws.BURGERS, 1, 3, (37,), GAUSS, "lf", 0.0),
]


@pytest.mark.parametrize("law,dim,N,n,family,flux,nu", APPLY_CASES)
def test_bjext_h_apply_parity(hb, law, dim, N, n, family, flux, nu):
    dt, a1, a2 = 0.15, 1.0, 1.0
    ctx, disc = pair(hb, law, dim, N, n, family, flux, nu, dt=dt, pc=hb.PC_BJEXT_H)
    W, S, rng = stage_point(disc, 51)
    X = np.concatenate([W.ravel(), S.ravel()])
    v = rng.standard_normal(2 * disc.ndof)
    sysm = newton.StageSystem(disc, W, a1, a2, dt)
    ref = newton.make_preconditioner(sysm, X, "bjext_h")(v)
    ref_no_h = newton.make_preconditioner(sysm, X, "bjext")(v)
    assert rel(ref_no_h, ref) > 1e-6          # the Hessian blocks matter here
    out = torch.empty(2 * disc.ndof, dtype=torch.float64, device="cuda")
    ctx.eval_pc(a1, a2, dev(X), dev(v), out)
    assert rel(host(out), ref) <= 1e-11
    ctx.close()


@pytest.mark.parametrize("law,dim,N,n,family,flux,nu", [APPLY_CASES[0], APPLY_CASES[4]])
def test_bjext_h_apply_parity_mixed(hb, law, dim, N, n, family, flux, nu):
    dt = 0.15
    ctx, disc = pair(hb, law, dim, N, n, family, flux, nu, dt=dt, pc=hb.PC_BJEXT_H, precision=hb.PREC_MIXED)
    W, S, rng = stage_point(disc, 52)
    X = np.concatenate([W.ravel(), S.ravel()])
    v = rng.standard_normal(2 * disc.ndof)
    ref = newton.make_preconditioner(newton.StageSystem(disc, W, 1.0, 1.0, dt), X, "bjext_h")(v)
    out = torch.empty(2 * disc.ndof, dtype=torch.float64, device="cuda")
    ctx.eval_pc(1.0, 1.0, dev(X), dev(v), out)
    err = rel(host(out), ref)
    assert err <= 1e-4, err
    ctx.close()


def test_linear_flux_bjext_h_is_bjext(hb):
    """H = 0 for a linear flux: BJ^H_ext and BJ_ext give the same P^-1."""
    dt = 0.1
    outs = []
    for pc in (hb.PC_BJEXT, hb.PC_BJEXT_H):
        ctx, disc = pair(hb, laws.ADVECTION, 2, 4, (7, 5), dt=dt, pc=pc)
        rng = np.random.default_rng(53)
        X = rng.standard_normal(2 * disc.ndof)
        v = rng.standard_normal(2 * disc.ndof)
        out = torch.empty(2 * disc.ndof, dtype=torch.float64, device="cuda")
        ctx.eval_pc(1.0, 1.0, dev(X), dev(v), out)
        outs.append(host(out))
        ctx.close()
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("law,dim,flux,alphas", [
    (laws.EULER, 2, "rusanov", (1.0, 1.0)), (laws.BURGERS, 2, "lf", (0.5, 1.0 / 6.0)),
    (laws.EULER, 1, "lf", (1.0 / 6.0, 1.0 / 54.0))])
def test_newton_solve_with_bjext_h_parity(hb, law, dim, flux, alphas):
    N, dt = 3, 0.08
    n = {1: (12,), 2: (5, 4)}[dim]
    ctx, disc = pair(hb, law, dim, N, n, LOBATTO, flux, dt=dt, tol_newton_rel=1e-13, tol_newton_abs=1e-13,
                     tol_gmres_rel=1e-9, gmres_restart=80, pc=hb.PC_BJEXT_H)
    X = disc.node_coords()
    W0 = inputs.density_wave(X) if law == laws.EULER else 0.5 + 0.25 * inputs.sine_product(X, k=1.0)
    b = W0 + dt * 0.1 * np.cos(3.0 * W0)
    a1, a2 = alphas
    opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-13, gmres_tol=1e-9, restart=80, jv="fd", pc="bjext_h")
    Wr, Sr, st = newton.newton_solve(disc, b, a1, a2, dt, W0, opts)
    Wd = torch.empty(disc.ndof, dtype=torch.float64, device="cuda")
    Sd = torch.empty_like(Wd)
    ctx.newton_solve(dev(b), a1, a2, dev(W0), Wd, Sd)
    assert rel(host(Wd), Wr.ravel()) <= 1e-11
    assert rel(host(Sd), Sr.ravel()) <= 1e-10
    ctx.close()


@pytest.mark.parametrize("schur", [False, True])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_hbpc_steps_with_bjext_h_match_bjext(hb, schur, prec):
    """HBPC(4, 1) steps of the Euler density wave at a large time step with
    BJ_ext and with BJ^H_ext (and with the Schur form, whose preconditioner is
    then the D block of either): the same states; the iteration counts of both
    are reported by stats()."""
    if schur and prec == "mixed":
        pytest.skip("the Schur form is FP64 only")
    res, its = [], []
    for pc in (hb.PC_BJEXT, hb.PC_BJEXT_H):
        ctx = hb.Context(2, (8, 8), (-1, -1), (1, 1), 3, law=hb.LAW_EULER, flux=hb.FLUX_RUSANOV, eps=1.0,
                         q=4, kmax=1, dt=0.05, tol_newton_rel=1e-12, tol_newton_abs=1e-13,
                         tol_gmres_rel=1e-9 if prec == "fp64" else 1e-5, gmres_restart=100, pc=pc,
                         precision=hb.PREC_FP64 if prec == "fp64" else hb.PREC_MIXED)
        if schur:
            ctx.set_schur(True)
        ctx.set_state(inputs.density_wave(ctx.node_coords()))
        ctx.step(2)
        res.append(ctx.get_state())
        its.append(ctx.stats()["gmres_its"])
        ctx.close()
    assert rel(res[1], res[0]) <= (1e-10 if prec == "fp64" else 1e-9)
    assert its[1] > 0 and its[0] > 0


def test_batch_with_bjext_h(hb):
    """A batch of viscous Burgers instances preconditioned by BJ^H_ext ends
    where the same batch with BJ_ext does."""
    meshes = [((6, 5), (0, 0), (1, 1)), ((4, 4), (0, 0), (1, 1))]
    res = []
    for pc in (hb.PC_BJEXT, hb.PC_BJEXT_H):
        b = hb.Batch(2, meshes, [3, 3], nus=[0.01, 0.0], law=hb.LAW_BURGERS, q=4, kmax=1, dt=0.02,
                     tol_newton_rel=1e-12, tol_newton_abs=1e-13, tol_gmres_rel=1e-9, gmres_restart=40, pc=pc)
        for i in range(2):
            b.set_state(i, 0.5 + 0.2 * inputs.burgers_fourier(b.node_coords(i), seed=i, n_modes=3, kmax=2))
        b.step(2)
        res.append([b.get_state(i) for i in range(2)])
        b.close()
    for i in range(2):
        assert rel(res[1][i], res[0][i]) <= 1e-10
