"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle on the same
seeded inputs.  Tolerances:
  * R1, R2, G, linear Jv: the same FP64 sums in a different order, so the
    element-wise error is a few ulps of the largest term: 1e-12 relative.
  * Eq. 23 difference quotients: both sides divide a difference of two O(|R|)
    values by eps_FD ~ 1.5e-8 / ||dW||, so rounding is amplified by ~1e8:
    1e-6 relative.
  * Newton and HBPC results: both sides stop on ||G|| <= tol ||G0|| or
    ||dW|| <= tol_abs (Sec. 5.2: the absolute test is needed because ||G0|| of a
    corrector stage can already sit at the rounding floor); with tol = 1e-13 and
    tol_abs = 1e-13 the answers agree to 1e-11 relative L2 (the spec bar).
"""
import numpy as np
import pytest
import torch

from oracle import dgsem, exact, hbpc as ohbpc, laws, newton
from oracle.basis import GAUSS, LOBATTO
from paper_2109_04804_gb300 import inputs

pytestmark = pytest.mark.gpu

LAWS = {laws.ADVECTION: 0, laws.BURGERS: 1, laws.EULER: 2}
FLUX = {"lf": 0, "rusanov": 1}
FAM = {LOBATTO: 0, GAUSS: 1}


@pytest.fixture(scope="module")
def hb():
    import __graft_entry__ as g
    g.build()
    from paper_2109_04804_gb300 import hbpc
    assert torch.cuda.is_available()
    return hbpc


def pair(hb, law, dim, N, n, family=LOBATTO, flux="lf", lo=(0, 0, 0), hi=(1, 1, 1),
         a=(1.0, -0.6, 0.35), eps=1.0, **solver):
    ctx = hb.Context(dim, n, lo, hi, N, law=LAWS[law], flux=FLUX[flux], a=a, eps=eps,
                     nodes=FAM[family], **solver)
    ph = laws.Physics(law, dim, a=a, eps=eps, flux=flux)
    disc = dgsem.Disc(dgsem.Mesh(dim, n, lo, hi), N, ph, family)
    return ctx, disc


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.cpu().numpy()


def euler_field(disc, seed, amp=0.05):
    rng = np.random.default_rng(seed)
    X = disc.node_coords()
    base = inputs.density_wave(X)
    return base * (1.0 + amp * rng.standard_normal(base.shape))


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


OP_CASES = (
    [(laws.ADVECTION, d, N, LOBATTO, "lf") for d in (1, 2, 3) for N in (1, 3, 5, 7)]
    + [(laws.ADVECTION, d, N, GAUSS, "lf") for d in (1, 2) for N in (2, 3)]
    + [(laws.BURGERS, d, N, LOBATTO, f) for d in (1, 2, 3) for N in (3, 5) for f in ("lf", "rusanov")]
    + [(laws.BURGERS, 2, 3, GAUSS, "rusanov")]
    + [(laws.EULER, d, N, LOBATTO, f) for d in (1, 2, 3) for N in (2, 3, 4, 5) for f in ("lf", "rusanov")]
    + [(laws.EULER, 2, 3, GAUSS, "rusanov"), (laws.EULER, 1, 2, GAUSS, "lf")]
)


def mesh_for(dim):
    # several blocks with a ragged tail in every dimension
    return {1: (37,), 2: (7, 5), 3: (3, 4, 2)}[dim]


@pytest.mark.parametrize("law,dim,N,family,flux", OP_CASES)
def test_r1_r2_parity(hb, law, dim, N, family, flux):
    ctx, disc = pair(hb, law, dim, N, mesh_for(dim), family, flux, eps=0.7 if law == laws.EULER else 1.0)
    coords = ctx.node_coords()
    oc = disc.node_coords()
    for m in range(dim):
        np.testing.assert_allclose(coords[m], oc[m], atol=1e-14)
    rng = np.random.default_rng(100 + dim * 10 + N)
    if law == laws.EULER:
        w = euler_field(disc, 7)
    else:
        w = rng.standard_normal(disc.shape)
    s = rng.standard_normal(disc.shape)
    r1_ref = dgsem.R1(disc, w)
    r2_ref = dgsem.R2(disc, w, s)
    wd, sd = dev(w), dev(s)
    out = torch.empty_like(wd)
    ctx.eval_R1(wd, out)
    r1 = host(out)
    ctx.eval_R2(wd, sd, out)
    r2 = host(out)
    for got, ref in ((r1, r1_ref), (r2, r2_ref)):
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= 1e-12 * scale
    ctx.close()


@pytest.mark.parametrize("law,dim,flux", [(laws.ADVECTION, 2, "lf"), (laws.EULER, 2, "rusanov"),
                                          (laws.BURGERS, 2, "lf"), (laws.EULER, 3, "lf")])
def test_residual_and_jv_parity(hb, law, dim, flux):
    N = 3
    ctx, disc = pair(hb, law, dim, N, mesh_for(dim), LOBATTO, flux, dt=0.03)
    rng = np.random.default_rng(5)
    if law == laws.EULER:
        W = euler_field(disc, 3)
    else:
        W = 0.5 + 0.3 * rng.standard_normal(disc.shape)
    S = dgsem.R1(disc, W) + 0.01 * rng.standard_normal(disc.shape)
    b = W + 0.01 * rng.standard_normal(disc.shape)
    a1, a2 = 0.5, 1.0 / 6.0
    sysm = newton.StageSystem(disc, b, a1, a2, 0.03)
    X = np.concatenate([W.ravel(), S.ravel()])
    G_ref, r1, r2 = sysm.residual(X)
    Gd = torch.empty(2 * disc.ndof, dtype=torch.float64, device="cuda")
    ctx.eval_G(dev(b), a1, a2, dev(X), Gd)
    G = host(Gd)
    assert np.abs(G - G_ref).max() <= 1e-12 * np.abs(G_ref).max()
    dX = rng.standard_normal(2 * disc.ndof)
    out = torch.empty_like(Gd)
    ctx.eval_Jv(a1, a2, dev(X), dev(dX), out)
    jv = host(out)
    if disc.ph.linear:
        ref = sysm.jv(X, r1, r2, dX, "linear")
        assert rel(jv, ref) <= 1e-13
    else:
        ref_fd = sysm.jv(X, r1, r2, dX, "fd")
        assert rel(jv, ref_fd) <= 1e-6
        if flux == "lf":
            # with a constant dissipation coefficient dR1/dw v = R2(w, v) exactly
            # (Sec. 3.2.1); Rusanov's coefficient depends on w, which the FD
            # quotient sees and the frozen-coefficient R2 does not
            ref_an = sysm.jv(X, r1, r2, dX, "analytic")
            assert rel(jv, ref_an) <= 1e-6
    ctx.close()


@pytest.mark.parametrize("law,dim,flux", [(laws.ADVECTION, 2, "lf"), (laws.BURGERS, 2, "lf"),
                                          (laws.EULER, 2, "lf"), (laws.EULER, 3, "lf")])
def test_mixed_precision_jv_parity(hb, law, dim, flux):
    """In the mixed mode hbpc_eval_Jv returns the FP32 product of the Krylov
    loop: the analytic linearisation of Eq. 18 (dR1/dW v = R2(W, v), Sec. 3.2.1,
    and the exact derivative of R2 for the Hessian block) in FP32 arithmetic.
    With a constant dissipation coefficient it equals the oracle's analytic
    form, whose Hessian block is the Eq. 23 quotient (error ~1e-8); the FP32
    operator's rounding (~1e-7 per term) sets the 2e-5 bound."""
    N = 3
    ctx, disc = pair(hb, law, dim, N, mesh_for(dim), LOBATTO, flux, dt=0.03, precision=hb.PREC_MIXED)
    rng = np.random.default_rng(8)
    W = euler_field(disc, 4) if law == laws.EULER else 0.5 + 0.3 * rng.standard_normal(disc.shape)
    S = dgsem.R1(disc, W) + 0.01 * rng.standard_normal(disc.shape)
    a1, a2 = 0.5, 1.0 / 6.0
    sysm = newton.StageSystem(disc, W, a1, a2, 0.03)
    X = np.concatenate([W.ravel(), S.ravel()])
    _, r1, r2 = sysm.residual(X)
    for k in range(2):
        dX = rng.standard_normal(2 * disc.ndof)
        out = torch.empty(2 * disc.ndof, dtype=torch.float64, device="cuda")
        ctx.eval_Jv(a1, a2, dev(X), dev(dX), out)
        ref = sysm.jv(X, r1, r2, dX, "linear" if disc.ph.linear else "analytic")
        assert rel(host(out), ref) <= 2e-5, (k, rel(host(out), ref))
    ctx.close()


@pytest.mark.parametrize("law,dim,N,family,flux", [
    (laws.ADVECTION, 2, 5, LOBATTO, "lf"), (laws.ADVECTION, 1, 3, GAUSS, "lf"),
    (laws.BURGERS, 2, 3, LOBATTO, "rusanov"), (laws.EULER, 2, 4, LOBATTO, "rusanov"),
    (laws.EULER, 2, 3, LOBATTO, "lf"), (laws.EULER, 2, 3, GAUSS, "rusanov"), (laws.EULER, 1, 3, LOBATTO, "lf")])
def test_bjext_apply_parity(hb, law, dim, N, family, flux):
    """P^-1 of the BJ_ext preconditioner (element Jacobians, S = I - c1 J + c2 J^2,
    inverse, block apply) against the oracle's dense construction."""
    dt = 0.04
    ctx, disc = pair(hb, law, dim, N, mesh_for(dim), family, flux, lo=(-1, -1, -1), hi=(1, 1, 1), dt=dt,
                     pc=hb.PC_BJEXT)
    rng = np.random.default_rng(31)
    if law == laws.EULER:
        W = euler_field(disc, 5, amp=0.02)
    else:
        W = 0.5 + 0.2 * rng.standard_normal(disc.shape)
    X = np.concatenate([W.ravel(), dgsem.R1(disc, W).ravel()])
    v = rng.standard_normal(2 * disc.ndof)
    a1, a2 = 1.0, 1.0
    sysm = newton.StageSystem(disc, W, a1, a2, dt)
    ref = newton.BJExt(sysm, W)(v)
    out = torch.empty(2 * disc.ndof, dtype=torch.float64, device="cuda")
    ctx.eval_pc(a1, a2, dev(X), dev(v), out)
    assert rel(host(out), ref) <= 1e-11
    ctx.close()


@pytest.mark.parametrize("law,dim,N,flux", [(laws.ADVECTION, 2, 5, "lf"), (laws.EULER, 2, 4, "rusanov"),
                                            (laws.BURGERS, 2, 3, "lf"), (laws.ADVECTION, 1, 3, "lf"),
                                            (laws.ADVECTION, 3, 2, "lf")])
def test_bjext_apply_parity_mixed(hb, law, dim, N, flux):
    """In the mixed mode the blocks S_e, their Gauss-Jordan inverses and the
    apply are FP32: the result against the oracle's FP64 construction is within
    FP32 rounding amplified by the blocks' condition numbers (1e-4 here)."""
    dt = 0.04
    ctx, disc = pair(hb, law, dim, N, mesh_for(dim), LOBATTO, flux, lo=(-1, -1, -1), hi=(1, 1, 1), dt=dt,
                     pc=hb.PC_BJEXT, precision=hb.PREC_MIXED)
    rng = np.random.default_rng(32)
    if law == laws.EULER:
        W = euler_field(disc, 6, amp=0.02)
    else:
        W = 0.5 + 0.2 * rng.standard_normal(disc.shape)
    X = np.concatenate([W.ravel(), dgsem.R1(disc, W).ravel()])
    v = rng.standard_normal(2 * disc.ndof)
    sysm = newton.StageSystem(disc, W, 1.0, 1.0, dt)
    ref = newton.BJExt(sysm, W)(v)
    out = torch.empty(2 * disc.ndof, dtype=torch.float64, device="cuda")
    ctx.eval_pc(1.0, 1.0, dev(X), dev(v), out)
    err = rel(host(out), ref)
    assert err <= 1e-4, err
    ctx.close()


@pytest.mark.parametrize("law,dim,flux,alphas,pc", [
    (laws.ADVECTION, 2, "lf", (0.5, 1.0 / 6.0), "none"), (laws.ADVECTION, 1, "lf", (1.0, 1.0), "none"),
    (laws.BURGERS, 1, "rusanov", (1.0, 1.0), "none"), (laws.EULER, 2, "rusanov", (1.0 / 6.0, 1.0 / 54.0), "none"),
    (laws.EULER, 2, "lf", (1.0, 1.0), "none"), (laws.ADVECTION, 2, "lf", (1.0, 1.0), "bjext"),
    (laws.EULER, 2, "rusanov", (1.0, 1.0), "bjext"), (laws.BURGERS, 2, "lf", (0.5, 1.0 / 6.0), "bjext")])
def test_newton_solve_parity(hb, law, dim, flux, alphas, pc):
    N, dt = 3, 0.05
    n = {1: (12,), 2: (5, 4)}[dim]
    ctx, disc = pair(hb, law, dim, N, n, LOBATTO, flux, lo=(-1, -1, -1), hi=(1, 1, 1), dt=dt,
                     tol_newton_rel=1e-13, tol_newton_abs=1e-13, tol_gmres_rel=1e-9, gmres_restart=80,
                     pc=hb.PC_BJEXT if pc == "bjext" else hb.PC_NONE)
    X = disc.node_coords()
    if law == laws.EULER:
        W0 = inputs.density_wave(X)
    elif law == laws.BURGERS:
        W0 = 0.5 + 0.25 * inputs.sine_product(X, k=1.0)
    else:
        W0 = inputs.sine_product(X, k=1.0)
    b = W0 + dt * 0.1 * np.cos(3.0 * W0)
    a1, a2 = alphas
    opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-13, gmres_tol=1e-9, restart=80,
                                jv="linear" if disc.ph.linear else "fd")
    Wr, Sr, st = newton.newton_solve(disc, b, a1, a2, dt, W0, opts)
    Wd = torch.empty(disc.ndof, dtype=torch.float64, device="cuda")
    Sd = torch.empty_like(Wd)
    ctx.newton_solve(dev(b), a1, a2, dev(W0), Wd, Sd)
    assert rel(host(Wd), Wr.ravel()) <= 1e-11
    assert rel(host(Sd), Sr.ravel()) <= 1e-10
    ctx.close()


def test_c1_advection_1d_full_run(hb):
    """1-D advection on [0,1], 16 elements, N=3, HBPC(4,0), CFL 1 -> dt = 1/64,
    T = 1: equals the exact per-mode HBPC result; error to the exact solution
    sin(2 pi (x - t)) is the method's."""
    dt = 1.0 / 64
    ctx, disc = pair(hb, laws.ADVECTION, 1, 3, (16,), a=(1.0,), q=4, kmax=0, dt=dt,
                     tol_newton_rel=1e-13, tol_newton_abs=1e-13, tol_gmres_rel=1e-10, gmres_restart=64)
    w0 = inputs.sine_product(ctx.node_coords())
    ctx.set_state(w0)
    ctx.step(64)
    w = ctx.get_state()
    w0o = inputs.sine_product(disc.node_coords())
    ref = exact.fourier_hbpc(disc, w0o, dt, 4, 0, 64)
    assert rel(w, ref) <= 1e-11
    err_exact = np.abs(w - w0o).max()           # T = 1 is one period
    assert 1e-6 < err_exact < 1e-3
    st = ctx.stats()
    assert st["steps"] == 64 and st["newton_solves"] == 64
    ctx.close()


@pytest.mark.parametrize("q,kmax", [(4, 1), (6, 2), (8, 4)])
def test_2d_advection_steps_vs_exact(hb, q, kmax):
    dt = 0.01
    n = (6, 5)
    ctx, disc = pair(hb, laws.ADVECTION, 2, 5, n, a=(1.0, 1.0), q=q, kmax=kmax, dt=dt,
                     tol_newton_rel=1e-13, tol_newton_abs=1e-13, tol_gmres_rel=1e-9, gmres_restart=100)
    w0 = inputs.sine_product(ctx.node_coords())
    ctx.set_state(w0)
    ctx.step(3)
    w = ctx.get_state()
    ref = exact.fourier_hbpc(disc, inputs.sine_product(disc.node_coords()), dt, q, kmax, 3)
    assert rel(w, ref) <= 1e-11
    ctx.close()


@pytest.mark.parametrize("flux", ["lf", "rusanov"])
def test_euler_steps_vs_oracle(hb, flux):
    dt = 0.04
    ctx, disc = pair(hb, laws.EULER, 2, 3, (4, 3), LOBATTO, flux, lo=(-1, -1), hi=(1, 1), q=6, kmax=1,
                     dt=dt, tol_newton_rel=1e-13, tol_newton_abs=1e-13, tol_gmres_rel=1e-8,
                     gmres_restart=100)
    w0 = inputs.density_wave(ctx.node_coords())
    ctx.set_state(w0)
    ctx.step(2)
    w = ctx.get_state()
    opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-13, gmres_tol=1e-8, restart=100, jv="fd")
    adv = ohbpc.dg_stepper(disc, dt, 6, 1, opts)
    ref = inputs.density_wave(disc.node_coords())
    for _ in range(2):
        ref = adv(ref)
    assert rel(w, ref) <= 1e-11
    # discrete conservation of every variable
    c0 = dgsem.cell_integral(disc, inputs.density_wave(disc.node_coords()))
    c1 = dgsem.cell_integral(disc, w)
    assert np.all(np.abs(c1 - c0) <= 1e-12 * np.abs(c0).max())
    ctx.close()


def test_c2_full_size_step_vs_exact(hb):
    """The bench workload: 2-D advection a = (1, 1), 64 x 64 elements, N = 5,
    HBPC(8, 4), CFL 8 (dt = 1/96), BJ_ext, eps_Newton 1e-12 (and ||dW|| <=
    1e-12), eps_GMRES 1e-5: one step equals the exact per-Fourier-mode HBPC step."""
    dt = 1.0 / 96
    ctx, disc = pair(hb, laws.ADVECTION, 2, 5, (64, 64), a=(1.0, 1.0), q=8, kmax=4, dt=dt,
                     tol_newton_rel=1e-12, tol_newton_abs=1e-12, tol_gmres_rel=1e-5, gmres_restart=100,
                     pc=hb.PC_BJEXT)
    w0 = inputs.sine_product(ctx.node_coords())
    ctx.set_state(w0)
    ctx.step(1)
    w = ctx.get_state()
    ref = exact.fourier_hbpc(disc, inputs.sine_product(disc.node_coords()), dt, 8, 4, 1)
    assert rel(w, ref) <= 1e-11
    ctx.close()


@pytest.mark.parametrize("law,dim,flux,pc", [
    (laws.ADVECTION, 2, "lf", "bjext"), (laws.ADVECTION, 2, "lf", "none"),
    (laws.EULER, 2, "rusanov", "bjext"), (laws.EULER, 2, "lf", "none"),
    (laws.BURGERS, 2, "rusanov", "bjext"), (laws.EULER, 3, "rusanov", "none")])
def test_mixed_precision_stage_solve_matches_oracle(hb, law, dim, flux, pc):
    """Mixed precision (FP32 Krylov loop with the analytic dual-number Jv, FP64
    Newton residual and update) reaches the same root as the FP64 oracle: the
    answer is fixed by G(X) = 0, which is evaluated in FP64."""
    N, dt = 3, 0.05
    n = {2: (5, 4), 3: (3, 2, 2)}[dim]
    ctx, disc = pair(hb, law, dim, N, n, LOBATTO, flux, lo=(-1, -1, -1), hi=(1, 1, 1), dt=dt,
                     tol_newton_rel=1e-13, tol_newton_abs=1e-13, tol_gmres_rel=1e-5, gmres_restart=80,
                     precision=hb.PREC_MIXED, pc=hb.PC_BJEXT if pc == "bjext" else hb.PC_NONE)
    X = disc.node_coords()
    if law == laws.EULER:
        W0 = inputs.density_wave(X)
    elif law == laws.BURGERS:
        W0 = 0.5 + 0.25 * inputs.sine_product(X, k=1.0)
    else:
        W0 = inputs.sine_product(X, k=1.0)
    b = W0 + dt * 0.1 * np.cos(3.0 * W0)
    opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-13, gmres_tol=1e-9, restart=80,
                                jv="linear" if disc.ph.linear else "fd")
    Wr, Sr, st = newton.newton_solve(disc, b, 1.0, 1.0, dt, W0, opts)
    Wd = torch.empty(disc.ndof, dtype=torch.float64, device="cuda")
    ctx.newton_solve(dev(b), 1.0, 1.0, dev(W0), Wd)
    assert rel(host(Wd), Wr.ravel()) <= 1e-11
    ctx.close()


def test_mixed_precision_c2_full_size_step_vs_exact(hb):
    """The bench workload in mixed precision: one HBPC(8,4) step of the 64x64,
    N=5 advection problem equals the exact per-Fourier-mode result."""
    dt = 1.0 / 96
    ctx, disc = pair(hb, laws.ADVECTION, 2, 5, (64, 64), a=(1.0, 1.0), q=8, kmax=4, dt=dt,
                     tol_newton_rel=1e-12, tol_newton_abs=1e-12, tol_gmres_rel=1e-5, gmres_restart=100,
                     pc=hb.PC_BJEXT, precision=hb.PREC_MIXED)
    w0 = inputs.sine_product(ctx.node_coords())
    ctx.set_state(w0)
    ctx.step(1)
    w = ctx.get_state()
    ref = exact.fourier_hbpc(disc, inputs.sine_product(disc.node_coords()), dt, 8, 4, 1)
    assert rel(w, ref) <= 1e-11
    ctx.close()


@pytest.mark.parametrize("flux", ["lf", "rusanov"])
def test_mixed_precision_euler_steps_vs_oracle(hb, flux):
    dt = 0.04
    ctx, disc = pair(hb, laws.EULER, 2, 3, (4, 3), LOBATTO, flux, lo=(-1, -1), hi=(1, 1), q=6, kmax=1,
                     dt=dt, tol_newton_rel=1e-13, tol_newton_abs=1e-13, tol_gmres_rel=1e-5,
                     gmres_restart=100, precision=hb.PREC_MIXED, pc=hb.PC_BJEXT)
    w0 = inputs.density_wave(ctx.node_coords())
    ctx.set_state(w0)
    ctx.step(2)
    w = ctx.get_state()
    opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-13, gmres_tol=1e-8, restart=100, jv="fd")
    adv = ohbpc.dg_stepper(disc, dt, 6, 1, opts)
    ref = inputs.density_wave(disc.node_coords())
    for _ in range(2):
        ref = adv(ref)
    assert rel(w, ref) <= 1e-11
    ctx.close()
