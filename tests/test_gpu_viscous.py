"""Parity of the CUDA path's BR2 viscous term (Sec. 5.1.1, scalar laws) with the
FP64 oracle, through the C-ABI.  Tolerances follow the inviscid parity tests:
element-wise 1e-12 of the largest term for the operators (same sums, other
order), 1e-6 for the Eq. 23 difference quotients, 1e-11 relative L2 for Newton
and HBPC results stopped on 1e-13 tolerances."""
import numpy as np
import pytest
import torch

from oracle import dgsem, exact, hbpc as ohbpc, laws, newton
from oracle.basis import GAUSS, LOBATTO
from paper_2109_04804_gb300 import inputs

pytestmark = pytest.mark.gpu

LAWS = {laws.ADVECTION: 0, laws.BURGERS: 1}
FLUX = {"lf": 0, "rusanov": 1}
FAM = {LOBATTO: 0, GAUSS: 1}


@pytest.fixture(scope="module")
def hb():
    import __graft_entry__ as g
    g.build()
    from paper_2109_04804_gb300 import hbpc
    assert torch.cuda.is_available()
    return hbpc


def pair(hb, law, dim, N, n, nu, family=LOBATTO, flux="lf", eta=None, lo=(0, 0, 0), hi=(1, 1, 1),
         a=(1.0, -0.6, 0.35), **solver):
    ctx = hb.Context(dim, n, lo, hi, N, law=LAWS[law], flux=FLUX[flux], a=a, nu=nu,
                     eta_br2=0.0 if eta is None else eta, nodes=FAM[family], **solver)
    ph = laws.Physics(law, dim, a=a, flux=flux, nu=nu, eta_br2=eta)
    disc = dgsem.Disc(dgsem.Mesh(dim, n, lo, hi), N, ph, family)
    return ctx, disc


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def mesh_for(dim):
    return {1: (37,), 2: (7, 5), 3: (3, 4, 2)}[dim]


OP_CASES = (
    [(laws.ADVECTION, d, N, LOBATTO, "lf", 0.05, None) for d in (1, 2, 3) for N in (1, 3, 5, 7)]
    + [(laws.ADVECTION, d, N, GAUSS, "lf", 0.02, None) for d in (1, 2) for N in (2, 3)]
    + [(laws.BURGERS, d, N, LOBATTO, f, 0.01, None) for d in (1, 2, 3) for N in (3, 5)
       for f in ("lf", "rusanov")]
    + [(laws.BURGERS, 2, 3, GAUSS, "rusanov", 0.03, None),
       (laws.BURGERS, 2, 4, LOBATTO, "lf", 0.02, 6.5), (laws.ADVECTION, 1, 3, GAUSS, "lf", 0.1, 1.0)]
)


@pytest.mark.parametrize("law,dim,N,family,flux,nu,eta", OP_CASES)
def test_r1_r2_parity_viscous(hb, law, dim, N, family, flux, nu, eta):
    ctx, disc = pair(hb, law, dim, N, mesh_for(dim), nu, family, flux, eta)
    rng = np.random.default_rng(300 + dim * 10 + N)
    w = rng.standard_normal(disc.shape)
    s = rng.standard_normal(disc.shape)
    r1_ref = dgsem.R1(disc, w)
    r2_ref = dgsem.R2(disc, w, s)
    out = torch.empty_like(dev(w))
    ctx.eval_R1(dev(w), out)
    r1 = host(out)
    ctx.eval_R2(dev(w), dev(s), out)
    r2 = host(out)
    for got, ref in ((r1, r1_ref), (r2, r2_ref)):
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    # the viscous part is really there: differs from the inviscid operator
    ph0 = laws.Physics(law, dim, a=(1.0, -0.6, 0.35), flux=flux)
    disc0 = dgsem.Disc(disc.mesh, N, ph0, family)
    assert rel(r1, dgsem.R1(disc0, w)) > 1e-3
    ctx.close()


@pytest.mark.parametrize("law,flux", [(laws.ADVECTION, "lf"), (laws.BURGERS, "lf"),
                                      (laws.BURGERS, "rusanov")])
def test_residual_and_jv_parity_viscous(hb, law, flux):
    dim, N, dt = 2, 3, 0.03
    ctx, disc = pair(hb, law, dim, N, mesh_for(dim), 0.02, LOBATTO, flux, dt=dt)
    rng = np.random.default_rng(8)
    W = 0.5 + 0.3 * rng.standard_normal(disc.shape)
    S = dgsem.R1(disc, W) + 0.01 * rng.standard_normal(disc.shape)
    b = W + 0.01 * rng.standard_normal(disc.shape)
    a1, a2 = 0.5, 1.0 / 6.0
    sysm = newton.StageSystem(disc, b, a1, a2, dt)
    X = np.concatenate([W.ravel(), S.ravel()])
    G_ref, r1, r2 = sysm.residual(X)
    Gd = torch.empty(2 * disc.ndof, dtype=torch.float64, device="cuda")
    ctx.eval_G(dev(b), a1, a2, dev(X), Gd)
    assert np.abs(host(Gd) - G_ref).max() <= 1e-12 * np.abs(G_ref).max()
    dX = rng.standard_normal(2 * disc.ndof)
    out = torch.empty_like(Gd)
    ctx.eval_Jv(a1, a2, dev(X), dev(dX), out)
    if disc.ph.linear:
        assert rel(host(out), sysm.jv(X, r1, r2, dX, "linear")) <= 1e-13
    else:
        assert rel(host(out), sysm.jv(X, r1, r2, dX, "fd")) <= 1e-6
    ctx.close()


@pytest.mark.parametrize("law,dim,N,family,flux", [
    (laws.ADVECTION, 2, 5, LOBATTO, "lf"), (laws.ADVECTION, 1, 3, GAUSS, "lf"),
    (laws.BURGERS, 2, 3, LOBATTO, "rusanov"), (laws.BURGERS, 2, 3, GAUSS, "lf"),
    (laws.BURGERS, 3, 2, LOBATTO, "lf")])
def test_bjext_apply_parity_viscous(hb, law, dim, N, family, flux):
    """BJ_ext with the viscous element-diagonal block in J_i against the
    oracle's dense construction from the frozen-neighbour R2."""
    dt = 0.04
    ctx, disc = pair(hb, law, dim, N, mesh_for(dim), 0.03, family, flux, lo=(-1, -1, -1), hi=(1, 1, 1),
                     dt=dt, pc=hb.PC_BJEXT)
    rng = np.random.default_rng(41)
    W = 0.5 + 0.2 * rng.standard_normal(disc.shape)
    X = np.concatenate([W.ravel(), dgsem.R1(disc, W).ravel()])
    v = rng.standard_normal(2 * disc.ndof)
    sysm = newton.StageSystem(disc, W, 1.0, 1.0, dt)
    ref = newton.BJExt(sysm, W)(v)
    out = torch.empty(2 * disc.ndof, dtype=torch.float64, device="cuda")
    ctx.eval_pc(1.0, 1.0, dev(X), dev(v), out)
    assert rel(host(out), ref) <= 1e-11
    ctx.close()


@pytest.mark.parametrize("law,flux,pc,prec", [
    (laws.BURGERS, "rusanov", "none", "fp64"), (laws.BURGERS, "lf", "bjext", "fp64"),
    (laws.ADVECTION, "lf", "bjext", "fp64"), (laws.BURGERS, "rusanov", "bjext", "mixed"),
    (laws.ADVECTION, "lf", "none", "mixed")])
def test_newton_solve_parity_viscous(hb, law, flux, pc, prec):
    N, dt, nu = 3, 0.05, 0.02
    ctx, disc = pair(hb, law, 2, N, (5, 4), nu, LOBATTO, flux, lo=(-1, -1), hi=(1, 1), dt=dt,
                     tol_newton_rel=1e-13, tol_newton_abs=1e-13,
                     tol_gmres_rel=1e-9 if prec == "fp64" else 1e-5, gmres_restart=80,
                     pc=hb.PC_BJEXT if pc == "bjext" else hb.PC_NONE,
                     precision=hb.PREC_MIXED if prec == "mixed" else hb.PREC_FP64)
    X = disc.node_coords()
    W0 = 0.5 + 0.25 * inputs.sine_product(X, k=1.0)
    b = W0 + dt * 0.1 * np.cos(3.0 * W0)
    opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-13, gmres_tol=1e-9, restart=80,
                                jv="linear" if disc.ph.linear else "fd")
    Wr, Sr, _ = newton.newton_solve(disc, b, 1.0, 1.0, dt, W0, opts)
    Wd = torch.empty(disc.ndof, dtype=torch.float64, device="cuda")
    Sd = torch.empty_like(Wd)
    ctx.newton_solve(dev(b), 1.0, 1.0, dev(W0), Wd, Sd)
    assert rel(host(Wd), Wr.ravel()) <= 1e-11
    assert rel(host(Sd), Sr.ravel()) <= 1e-10
    ctx.close()


@pytest.mark.parametrize("q,kmax,pc", [(4, 1, "none"), (6, 2, "bjext"), (8, 4, "bjext")])
def test_advection_diffusion_steps_vs_exact(hb, q, kmax, pc):
    """2-D advection-diffusion: three HBPC steps equal the exact per-Fourier-mode
    HBPC result of the oracle's advection-diffusion symbol."""
    dt, nu = 0.01, 0.01
    ctx, disc = pair(hb, laws.ADVECTION, 2, 5, (6, 5), nu, a=(1.0, 1.0), q=q, kmax=kmax, dt=dt,
                     tol_newton_rel=1e-13, tol_newton_abs=1e-13, tol_gmres_rel=1e-9, gmres_restart=100,
                     pc=hb.PC_BJEXT if pc == "bjext" else hb.PC_NONE)
    w0 = inputs.sine_product(ctx.node_coords())
    ctx.set_state(w0)
    ctx.step(3)
    w = ctx.get_state()
    ref = exact.fourier_hbpc(disc, inputs.sine_product(disc.node_coords()), dt, q, kmax, 3)
    assert rel(w, ref) <= 1e-11
    ctx.close()


def test_heat_decay_full_run(hb):
    """u_t = nu Laplace(u) on [0,1]^2 (a = 0) from sin(2 pi x) sin(2 pi y): after
    T = 0.5 the mode has decayed by exp(-8 pi^2 nu T) up to the method's error."""
    nu, dt, steps = 0.02, 0.05, 10
    ctx, disc = pair(hb, laws.ADVECTION, 2, 6, (8, 8), nu, a=(0.0, 0.0), q=6, kmax=2, dt=dt,
                     tol_newton_rel=1e-13, tol_newton_abs=1e-13, tol_gmres_rel=1e-10, gmres_restart=100,
                     pc=hb.PC_BJEXT)
    w0 = inputs.sine_product(ctx.node_coords())
    ctx.set_state(w0)
    ctx.step(steps)
    w = ctx.get_state()
    ex = np.exp(-8 * np.pi ** 2 * nu * dt * steps) * w0
    assert rel(w, ex) < 1e-6
    ctx.close()


@pytest.mark.parametrize("flux", ["lf", "rusanov"])
def test_viscous_burgers_steps_vs_oracle(hb, flux):
    dt, nu = 0.02, 0.01
    ctx, disc = pair(hb, laws.BURGERS, 2, 3, (5, 4), nu, LOBATTO, flux, q=6, kmax=1, dt=dt,
                     tol_newton_rel=1e-13, tol_newton_abs=1e-13, tol_gmres_rel=1e-8, gmres_restart=100,
                     pc=hb.PC_BJEXT)
    w0 = inputs.burgers_fourier(ctx.node_coords(), seed=3)
    ctx.set_state(w0)
    ctx.step(2)
    w = ctx.get_state()
    opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-13, gmres_tol=1e-8, restart=100, jv="fd")
    adv = ohbpc.dg_stepper(disc, dt, 6, 1, opts)
    ref = inputs.burgers_fourier(disc.node_coords(), seed=3)
    for _ in range(2):
        ref = adv(ref)
    assert rel(w, ref) <= 1e-11
    c0 = dgsem.cell_integral(disc, inputs.burgers_fourier(disc.node_coords(), seed=3))
    assert np.all(np.abs(dgsem.cell_integral(disc, w) - c0) <= 1e-12 * np.abs(w).max())
    ctx.close()
