"""Parity of the CUDA path's Navier-Stokes viscous term (Sec. 5: Eq. 25 with the
BR2 lifting of (v, T), Sec. 5.1.1, and its linearisation for R^(2), Sec. 5.1.2)
with the FP64 oracle, through the C-ABI.

Tolerances: the operators sum the same terms as the oracle in another order
(element-wise 1e-12 of the largest term); the Eq. 23 difference quotients
agree to 1e-6; Newton and HBPC results stopped on 1e-13 tolerances agree to
1e-11 relative L2 (the Newton residual is FP64 in both precisions); FP32
preconditioner blocks agree to 1e-4."""
import numpy as np
import pytest
import torch

from oracle import dgsem, hbpc as ohbpc, laws, newton
from oracle.basis import GAUSS, LOBATTO
from paper_2109_04804_gb300 import inputs

pytestmark = pytest.mark.gpu

FLUX = {"lf": 0, "rusanov": 1}
FAM = {LOBATTO: 0, GAUSS: 1}


@pytest.fixture(scope="module")
def hb():
    import __graft_entry__ as g
    g.build()
    from paper_2109_04804_gb300 import hbpc
    assert torch.cuda.is_available()
    return hbpc


def pair(hb, dim, N, n, mu, family=LOBATTO, flux="lf", eta=None, lo=(0, 0, 0), hi=(1, 1, 1), eps=1.0,
         prandtl=0.72, **solver):
    ctx = hb.Context(dim, n, lo, hi, N, law=hb.LAW_NAVIER_STOKES, flux=FLUX[flux], mu=mu, eps=eps,
                     prandtl=prandtl, eta_br2=0.0 if eta is None else eta, nodes=FAM[family], **solver)
    ph = laws.Physics(laws.NAVIER_STOKES, dim, flux=flux, mu=mu, eta_br2=eta, eps=eps, prandtl=prandtl)
    disc = dgsem.Disc(dgsem.Mesh(dim, n, lo, hi), N, ph, family)
    return ctx, disc


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def random_state(disc, seed, amp=0.3):
    """Positive density and pressure with random nodal perturbations."""
    rng = np.random.default_rng(seed)
    shp = disc.shape[:1] + disc.shape[2:]
    rho = 1.0 + 0.2 * rng.random(shp)
    v = [amp * rng.standard_normal(shp) for _ in range(disc.d)]
    p = 1.0 + 0.2 * rng.random(shp)
    return inputs.euler_from_primitive(rho, v, p, disc.ph.gamma, disc.ph.eps)


def smooth_state(disc):
    X = disc.node_coords()
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * X[0]) * np.cos(2 * np.pi * X[1])
    v = [0.3 * np.sin(2 * np.pi * X[1]), 0.2 * np.cos(2 * np.pi * X[0])] + ([0.1 * np.sin(2 * np.pi * X[2])]
                                                                        if disc.d == 3 else [])
    p = 1.0 + 0.1 * np.cos(2 * np.pi * (X[0] - X[1]))
    return inputs.euler_from_primitive(rho, v, p, disc.ph.gamma, disc.ph.eps)


def mesh_for(dim):
    return {2: (5, 4), 3: (3, 2, 2)}[dim]


OP_CASES = ([(2, N, LOBATTO, f) for N in (2, 3, 4, 5) for f in ("lf", "rusanov")]
            + [(2, N, GAUSS, "rusanov") for N in (2, 3)]
            + [(3, N, LOBATTO, "rusanov") for N in (2, 3, 4, 5)])


@pytest.mark.parametrize("dim,N,family,flux", OP_CASES)
def test_r1_r2_parity_navier_stokes(hb, dim, N, family, flux):
    ctx, disc = pair(hb, dim, N, mesh_for(dim), 0.02, family, flux, lo=(-1, 0, 0.5), hi=(1, 2, 1.0), eps=0.7)
    w = random_state(disc, 500 + 10 * dim + N)
    s = np.random.default_rng(600 + N).standard_normal(disc.shape)
    r1_ref = dgsem.R1(disc, w)
    r2_ref = dgsem.R2(disc, w, s)
    out = torch.empty_like(dev(w))
    ctx.eval_R1(dev(w), out)
    r1 = host(out)
    ctx.eval_R2(dev(w), dev(s), out)
    r2 = host(out)
    for got, ref in ((r1, r1_ref), (r2, r2_ref)):
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    # the viscous part is there: the operators differ from the Euler ones
    eu = dgsem.Disc(disc.mesh, N, laws.Physics(laws.EULER, dim, flux=flux, eps=0.7), family)
    assert rel(r1, dgsem.R1(eu, w)) > 1e-3
    assert rel(r2, dgsem.R2(eu, w, s)) > 1e-3
    ctx.close()


def test_eta_and_prandtl_reach_the_kernel(hb):
    ctx, disc = pair(hb, 2, 3, (4, 4), 0.05, eta=7.0, prandtl=0.3)
    w = random_state(disc, 77)
    out = torch.empty_like(dev(w))
    ctx.eval_R1(dev(w), out)
    ref = dgsem.R1(disc, w)
    assert np.abs(host(out) - ref).max() <= 1e-12 * np.abs(ref).max()
    ctx.close()


@pytest.mark.parametrize("flux", ["lf", "rusanov"])
def test_residual_and_jv_parity_navier_stokes(hb, flux):
    dim, N, dt = 2, 3, 0.02
    ctx, disc = pair(hb, dim, N, (4, 5), 0.03, LOBATTO, flux, dt=dt)
    rng = np.random.default_rng(18)
    W = smooth_state(disc)
    S = dgsem.R1(disc, W) + 0.01 * rng.standard_normal(disc.shape)
    b = W + 0.001 * rng.standard_normal(disc.shape)
    a1, a2 = 0.5, 1.0 / 6.0
    sysm = newton.StageSystem(disc, b, a1, a2, dt)
    X = np.concatenate([W.ravel(), S.ravel()])
    G_ref, r1, r2 = sysm.residual(X)
    Gd = torch.empty(2 * disc.ndof, dtype=torch.float64, device="cuda")
    ctx.eval_G(dev(b), a1, a2, dev(X), Gd)
    # G is a small difference of O(1) terms: compare on the scale of the terms
    scale = max(np.abs(W).max(), np.abs(S).max(), np.abs(r1).max(), np.abs(G_ref).max())
    assert np.abs(host(Gd) - G_ref).max() <= 1e-12 * scale
    dX = rng.standard_normal(2 * disc.ndof)
    out = torch.empty_like(Gd)
    ctx.eval_Jv(a1, a2, dev(X), dev(dX), out)
    assert rel(host(out), sysm.jv(X, r1, r2, dX, "fd")) <= 1e-6
    ctx.close()


@pytest.mark.parametrize("dim,N,family,flux,prec", [
    (2, 2, LOBATTO, "rusanov", "fp64"), (2, 3, LOBATTO, "lf", "fp64"), (2, 2, GAUSS, "rusanov", "fp64"),
    (3, 2, LOBATTO, "rusanov", "fp64"), (2, 3, LOBATTO, "rusanov", "mixed")])
def test_bjext_apply_parity_navier_stokes(hb, dim, N, family, flux, prec):
    """BJ_ext with J_i assembled by columns of the frozen-neighbour R2 against
    the oracle's dense construction (the same definition, evaluated by the
    oracle's operator on unit vectors)."""
    dt = 0.03
    n = {2: (3, 4), 3: (2, 3, 2)}[dim]
    ctx, disc = pair(hb, dim, N, n, 0.04, family, flux, lo=(-1, -1, -1), hi=(1, 1, 1), dt=dt,
                     pc=hb.PC_BJEXT, precision=hb.PREC_MIXED if prec == "mixed" else hb.PREC_FP64)
    rng = np.random.default_rng(43)
    W = random_state(disc, 44, amp=0.2)
    X = np.concatenate([W.ravel(), dgsem.R1(disc, W).ravel()])
    v = rng.standard_normal(2 * disc.ndof)
    sysm = newton.StageSystem(disc, W, 1.0, 1.0, dt)
    ref = newton.BJExt(sysm, W)(v)
    out = torch.empty(2 * disc.ndof, dtype=torch.float64, device="cuda")
    ctx.eval_pc(1.0, 1.0, dev(X), dev(v), out)
    assert rel(host(out), ref) <= (1e-4 if prec == "mixed" else 1e-11)
    ctx.close()


@pytest.mark.parametrize("flux,pc,prec", [("rusanov", "none", "fp64"), ("lf", "bjext", "fp64"),
                                          ("rusanov", "bjext", "mixed"), ("lf", "none", "mixed")])
def test_newton_solve_parity_navier_stokes(hb, flux, pc, prec):
    N, dt, mu = 3, 0.02, 0.02
    ctx, disc = pair(hb, 2, N, (4, 4), mu, LOBATTO, flux, dt=dt, tol_newton_rel=1e-13, tol_newton_abs=1e-13,
                     tol_gmres_rel=1e-9 if prec == "fp64" else 1e-5, gmres_restart=80,
                     pc=hb.PC_BJEXT if pc == "bjext" else hb.PC_NONE,
                     precision=hb.PREC_MIXED if prec == "mixed" else hb.PREC_FP64)
    W0 = smooth_state(disc)
    b = W0 + dt * 0.05 * np.sin(3.0 * W0)
    opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-13, gmres_tol=1e-9, restart=80, jv="fd")
    Wr, Sr, _ = newton.newton_solve(disc, b, 1.0, 1.0, dt, W0, opts)
    Wd = torch.empty(disc.ndof, dtype=torch.float64, device="cuda")
    Sd = torch.empty_like(Wd)
    ctx.newton_solve(dev(b), 1.0, 1.0, dev(W0), Wd, Sd)
    assert rel(host(Wd), Wr.ravel()) <= 1e-11
    assert rel(host(Sd), Sr.ravel()) <= 1e-10
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_navier_stokes_steps_vs_oracle(hb, prec):
    """Two HBPC(6,1) steps of a 2-D viscous flow against the oracle; mass,
    momentum and energy are conserved (periodic, central viscous fluxes)."""
    dt = 0.02
    ctx, disc = pair(hb, 2, 3, (4, 3), 0.01, LOBATTO, "rusanov", q=6, kmax=1, dt=dt, tol_newton_rel=1e-13,
                     tol_newton_abs=1e-13, tol_gmres_rel=1e-8 if prec == "fp64" else 1e-5, gmres_restart=100,
                     pc=hb.PC_BJEXT, precision=hb.PREC_MIXED if prec == "mixed" else hb.PREC_FP64)
    w0 = smooth_state(disc)
    ctx.set_state(w0)
    ctx.step(2)
    w = ctx.get_state()
    opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-13, gmres_tol=1e-8, restart=100, jv="fd")
    adv = ohbpc.dg_stepper(disc, dt, 6, 1, opts)
    ref = w0
    for _ in range(2):
        ref = adv(ref)
    assert rel(w, ref) <= 1e-11
    c0 = dgsem.cell_integral(disc, w0)
    assert np.all(np.abs(dgsem.cell_integral(disc, w) - c0) <= 1e-12 * np.abs(c0).max())
    ctx.close()


def test_taylor_green_3d_step_vs_oracle(hb):
    """One HBPC(4,1) step of a small 3-D Taylor-Green vortex (Mach 0.1 through
    the reference Mach number, Re 1600) against the oracle."""
    dt = 0.05
    two_pi = 2 * np.pi
    ctx, disc = pair(hb, 3, 2, (2, 2, 2), 1.0 / 1600, LOBATTO, "rusanov", lo=(0, 0, 0), hi=(two_pi,) * 3,
                     eps=0.1, q=4, kmax=1, dt=dt, tol_newton_rel=1e-12, tol_newton_abs=1e-12,
                     tol_gmres_rel=1e-8, gmres_restart=100)
    w0 = inputs.taylor_green(ctx.node_coords(), eps=0.1)
    ctx.set_state(w0)
    ctx.step(1)
    w = ctx.get_state()
    opts = newton.NewtonOptions(tol_rel=1e-12, tol_abs=1e-12, gmres_tol=1e-8, restart=100, jv="fd")
    ref = ohbpc.dg_stepper(disc, dt, 4, 1, opts)(inputs.taylor_green(disc.node_coords(), eps=0.1))
    assert rel(w, ref) <= 1e-10
    ctx.close()


def test_taylor_green_full_size_sampled_parity(hb):
    """The bench's Taylor-Green configuration at full size (32^3 elements,
    N = 5, 35.4 M values): R1 and R2 on sampled elements against the oracle.
    An element's operators depend only on it and its face neighbours (BR2 is
    compact), so the oracle evaluates a periodic 3 x 3 x 3 patch of elements
    centred on the sample and its centre element is compared."""
    n, N = 32, 5
    L = 2 * np.pi
    ctx = hb.Context(3, (n, n, n), (0, 0, 0), (L, L, L), N, law=hb.LAW_NAVIER_STOKES, flux=FLUX["rusanov"],
                     mu=1.0 / 1600, eps=0.1, q=4, kmax=0, dt=0.02, gmres_restart=2)
    w = inputs.taylor_green(ctx.node_coords(), eps=0.1)
    rng = np.random.default_rng(70)
    w = w * (1.0 + 1e-3 * rng.standard_normal(w.shape))
    s = rng.standard_normal(w.shape)
    wd, sd = dev(w), dev(s)
    out = torch.empty_like(wd)
    ctx.eval_R1(wd, out)
    r1 = host(out)
    ctx.eval_R2(wd, sd, out)
    r2 = host(out)
    ctx.close()
    del wd, sd, out
    h = L / n
    ph = laws.Physics(laws.NAVIER_STOKES, 3, flux="rusanov", mu=1.0 / 1600, eps=0.1)
    patch = dgsem.Disc(dgsem.Mesh(3, (3, 3, 3), (0, 0, 0), (3 * h,) * 3), N, ph, LOBATTO)
    for e in rng.integers(0, n ** 3, size=8):
        ex, ey, ez = e % n, (e // n) % n, e // (n * n)
        idx = [((ex + a) % n) + n * (((ey + b) % n) + n * ((ez + c) % n))
               for c in (-1, 0, 1) for b in (-1, 0, 1) for a in (-1, 0, 1)]
        ref1 = dgsem.R1(patch, w[idx])[13]
        ref2 = dgsem.R2(patch, w[idx], s[idx])[13]
        assert np.abs(r1[e] - ref1).max() <= 1e-12 * np.abs(ref1).max(), e
        assert np.abs(r2[e] - ref2).max() <= 1e-12 * np.abs(ref2).max(), e


@pytest.mark.parametrize("dim,n", [(2, (1, 4)), (3, (2, 1, 3))])
def test_single_element_direction_is_its_own_neighbour(hb, dim, n):
    """A direction with one element: the element is its own periodic neighbour
    across both faces (the degenerate mesh of the lifting and the fluxes)."""
    ctx, disc = pair(hb, dim, 3 if dim == 2 else 2, n, 0.03, LOBATTO, "rusanov", lo=(0, 0, 0), hi=(1.0, 0.5, 2.0))
    w = random_state(disc, 900 + dim)
    s = np.random.default_rng(901).standard_normal(disc.shape)
    out = torch.empty_like(dev(w))
    ctx.eval_R1(dev(w), out)
    ref = dgsem.R1(disc, w)
    assert np.abs(host(out) - ref).max() <= 1e-12 * np.abs(ref).max()
    ctx.eval_R2(dev(w), dev(s), out)
    ref = dgsem.R2(disc, w, s)
    assert np.abs(host(out) - ref).max() <= 1e-12 * np.abs(ref).max()
    ctx.close()
