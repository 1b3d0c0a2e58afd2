"""Non-periodic boundaries on the GPU (hbpc_set_boundary): constant Dirichlet
exterior states and Euler slip walls through the numerical flux, against the
oracle's boundary treatment.  Tolerances as for the periodic parity tests:
R1 and R2 1e-12 of the largest entry, the linear Jv 1e-13 and the difference
quotients of Eq. 23 1e-6 relative, the FP32 analytic Jv 2e-5, block
preconditioners 1e-11, HBPC steps 1e-11 (FP64 stopping tests at 1e-13)."""
import numpy as np
import pytest
import torch

from oracle import dgsem, hbpc as ohbpc, laws, newton
from oracle.basis import GAUSS, LOBATTO
from paper_2109_04804_gb300 import inputs
from tests.test_gpu_parity import FAM, FLUX, LAWS, dev, host, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    import __graft_entry__ as g
    g.build()
    from paper_2109_04804_gb300 import hbpc
    assert torch.cuda.is_available()
    return hbpc


def euler_state_of(rho, vel, p, eps=1.0):
    return inputs.euler_from_primitive(np.array([rho]), [np.array([v]) for v in vel], np.array([p]),
                                       1.4, eps)[0]


def make(hb, law, dim, N, n, bcs, family=LOBATTO, flux="lf", eps=1.0, a=(1.0, -0.6, 0.35), **solver):
    """A context and its oracle twin with the boundaries bcs: one entry per
    direction, None (periodic) or (lo, hi) with "wall" or a Dirichlet state."""
    lo, hi = (-1.0, -1.0, -1.0), (1.0, 0.5, 0.7)
    ctx = hb.Context(dim, n, lo, hi, N, law=LAWS[law], flux=FLUX[flux], a=a, eps=eps, nodes=FAM[family],
                     **solver)
    spec = lambda b: ("wall",) if isinstance(b, str) else ("dirichlet", np.asarray(b, dtype=np.float64))
    obc = []
    for m, b in enumerate(bcs):
        if b is None:
            obc.append(None)
        else:
            ctx.set_boundary(m, b[0], b[1])
            obc.append((spec(b[0]), spec(b[1])))
    ph = laws.Physics(law, dim, a=a, eps=eps, flux=flux)
    disc = dgsem.Disc(dgsem.Mesh(dim, n, lo, hi, bc=obc), N, ph, family)
    return ctx, disc


def gas(disc, seed, amp=0.03):
    rng = np.random.default_rng(seed)
    X = disc.node_coords()
    base = inputs.density_wave(X, eps=disc.ph.eps)
    return base * (1.0 + amp * rng.standard_normal(base.shape))


# inflow and outflow states in 1-D, 2-D and 3-D (conservative variables)
IN = {d: euler_state_of(1.0, (0.3, 0.1, 0.05)[:d], 1.0) for d in (1, 2, 3)}
OUT = {d: euler_state_of(0.95, (0.3, 0.0, 0.0)[:d], 0.98) for d in (1, 2, 3)}

OP_CASES = [
    # law, dim, N, n, bcs, family, flux
    (laws.EULER, 2, 4, (5, 3), [(IN[2], OUT[2]), ("wall", "wall")], LOBATTO, "rusanov"),
    (laws.EULER, 2, 3, (4, 5), [("wall", "wall"), (IN[2], OUT[2])], GAUSS, "lf"),
    (laws.EULER, 3, 2, (3, 2, 4), [("wall", "wall"), None, (IN[3], OUT[3])], LOBATTO, "rusanov"),
    (laws.EULER, 1, 3, (9,), [("wall", OUT[1])], GAUSS, "rusanov"),
    (laws.ADVECTION, 2, 5, (6, 4), [([0.7], [-0.2]), None], LOBATTO, "lf"),
    (laws.BURGERS, 2, 3, (5, 4), [([0.4], [0.6]), ([0.5], [0.5])], GAUSS, "rusanov"),
]


@pytest.mark.parametrize("law,dim,N,n,bcs,family,flux", OP_CASES)
def test_operator_parity_with_boundaries(hb, law, dim, N, n, bcs, family, flux):
    ctx, disc = make(hb, law, dim, N, n, bcs, family, flux)
    rng = np.random.default_rng(71)
    w = gas(disc, 72) if law == laws.EULER else 0.5 + 0.3 * rng.standard_normal(disc.shape)
    s = rng.standard_normal(disc.shape)
    r1 = torch.empty(disc.ndof, dtype=torch.float64, device="cuda")
    r2 = torch.empty_like(r1)
    ctx.eval_R1(dev(w), r1)
    ctx.eval_R2(dev(w), dev(s), r2)
    ref1, ref2 = dgsem.R1(disc, w), dgsem.R2(disc, w, s)
    assert np.abs(host(r1) - ref1.ravel()).max() <= 1e-12 * np.abs(ref1).max()
    assert np.abs(host(r2) - ref2.ravel()).max() <= 1e-12 * np.abs(ref2).max()
    ctx.close()


@pytest.mark.parametrize("law,dim,N,n,bcs,family,flux", OP_CASES[:2] + OP_CASES[4:])
def test_jv_parity_with_boundaries(hb, law, dim, N, n, bcs, family, flux):
    """Eq. 23 (nonlinear) and Eq. 24 (advection: R1 of a Krylov vector sees
    the exterior direction zero, not the Dirichlet state)."""
    dt, a1, a2 = 0.05, 0.5, 1.0 / 6.0
    ctx, disc = make(hb, law, dim, N, n, bcs, family, flux, dt=dt)
    rng = np.random.default_rng(73)
    W = gas(disc, 74) if law == laws.EULER else 0.5 + 0.3 * rng.standard_normal(disc.shape)
    S = dgsem.R1(disc, W) + 0.05 * rng.standard_normal(disc.shape)
    X = np.concatenate([W.ravel(), S.ravel()])
    dX = rng.standard_normal(2 * disc.ndof)
    sysm = newton.StageSystem(disc, W, a1, a2, dt)
    _, r1, r2 = sysm.residual(X)
    mode = "linear" if disc.ph.linear else "fd"
    ref = sysm.jv(X, r1, r2, dX, mode)
    out = torch.empty(2 * disc.ndof, dtype=torch.float64, device="cuda")
    ctx.eval_Jv(a1, a2, dev(X), dev(dX), out)
    assert rel(host(out), ref) <= (1e-13 if disc.ph.linear else 1e-6)
    ctx.close()


@pytest.mark.parametrize("pc", ["bjext", "bjext_h"])
@pytest.mark.parametrize("case", [0, 1, 3, 5])
def test_block_preconditioners_with_boundaries(hb, pc, case):
    law, dim, N, n, bcs, family, flux = OP_CASES[case]
    dt = 0.1
    ctx, disc = make(hb, law, dim, N, n, bcs, family, flux, dt=dt,
                     pc=hb.PC_BJEXT if pc == "bjext" else hb.PC_BJEXT_H)
    rng = np.random.default_rng(75)
    W = gas(disc, 76, 0.02) if law == laws.EULER else 0.5 + 0.2 * rng.standard_normal(disc.shape)
    S = dgsem.R1(disc, W) + 0.05 * rng.standard_normal(disc.shape)
    X = np.concatenate([W.ravel(), S.ravel()])
    v = rng.standard_normal(2 * disc.ndof)
    ref = newton.make_preconditioner(newton.StageSystem(disc, W, 1.0, 1.0, dt), X, pc)(v)
    out = torch.empty(2 * disc.ndof, dtype=torch.float64, device="cuda")
    ctx.eval_pc(1.0, 1.0, dev(X), dev(v), out)
    assert rel(host(out), ref) <= 1e-11
    ctx.close()


def test_linear_advection_block_with_boundaries(hb):
    """Advection with Dirichlet ends keeps per-element blocks (the boundary
    elements' blocks differ from the interior ones)."""
    law, dim, N, n, bcs, family, flux = OP_CASES[4]
    dt = 0.1
    ctx, disc = make(hb, law, dim, N, n, bcs, family, flux, dt=dt, pc=hb.PC_BJEXT)
    rng = np.random.default_rng(77)
    W = rng.standard_normal(disc.shape)
    X = np.concatenate([W.ravel(), rng.standard_normal(disc.ndof)])
    v = rng.standard_normal(2 * disc.ndof)
    ref = newton.make_preconditioner(newton.StageSystem(disc, W, 1.0, 1.0, dt), X, "bjext")(v)
    out = torch.empty(2 * disc.ndof, dtype=torch.float64, device="cuda")
    ctx.eval_pc(1.0, 1.0, dev(X), dev(v), out)
    assert rel(host(out), ref) <= 1e-11
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_mixed_precision_jv_with_boundaries(hb, prec):
    """The FP32 analytic Jv (dual numbers through the exterior states) against
    the oracle's analytic form (global LF: constant dissipation), 2e-5 as for
    the periodic mixed test; FP64 against Eq. 23."""
    law, dim, N, n, bcs, family, flux = OP_CASES[1]
    dt, a1, a2 = 0.05, 1.0, 1.0
    ctx, disc = make(hb, law, dim, N, n, bcs, family, flux, dt=dt,
                     precision=hb.PREC_MIXED if prec == "mixed" else hb.PREC_FP64)
    rng = np.random.default_rng(78)
    W = gas(disc, 79)
    S = dgsem.R1(disc, W)
    X = np.concatenate([W.ravel(), S.ravel()])
    dX = rng.standard_normal(2 * disc.ndof)
    sysm = newton.StageSystem(disc, W, a1, a2, dt)
    _, r1, r2 = sysm.residual(X)
    ref = sysm.jv(X, r1, r2, dX, "analytic" if prec == "mixed" else "fd")
    out = torch.empty(2 * disc.ndof, dtype=torch.float64, device="cuda")
    ctx.eval_Jv(a1, a2, dev(X), dev(dX), out)
    assert rel(host(out), ref) <= (2e-5 if prec == "mixed" else 1e-6)
    ctx.close()


@pytest.mark.parametrize("pc", ["none", "bjext", "bjext_h"])
def test_euler_box_steps_vs_oracle(hb, pc):
    """Euler in a box of slip walls, HBPC(4, 1): the oracle's steps; mass and
    energy stay constant to rounding (walls pass no mass or energy)."""
    dt = 0.04
    pcs = {"none": hb.PC_NONE, "bjext": hb.PC_BJEXT, "bjext_h": hb.PC_BJEXT_H}
    ctx, disc = make(hb, laws.EULER, 2, 3, (4, 3), [("wall", "wall"), ("wall", "wall")], LOBATTO, "rusanov",
                     q=4, kmax=1, dt=dt, tol_newton_rel=1e-13, tol_newton_abs=1e-13, tol_gmres_rel=1e-9,
                     gmres_restart=100, pc=pcs[pc])
    w0 = gas(disc, 80, 0.02)
    ctx.set_state(w0)
    ctx.step(2)
    w = ctx.get_state()
    opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-13, gmres_tol=1e-9, restart=100, jv="fd")
    adv = ohbpc.dg_stepper(disc, dt, 4, 1, opts)
    ref = w0
    for _ in range(2):
        ref = adv(ref)
    assert rel(w, ref) <= 1e-11
    c0, c1 = dgsem.cell_integral(disc, w0), dgsem.cell_integral(disc, w)
    assert abs(c1[0] - c0[0]) <= 1e-12 * abs(c0[0]) and abs(c1[3] - c0[3]) <= 1e-12 * abs(c0[3])
    ctx.close()


def test_advection_pulse_leaves_through_dirichlet_ends(hb):
    """1-D advection with zero inflow data: HBPC(6, 2) steps equal the oracle's,
    and the pulse's mass leaves through the outflow end."""
    dt = 0.02
    ctx, disc = make(hb, laws.ADVECTION, 1, 4, (20,), [([0.0], [0.0])], LOBATTO, "lf", a=(1.0,), q=6, kmax=2,
                     dt=dt, tol_newton_rel=1e-13, tol_newton_abs=1e-13, tol_gmres_rel=1e-10, gmres_restart=100,
                     pc=hb.PC_BJEXT)
    x = disc.node_coords()[0]
    w0 = np.exp(-40.0 * (x - 0.8) ** 2)[:, None, :]
    ctx.set_state(w0)
    ctx.step(10)
    w = ctx.get_state()
    opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-13, gmres_tol=1e-10, restart=100, jv="linear")
    adv = ohbpc.dg_stepper(disc, dt, 6, 2, opts)
    ref = w0
    for _ in range(10):
        ref = adv(ref)
    assert rel(w, ref) <= 1e-11
    assert dgsem.cell_integral(disc, w)[0] < 0.9 * dgsem.cell_integral(disc, w0)[0]
    ctx.close()


def test_corrector_batch_with_boundaries(hb):
    res = []
    for batch in (False, True):
        ctx, disc = make(hb, laws.EULER, 2, 3, (4, 4), [(IN[2], OUT[2]), ("wall", "wall")], LOBATTO,
                         "rusanov", q=6, kmax=2, dt=0.03, tol_newton_rel=1e-13, tol_newton_abs=1e-13,
                         tol_gmres_rel=1e-10, gmres_restart=100, pc=hb.PC_BJEXT)
        if batch:
            ctx.set_corrector_batch(True)
        ctx.set_state(gas(disc, 81, 0.02))
        ctx.step(2)
        res.append(ctx.get_state())
        ctx.close()
    assert rel(res[1], res[0]) <= 1e-11


def test_boundary_argument_checks(hb):
    ctx = hb.Context(2, (3, 3), (0, 0), (1, 1), 3, law=hb.LAW_BURGERS)
    w = dev(0.5 + 0.1 * np.random.default_rng(82).standard_normal(ctx.ndof))
    r0 = torch.empty_like(w)
    ctx.eval_R1(w, r0)
    for args, code in (((0, None, [0.1]), 1),              # periodic at one end only
                       ((2, [0.1], [0.1]), 1),             # no such direction
                       ((0, "wall", "wall"), 1),           # a wall needs Euler
                       ((0, [float("nan")], [0.1]), 1)):   # non-finite state
        with pytest.raises(hb.HBPCError) as ei:
            ctx.set_boundary(*args)
        assert ei.value.status == code
    r1 = torch.empty_like(w)
    ctx.eval_R1(w, r1)
    assert torch.equal(r0, r1)          # nothing changed
    ctx.close()
    ctx = hb.Context(2, (3, 3), (0, 0), (1, 1), 3, law=hb.LAW_BURGERS, nu=0.01)
    with pytest.raises(hb.HBPCError) as ei:
        ctx.set_boundary(0, [0.1], [0.1])
    assert ei.value.status == 7
    ctx.close()
    ctx = hb.Context(2, (3, 3), (0, 0), (1, 1), 3, law=hb.LAW_EULER)
    with pytest.raises(hb.HBPCError) as ei:     # negative pressure
        ctx.set_boundary(1, [1.0, 0.0, 0.0, -1.0], "wall")
    assert ei.value.status == 1
    ctx.close()


# ---- Navier-Stokes: adiabatic no-slip walls and a lid (Dirichlet state) -------

def make_ns(hb, dim, N, n, bcs, family=LOBATTO, flux="lf", mu=0.05, **solver):
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    ctx = hb.Context(dim, n, lo, hi, N, law=hb.LAW_NAVIER_STOKES, flux=FLUX[flux], mu=mu, eps=1.0,
                     nodes=FAM[family], **solver)
    spec = lambda b: ("noslip",) if isinstance(b, str) else ("dirichlet", np.asarray(b, dtype=np.float64))
    obc = []
    for m, b in enumerate(bcs):
        if b is None:
            obc.append(None)
        else:
            ctx.set_boundary(m, b[0], b[1])
            obc.append((spec(b[0]), spec(b[1])))
    ph = laws.Physics(laws.NAVIER_STOKES, dim, flux=flux, mu=mu, eps=1.0)
    disc = dgsem.Disc(dgsem.Mesh(dim, n, lo, hi, bc=obc), N, ph, family)
    return ctx, disc


LID = {2: euler_state_of(1.0, (1.0, 0.0), 1.0 / 1.4), 3: euler_state_of(1.0, (1.0, 0.0, 0.0), 1.0 / 1.4)}
NS_CASES = [
    # dim, N, n, bcs, family, flux
    (2, 3, (4, 3), [("noslip", "noslip"), ("noslip", LID[2])], LOBATTO, "rusanov"),
    (2, 2, (3, 4), [("noslip", "noslip"), ("noslip", LID[2])], GAUSS, "lf"),
    (3, 2, (3, 2, 3), [("noslip", "noslip"), None, ("noslip", LID[3])], LOBATTO, "lf"),
]


def cavity_gas(disc, seed):
    X = disc.node_coords()
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.05 * np.sin(2.0 * X[0] + 0.3) + 0.01 * rng.standard_normal(X[0].shape)
    v = [0.2 * np.sin(np.pi * X[0]) * np.sin(np.pi * X[-1]) + 0.02 * rng.standard_normal(X[0].shape)
         for _ in range(disc.d)]
    p = 1.0 / 1.4 + 0.02 * np.cos(X[0] + X[-1])
    return inputs.euler_from_primitive(rho, v, p, 1.4, 1.0)


@pytest.mark.parametrize("dim,N,n,bcs,family,flux", NS_CASES)
def test_ns_operator_parity_with_walls(hb, dim, N, n, bcs, family, flux):
    ctx, disc = make_ns(hb, dim, N, n, bcs, family, flux)
    w = cavity_gas(disc, 101)
    s = np.random.default_rng(102).standard_normal(disc.shape)
    r1 = torch.empty(disc.ndof, dtype=torch.float64, device="cuda")
    r2 = torch.empty_like(r1)
    ctx.eval_R1(dev(w), r1)
    ctx.eval_R2(dev(w), dev(s), r2)
    ref1, ref2 = dgsem.R1(disc, w), dgsem.R2(disc, w, s)
    assert np.abs(host(r1) - ref1.ravel()).max() <= 1e-12 * np.abs(ref1).max()
    assert np.abs(host(r2) - ref2.ravel()).max() <= 1e-12 * np.abs(ref2).max()
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_ns_jv_and_blocks_with_walls(hb, prec):
    """Eq. 23 (FP64) / the FP32 analytic form (mixed, global LF) and the BJ_ext
    blocks (assembled by columns of the frozen-neighbour R2) at walls and lid."""
    dim, N, n, bcs, family, flux = NS_CASES[1]
    dt, a1, a2 = 0.02, 0.5, 1.0 / 6.0
    ctx, disc = make_ns(hb, dim, N, n, bcs, family, flux, dt=dt, pc=hb.PC_BJEXT,
                        precision=hb.PREC_MIXED if prec == "mixed" else hb.PREC_FP64)
    rng = np.random.default_rng(103)
    W = cavity_gas(disc, 104)
    S = dgsem.R1(disc, W) + 0.05 * rng.standard_normal(disc.shape)
    X = np.concatenate([W.ravel(), S.ravel()])
    dX = rng.standard_normal(2 * disc.ndof)
    sysm = newton.StageSystem(disc, W, a1, a2, dt)
    _, r1, r2 = sysm.residual(X)
    ref = sysm.jv(X, r1, r2, dX, "analytic" if prec == "mixed" else "fd")
    out = torch.empty(2 * disc.ndof, dtype=torch.float64, device="cuda")
    ctx.eval_Jv(a1, a2, dev(X), dev(dX), out)
    assert rel(host(out), ref) <= (2e-5 if prec == "mixed" else 1e-6)
    v = rng.standard_normal(2 * disc.ndof)
    refp = newton.make_preconditioner(sysm, X, "bjext")(v)
    ctx.eval_pc(a1, a2, dev(X), dev(v), out)
    assert rel(host(out), refp) <= (1e-4 if prec == "mixed" else 1e-11)
    ctx.close()


def test_lid_driven_cavity_steps_vs_oracle(hb):
    """The paper's lid-driven cavity setting on a small mesh: walls left, right
    and below, the lid state (rho 1, v (1, 0), p 1/gamma) above; HBPC(4, 1)
    steps equal the oracle's and the lid sets the gas in motion."""
    dt = 0.01
    ctx, disc = make_ns(hb, 2, 2, (3, 3), [("noslip", "noslip"), ("noslip", LID[2])], LOBATTO, "rusanov",
                        mu=0.025, q=4, kmax=1, dt=dt, tol_newton_rel=1e-13, tol_newton_abs=1e-13,
                        tol_gmres_rel=1e-9, gmres_restart=100, pc=hb.PC_BJEXT)
    X = disc.node_coords()
    w0 = inputs.euler_from_primitive(np.ones_like(X[0]), [0 * X[0], 0 * X[0]], np.full_like(X[0], 1 / 1.4))
    ctx.set_state(w0)
    ctx.step(2)
    w = ctx.get_state()
    opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-13, gmres_tol=1e-9, restart=100, jv="fd")
    adv = ohbpc.dg_stepper(disc, dt, 4, 1, opts)
    ref = w0
    for _ in range(2):
        ref = adv(ref)
    assert rel(w, ref) <= 1e-11
    assert np.abs(w - w0).max() > 1e-4          # the lid drives the flow
    ctx.close()


def test_ns_noslip_box_conserves_mass_and_energy_on_the_gpu(hb):
    """Steps of a gas in a box of adiabatic no-slip walls keep total mass and
    energy to rounding (the walls pass neither, see the oracle's pins)."""
    ctx, disc = make_ns(hb, 2, 3, (4, 4), [("noslip", "noslip"), ("noslip", "noslip")], LOBATTO, "rusanov",
                        mu=0.02, q=4, kmax=1, dt=0.01, tol_newton_rel=1e-12, tol_newton_abs=1e-13,
                        tol_gmres_rel=1e-9, gmres_restart=100, pc=hb.PC_BJEXT)
    w0 = cavity_gas(disc, 105)
    ctx.set_state(w0)
    ctx.step(3)
    w = ctx.get_state()
    c0, c1 = dgsem.cell_integral(disc, w0), dgsem.cell_integral(disc, w)
    assert abs(c1[0] - c0[0]) <= 1e-12 * abs(c0[0]) and abs(c1[3] - c0[3]) <= 1e-12 * abs(c0[3])
    assert np.abs(w - w0).max() > 1e-5
    ctx.close()
