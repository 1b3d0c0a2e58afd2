"""The shared FP64 BJ_ext block applied on the tensor cores (digit-plane
splitting of P = [[M, -c2 J M], [J M, M - c1 J M]] and of every element's
(w, sigma), BF16 products summed exactly in FP32 tensor memory): the result
against the oracle's dense construction (Sec. 3.2.3), against the FP64
CUDA-core apply (HBPC_PC_TC=0) element by element, with unbalanced halves,
NaN propagation per element, and whole HBPC steps."""
import os

import numpy as np
import pytest
import torch

from oracle import dgsem, laws, newton
from oracle import hbpc as ohbpc
from oracle.basis import LOBATTO
from paper_2109_04804_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    import __graft_entry__ as g
    g.build()
    from paper_2109_04804_gb300 import hbpc
    assert torch.cuda.is_available()
    return hbpc


def make(hb, dim, N, n, tc, **kw):
    old = os.environ.get("HBPC_PC_TC")
    os.environ["HBPC_PC_TC"] = "1" if tc else "0"
    try:
        a = (1.0, 0.5, 0.25)[:dim]
        ctx = hb.Context(dim, n, (-1.0,) * dim, (1.0,) * dim, N, law=hb.LAW_ADVECTION, a=a, pc=hb.PC_BJEXT, **kw)
    finally:
        if old is None:
            del os.environ["HBPC_PC_TC"]
        else:
            os.environ["HBPC_PC_TC"] = old
    return ctx


def oracle_disc(dim, N, n):
    ph = laws.Physics(laws.ADVECTION, dim, a=(1.0, 0.5, 0.25)[:dim])
    return dgsem.Disc(dgsem.Mesh(dim, n, (-1.0,) * dim, (1.0,) * dim), N, ph, LOBATTO)


def dev(x):
    return torch.tensor(np.ascontiguousarray(x).ravel(), dtype=torch.float64, device="cuda")


def apply(ctx, X, v, a1, a2):
    out = torch.empty(v.size, dtype=torch.float64, device="cuda")
    ctx.eval_pc(a1, a2, dev(X), dev(v), out)
    return out.cpu().numpy()


CASES = [(1, 3, (40,)), (2, 3, (7, 5)), (2, 5, (9, 7)), (2, 4, (64, 3)), (3, 2, (4, 3, 5))]


@pytest.mark.parametrize("dim,N,n", CASES)
def test_tc_apply_matches_oracle_and_cuda_core_apply(hb, dim, N, n):
    dt, a1, a2 = 0.05, 1.0, 1.0
    disc = oracle_disc(dim, N, n)
    rng = np.random.default_rng(200 + N)
    W = 0.5 + 0.2 * rng.standard_normal(disc.shape)
    X = np.concatenate([W.ravel(), dgsem.R1(disc, W).ravel()])
    # the halves 1e3 apart, as sigma ~ R1(w) on a fine mesh
    v = np.concatenate([rng.standard_normal(disc.ndof), 1e3 * rng.standard_normal(disc.ndof)])
    sysm = newton.StageSystem(disc, W, a1, a2, dt)
    ref = newton.BJExt(sysm, W)(v)
    outs = []
    for tc in (True, False):
        ctx = make(hb, dim, N, n, tc, dt=dt)
        outs.append(apply(ctx, X, v, a1, a2))
        ctx.close()
    y_tc, y_cc = outs
    assert np.linalg.norm(y_tc - ref) <= 1e-11 * np.linalg.norm(ref)
    # element by element against the CUDA-core FP64 apply: both are FP64
    # accurate, the tensor-core one rounds once per output
    scale = np.abs(y_cc).max()
    assert np.abs(y_tc - y_cc).max() <= 1e-14 * scale, np.abs(y_tc - y_cc).max() / scale
    assert not np.array_equal(y_tc, y_cc)      # the two paths really differ (rounding)


def test_tc_apply_nan_stays_in_its_element(hb):
    dim, N, n, dt = 2, 5, (9, 7), 0.05
    disc = oracle_disc(dim, N, n)
    rng = np.random.default_rng(210)
    W = 0.5 + 0.2 * rng.standard_normal(disc.shape)
    X = np.concatenate([W.ravel(), dgsem.R1(disc, W).ravel()])
    v = rng.standard_normal(2 * disc.ndof)
    ctx = make(hb, dim, N, n, True, dt=dt)
    good = apply(ctx, X, v, 1.0, 1.0)
    nb = (N + 1) ** dim
    e_bad = 37
    vb = v.copy()
    vb[disc.ndof + e_bad * nb + 5] = np.nan     # in sigma of element 37
    bad = apply(ctx, X, vb, 1.0, 1.0)
    ctx.close()
    gw, gs = good[:disc.ndof].reshape(-1, nb), good[disc.ndof:].reshape(-1, nb)
    bw, bs = bad[:disc.ndof].reshape(-1, nb), bad[disc.ndof:].reshape(-1, nb)
    assert np.isnan(bw[e_bad]).all() and np.isnan(bs[e_bad]).all()
    keep = np.arange(gw.shape[0]) != e_bad
    assert np.array_equal(bw[keep], gw[keep]) and np.array_equal(bs[keep], gs[keep])


def test_tc_apply_zero_and_tiny_inputs(hb):
    """A zero vector gives zeros; a vector scaled by 2^-1000 gives the scaled
    result (the slow scaling path, exact for a power of two)."""
    dim, N, n, dt = 2, 3, (6, 6), 0.05
    disc = oracle_disc(dim, N, n)
    rng = np.random.default_rng(211)
    W = 0.5 + 0.2 * rng.standard_normal(disc.shape)
    X = np.concatenate([W.ravel(), dgsem.R1(disc, W).ravel()])
    v = rng.standard_normal(2 * disc.ndof)
    ctx = make(hb, dim, N, n, True, dt=dt)
    assert np.array_equal(apply(ctx, X, 0.0 * v, 1.0, 1.0), np.zeros_like(v))
    y = apply(ctx, X, v, 1.0, 1.0)
    ys = apply(ctx, X, v * 2.0 ** -1000, 1.0, 1.0)
    ctx.close()
    assert np.array_equal(ys * 2.0 ** 1000, y)


def test_tc_apply_steps_vs_oracle_and_cuda_core(hb):
    """Whole HBPC steps with the tensor-core apply in every GMRES iteration:
    the oracle's step (Newton-GMRES to the same tolerances) and the CUDA-core
    run agree to the solver tolerance."""
    dim, N, n, dt, q, kmax = 2, 5, (8, 8), 0.02, 6, 2
    opts = dict(q=q, kmax=kmax, dt=dt, tol_newton_rel=1e-12, tol_newton_abs=1e-13, tol_gmres_rel=1e-10,
                gmres_restart=40)
    disc = oracle_disc(dim, N, n)
    w0 = inputs.sine_product(disc.node_coords())
    res = []
    for tc in (True, False):
        ctx = make(hb, dim, N, n, tc, **opts)
        ctx.set_state(w0)
        ctx.step(2)
        st = ctx.stats()
        assert st["pc_apply_tc"] == (1 if tc else 0)
        res.append((ctx.get_state(), st["gmres_its"]))
        ctx.close()
    o = newton.NewtonOptions(tol_rel=1e-12, tol_abs=1e-13, gmres_tol=1e-10, restart=40, jv="linear", pc="bjext")
    adv = ohbpc.dg_stepper(disc, dt, q, kmax, o)
    ref = adv(adv(w0))
    (w_tc, its_tc), (w_cc, its_cc) = res
    assert np.linalg.norm(w_tc - ref) <= 1e-11 * np.linalg.norm(ref)
    assert np.linalg.norm(w_tc - w_cc) <= 1e-12 * np.linalg.norm(w_cc)
    assert abs(its_tc - its_cc) <= 2
