"""The allocation-free Jacobian-vector product (hbpc_eval_Jv_noalloc) against
the context-based one (hbpc_eval_Jv).

The allocation-free entry point is for callers that cannot call cudaMalloc,
for instance code whose device memory is owned by a framework's pool or a fixed
budget; it keeps its scratch in a file-scope device array shared by all calls.
This file is collected last so that a failure here comes after every other
test has run; it also passes when run alone in a fresh process.  Tolerances are
those of the Jv parity tests: 1e-13 for the linear form (Eq. 24), 1e-6 for the
difference quotients (Eq. 23); both paths use the same kernels and reduction
order, so in practice the results agree to the last bit.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    import __graft_entry__ as g
    g.build()
    from paper_2109_04804_gb300 import hbpc
    assert torch.cuda.is_available()
    return hbpc


CASES = [
    # (law, flux, dim, n, N, tolerance)
    (0, 0, 2, (7, 5), 5, 1e-13),
    (2, 1, 2, (6, 5), 3, 1e-6),
    (2, 0, 3, (3, 3, 2), 3, 1e-6),
]


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("law,flux,dim,n,N,tol", CASES)
def test_noalloc_jv_matches_context_jv_twice(hb, law, flux, dim, n, N, tol):
    from paper_2109_04804_gb300 import inputs
    lo, hi = (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0)
    dt, a1, a2 = 0.03, 0.5, 1.0 / 6.0
    ctx = hb.Context(dim, n, lo, hi, N, law=law, flux=flux, a=(1.0, -0.6, 0.35), eps=0.8, dt=dt)
    coords = ctx.node_coords()
    rng = np.random.default_rng(2024 + law)
    if law == 2:
        W = inputs.density_wave(coords) * (1.0 + 0.02 * rng.standard_normal(ctx.shape))
    else:
        W = inputs.sine_product(coords, k=1.0)
    for call in range(2):   # two calls in a row, different inputs
        S = 0.1 * rng.standard_normal(ctx.shape)
        X = torch.from_numpy(np.concatenate([W.ravel(), S.ravel()])).cuda()
        dX = torch.from_numpy(rng.standard_normal(2 * ctx.ndof)).cuda()
        ref = torch.empty_like(X)
        ctx.eval_Jv(a1, a2, X, dX, ref)
        out = torch.full_like(X, float("nan"))
        hb.eval_Jv_noalloc(dim, n, lo, hi, N, dt, a1, a2, X, dX, out, law=law, flux=flux,
                           a=(1.0, -0.6, 0.35), eps=0.8)
        assert torch.isfinite(out).all()
        assert rel(out, ref) <= tol, (call, rel(out, ref))
        W = W * (1.0 + 0.01 * call)
    ctx.close()


def test_noalloc_rejects_oversized_problem(hb):
    X = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(hb.HBPCError) as ei:
        # 128 x 128 elements, N = 5: n_dof = 589824 > 262144
        hb.eval_Jv_noalloc(2, (128, 128), (0, 0), (1, 1), 5, 0.01, 1.0, 1.0, X, X, X)
    assert ei.value.status == hb.ERR_INVALID_ARG
    assert "262144" in str(ei.value)


def test_noalloc_jv_on_a_side_stream(hb):
    """Work enqueued on a caller's (non-default) stream: the same product as
    the context-based entry point, twice in a row."""
    dim, n, N, lo, hi = 2, (5, 6), 4, (0.0, 0.0), (1.0, 1.0)
    dt, a1, a2 = 0.02, 1.0, 1.0
    ctx = hb.Context(dim, n, lo, hi, N, law=hb.LAW_EULER, flux=hb.FLUX_RUSANOV, eps=0.8, dt=dt)
    from paper_2109_04804_gb300 import inputs
    rng = np.random.default_rng(77)
    W = inputs.density_wave(ctx.node_coords()) * (1.0 + 0.02 * rng.standard_normal(ctx.shape))
    side = torch.cuda.Stream()
    for call in range(2):
        S = 0.1 * rng.standard_normal(ctx.shape)
        X = torch.from_numpy(np.concatenate([W.ravel(), S.ravel()])).cuda()
        dX = torch.from_numpy(rng.standard_normal(2 * ctx.ndof)).cuda()
        ref = torch.empty_like(X)
        ctx.eval_Jv(a1, a2, X, dX, ref)
        out = torch.full_like(X, float("nan"))
        torch.cuda.synchronize()
        hb.eval_Jv_noalloc(dim, n, lo, hi, N, dt, a1, a2, X, dX, out, law=hb.LAW_EULER,
                           flux=hb.FLUX_RUSANOV, eps=0.8, stream=side.cuda_stream)
        assert rel(out, ref) <= 1e-6, (call, rel(out, ref))
    ctx.close()


def test_noalloc_rejects_aliased_output_and_viscous_law(hb):
    """out == dX or out == X is rejected (the kernels read both while writing
    out) and leaves the inputs untouched; a viscous law is unsupported."""
    n, N = (4, 4), 3
    ndof = 16 * 16
    X = torch.randn(2 * ndof, dtype=torch.float64, device="cuda")
    dX = torch.randn(2 * ndof, dtype=torch.float64, device="cuda")
    X0, dX0 = X.clone(), dX.clone()
    for out in (dX, X, X[1:]):
        with pytest.raises(hb.HBPCError) as ei:
            hb.eval_Jv_noalloc(2, n, (0, 0), (1, 1), N, 0.01, 0.5, 0.1, X, dX, out)
        assert ei.value.status == hb.ERR_INVALID_ARG
    assert torch.equal(X, X0) and torch.equal(dX, dX0)
    out = torch.empty_like(X)
    with pytest.raises(hb.HBPCError) as ei:
        hb.eval_Jv_noalloc(2, n, (0, 0), (1, 1), N, 0.01, 0.5, 0.1, X, dX, out, nu=0.01)
    assert ei.value.status == hb.ERR_UNSUPPORTED
