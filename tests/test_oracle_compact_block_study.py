"""Why the compact (Kronecker / low-rank) learned block is not built for the
3-D Navier-Stokes Taylor-Green workload: with the oracle, on the stage system
of that workload (eps = 0.1, Re 1600, CFL 20, here on 2^3 elements of N = 3,
n_b = 320), the SVD-optimal approximation of every exact BJ_ext inverse block
M_e = S_e^-1 (Sec. 3.2.3) by r Kronecker products (5 x 5 variables) x
(64 x 64 nodes) leaves ||M~_e S_e - I||_2 above 1 up to r = 16 of 25, and such
a block then preconditions worse than none at all, while the exact blocks cut
the GMRES iterations."""
import numpy as np
import pytest

from oracle import dgsem, laws, newton
from paper_2109_04804_gb300 import inputs


@pytest.fixture(scope="module")
def study():
    n, N, cfl, eps = 2, 3, 20.0, 0.1
    L = 2.0 * np.pi
    ph = laws.Physics(laws.NAVIER_STOKES, 3, flux="rusanov", mu=1.0 / 1600.0, eps=eps, prandtl=0.72)
    disc = dgsem.Disc(dgsem.Mesh(3, (n, n, n), (0, 0, 0), (L, L, L)), N, ph, "lobatto")
    dt = cfl / (3 * (1.0 + 1.0 / eps) * (N + 1) / (L / n))
    W = inputs.taylor_green(disc.node_coords(), eps=eps)
    sysm = newton.StageSystem(disc, W, 0.5, 1.0 / 6.0, dt)
    X = np.concatenate([W.ravel(), dgsem.R1(disc, W).ravel()])
    G, r1, r2 = sysm.residual(X)
    bj = newton.BJExt(sysm, W)
    S = np.linalg.inv(bj.M)
    return dict(sysm=sysm, X=X, G=G, r1=r1, r2=r2, bj=bj, S=S)


def kron_approx(M, r, nv=5):
    nn = M.shape[0] // nv
    R = M.reshape(nv, nn, nv, nn).transpose(0, 2, 1, 3).reshape(nv * nv, nn * nn)
    U, s, Vt = np.linalg.svd(R, full_matrices=False)
    out = np.zeros_like(M)
    for k in range(r):
        out += np.kron((U[:, k] * s[k]).reshape(nv, nv), Vt[k].reshape(nn, nn))
    return out


def with_blocks(bj, Mt):
    I = np.eye(bj.nb)[None]
    A, B, C = I - bj.c1 * bj.J, bj.c2 * bj.J, -bj.J
    D, E, F, Gb = Mt, -B @ Mt, -C @ Mt, A @ Mt

    def pc(x):
        w = x[:bj.n].reshape(bj.nE, bj.nb, 1)
        s = x[bj.n:].reshape(bj.nE, bj.nb, 1)
        return np.concatenate([(D @ w + E @ s).ravel(), (F @ w + Gb @ s).ravel()])
    return pc


def test_kronecker_blocks_stay_far_from_the_inverse(study):
    bj, S = study["bj"], study["S"]
    I = np.eye(bj.nb)
    for r in (1, 8, 16):
        assert np.linalg.norm(kron_approx(bj.M[0], r) @ S[0] - I, 2) > 1.0, r
    # the full rank reproduces the block: the rearrangement is exact
    assert np.linalg.norm(kron_approx(bj.M[0], 25) @ S[0] - I, 2) < 1e-8


def test_exact_blocks_help_and_a_rank_one_block_hurts(study):
    sysm, X, G, r1, r2, bj = (study[k] for k in ("sysm", "X", "G", "r1", "r2", "bj"))
    mv = lambda v: sysm.jv(X, r1, r2, v, "fd")
    _, its_none, ok_none = newton.gmres(mv, -G, 1e-3, 100, 400, None)
    _, its_bj, ok_bj = newton.gmres(mv, -G, 1e-3, 100, 400, bj)
    assert ok_none and ok_bj and its_bj < 0.5 * its_none
    Mt = np.stack([kron_approx(bj.M[e], 1) for e in range(bj.nE)])
    _, its_k, ok_k = newton.gmres(mv, -G, 1e-3, 100, 4 * its_none, with_blocks(bj, Mt))
    assert not ok_k or its_k > 4 * its_none
