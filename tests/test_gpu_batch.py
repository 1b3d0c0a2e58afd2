"""Batches of independent instances (own mesh, N and viscosity each) against
the FP64 oracle and against the same instances run one by one.

Tolerances: the batched operator sums the same terms as the oracle in another
order (1e-12 of the largest term); batched Newton stops every instance on the
same 1e-13 tests as a single run, so states agree to 1e-11 relative L2."""
import numpy as np
import pytest
import torch

from oracle import dgsem, hbpc as ohbpc, laws, newton
from oracle.basis import LOBATTO
from paper_2109_04804_gb300 import inputs

pytestmark = pytest.mark.gpu

# (n, lo, hi), N, nu: several groups, ragged element counts (padding inside a
# group), different element sizes and viscosities (0 included)
INST = [
    (((5, 4), (0.0, 0.0), (1.0, 1.0)), 3, 0.01),
    (((3, 3), (-1.0, 0.0), (1.0, 2.0)), 3, 0.004),
    (((6, 5), (0.0, 0.0), (1.0, 1.0)), 4, 0.0),
    (((4, 7), (0.0, 0.0), (2.0, 1.0)), 2, 0.02),
    (((2, 2), (0.0, 0.0), (1.0, 1.0)), 4, 0.008),
    (((7, 3), (0.0, -0.5), (1.0, 0.5)), 5, 0.003),
]


@pytest.fixture(scope="module")
def hb():
    import __graft_entry__ as g
    g.build()
    from paper_2109_04804_gb300 import hbpc
    assert torch.cuda.is_available()
    return hbpc


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def oracle_disc(mesh, N, nu, flux="lf"):
    n, lo, hi = mesh
    ph = laws.Physics(laws.BURGERS, 2, flux=flux, nu=nu)
    return dgsem.Disc(dgsem.Mesh(2, n, lo, hi), N, ph, LOBATTO)


def make_batch(hb, **solver):
    return hb.Batch(2, [m for m, _, _ in INST], [N for _, N, _ in INST], nus=[nu for _, _, nu in INST],
                    law=hb.LAW_BURGERS, **solver)


def initial(coords, seed):
    return 0.5 + 0.3 * inputs.burgers_fourier(coords, seed=seed, n_modes=4, kmax=2)


def test_batch_groups_and_r1_per_instance(hb):
    b = make_batch(hb)
    assert b.groups() == 4
    rng = np.random.default_rng(9)
    states = []
    for i in range(len(INST)):
        w = rng.standard_normal(b.shape(i))
        b.set_state(i, w)
        states.append(w)
    for i, (mesh, N, nu) in enumerate(INST):
        disc = oracle_disc(mesh, N, nu)
        for m in range(2):
            np.testing.assert_allclose(b.node_coords(i)[m], disc.node_coords()[m], atol=1e-14)
        ref = dgsem.R1(disc, states[i])
        got = b.eval_R1(i)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), i
        np.testing.assert_array_equal(b.get_state(i), states[i])
    b.close()


@pytest.mark.parametrize("pc,prec", [("none", "fp64"), ("bjext", "fp64"), ("bjext", "mixed")])
def test_batch_steps_match_single_runs(hb, pc, prec):
    """Two HBPC(4,1) steps of the batch equal the same instances stepped one by
    one in single-problem contexts."""
    kw = dict(q=4, kmax=1, dt=0.01, tol_newton_rel=1e-13, tol_newton_abs=1e-13,
              tol_gmres_rel=1e-9 if prec == "fp64" else 1e-5, gmres_restart=60,
              pc=hb.PC_BJEXT if pc == "bjext" else hb.PC_NONE,
              precision=hb.PREC_MIXED if prec == "mixed" else hb.PREC_FP64)
    b = make_batch(hb, **kw)
    w0 = []
    for i in range(len(INST)):
        w = initial(b.node_coords(i), seed=20 + i)
        b.set_state(i, w)
        w0.append(w)
    b.step(2)
    st = b.stats()
    assert st["steps"] == 2 and st["newton_solves"] == 4 * 2 * 2   # 4 groups x 2 stages x 2 steps
    for i, ((n, lo, hi), N, nu) in enumerate(INST):
        c = hb.Context(2, n, lo, hi, N, law=hb.LAW_BURGERS, nu=nu, **kw)
        c.set_state(w0[i])
        c.step(2)
        ref = c.get_state()
        c.close()
        assert rel(b.get_state(i), ref) <= 1e-11, i
    b.close()


def test_batch_instance_matches_oracle(hb):
    """One instance of a batch stepped by HBPC(6,1) against the oracle."""
    dt = 0.02
    b = make_batch(hb, q=6, kmax=1, dt=dt, tol_newton_rel=1e-13, tol_newton_abs=1e-13, tol_gmres_rel=1e-9,
                   gmres_restart=80, pc=hb.PC_BJEXT)
    for i in range(len(INST)):
        b.set_state(i, initial(b.node_coords(i), seed=40 + i))
    b.step(1)
    k = 0
    mesh, N, nu = INST[k]
    disc = oracle_disc(mesh, N, nu)
    opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-13, gmres_tol=1e-9, restart=80, jv="fd")
    ref = ohbpc.dg_stepper(disc, dt, 6, 1, opts)(initial(disc.node_coords(), seed=40 + k))
    assert rel(b.get_state(k), ref) <= 1e-11
    b.close()


def test_batch_grouping_does_not_change_the_answer(hb):
    """The same instances in one group per N, in groups of at most two, and one
    per group (mixed precision: per-instance GMRES inside every group) reach the
    same states: every instance stops on its own Newton tests."""
    kw = dict(q=4, kmax=1, dt=0.01, tol_newton_rel=1e-13, tol_newton_abs=1e-13, tol_gmres_rel=1e-5,
              gmres_restart=60, pc=hb.PC_BJEXT, precision=hb.PREC_MIXED)
    out = []
    for mpg in (0, 2, 1):
        b = make_batch(hb, max_per_group=mpg, **kw)
        assert b.groups() == {0: 4, 2: 4, 1: 6}[mpg]
        for i in range(len(INST)):
            b.set_state(i, initial(b.node_coords(i), seed=60 + i))
        b.step(2)
        out.append([b.get_state(i) for i in range(len(INST))])
        b.close()
    for k in (1, 2):
        for i in range(len(INST)):
            assert rel(out[k][i], out[0][i]) <= 1e-11, (k, i)
