"""The device-driven step (hbpc_set_step_graph): one CUDA graph launch per HBPC
step with the Newton and GMRES loops as conditional graph nodes.  It launches
the kernels of the host-driven step in the same order with the same
arguments, so the states agree to the last bit and the iteration counters are
equal; failures end the step with the host-driven status and leave the state
at the previous step."""
import numpy as np
import pytest
import torch

from paper_2109_04804_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    import __graft_entry__ as g
    g.build()
    from paper_2109_04804_gb300 import hbpc
    assert torch.cuda.is_available()
    return hbpc


COUNTERS = ("newton_solves", "newton_its", "gmres_its", "arnoldi_cols", "r1_evals", "r2_evals", "steps")


def run(hb, graph, make, init, steps=2):
    c = make()
    if graph:
        c.set_step_graph(True)
    c.set_state(init(c))
    c.step(steps)
    w = c.get_state()
    st = c.stats()
    c.close()
    return w, st


CASES = {
    "advection_fp64_bjext": lambda hb: (
        lambda: hb.Context(2, (8, 6), (0, 0), (1, 1), 4, law=hb.LAW_ADVECTION, a=(1.0, 0.5), q=6, kmax=2,
                           dt=0.02, tol_newton_rel=1e-12, tol_newton_abs=1e-12, tol_gmres_rel=1e-8,
                           gmres_restart=30, pc=hb.PC_BJEXT),
        lambda c: inputs.sine_product(c.node_coords())),
    "euler_fp64_bjext": lambda hb: (
        lambda: hb.Context(2, (6, 5), (-1, -1), (1, 1), 3, law=hb.LAW_EULER, flux=hb.FLUX_RUSANOV, q=4, kmax=1,
                           dt=0.04, tol_newton_rel=1e-12, tol_newton_abs=1e-13, tol_gmres_rel=1e-8,
                           gmres_restart=12, pc=hb.PC_BJEXT),
        lambda c: inputs.density_wave(c.node_coords())),
    "euler_fp64_plain": lambda hb: (
        lambda: hb.Context(2, (4, 4), (-1, -1), (1, 1), 3, law=hb.LAW_EULER, flux=hb.FLUX_GLOBAL_LF, q=4, kmax=1,
                           dt=0.02, tol_newton_rel=1e-12, tol_newton_abs=1e-13, tol_gmres_rel=1e-8,
                           gmres_restart=20, pc=hb.PC_NONE),
        lambda c: inputs.density_wave(c.node_coords())),
    "euler_mixed_bjext_h": lambda hb: (
        lambda: hb.Context(2, (6, 5), (-1, -1), (1, 1), 3, law=hb.LAW_EULER, flux=hb.FLUX_RUSANOV, q=6, kmax=2,
                           dt=0.04, tol_newton_rel=1e-10, tol_newton_abs=1e-12, tol_gmres_rel=1e-5,
                           gmres_restart=10, pc=hb.PC_BJEXT_H, precision=hb.PREC_MIXED),
        lambda c: inputs.density_wave(c.node_coords())),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_step_graph_equals_host_driven_step(hb, case):
    make, init = CASES[case](hb)
    w0, s0 = run(hb, False, make, init)
    w1, s1 = run(hb, True, make, init)
    assert np.array_equal(w0, w1), np.abs(w0 - w1).max()
    for k in COUNTERS:
        assert s0[k] == s1[k], (k, s0[k], s1[k])
    assert s1["gmres_its"] > 0


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_step_graph_equals_host_driven(hb, prec):
    """Batch groups (per-instance FP32 GMRES in the mixed mode, the shared
    row-scaled GMRES in FP64): every instance's state and the summed counters."""
    meshes = [((6, 5), (0, 0), (1, 1)), ((4, 4), (0, 0), (1, 1)), ((5, 3), (0, 0), (1, 1))]

    def batch(graph):
        b = hb.Batch(2, meshes, [3, 4, 3], nus=[0.01, 0.0, 0.005], law=hb.LAW_BURGERS, q=4, kmax=1, dt=0.01,
                     tol_newton_rel=1e-10, tol_newton_abs=1e-13, tol_gmres_rel=1e-6 if prec == "mixed" else 1e-9,
                     gmres_restart=20, pc=hb.PC_BJEXT,
                     precision=hb.PREC_MIXED if prec == "mixed" else hb.PREC_FP64)
        if graph:
            b.set_step_graph(True)
        for i in range(3):
            b.set_state(i, 0.5 + 0.2 * inputs.burgers_fourier(b.node_coords(i), seed=i, n_modes=3, kmax=2))
        b.step(2)
        out = [b.get_state(i) for i in range(3)]
        st = b.stats()
        b.close()
        return out, st

    w0, s0 = batch(False)
    w1, s1 = batch(True)
    for a, c in zip(w0, w1):
        assert np.array_equal(a, c), np.abs(a - c).max()
    for k in ("newton_solves", "newton_its", "gmres_its", "arnoldi_cols"):
        assert s0[k] == s1[k], (k, s0[k], s1[k])


def test_step_graph_failures_keep_the_state(hb):
    """A NaN in the state: HBPC_ERR_NONFINITE; a Newton cap of one iteration:
    HBPC_ERR_NO_CONVERGENCE; both leave the state of the previous step, and a
    later step with a valid state succeeds."""
    make, init = CASES["euler_fp64_bjext"](hb)
    c = make()
    c.set_step_graph(True)
    w = init(c)
    c.set_state(w)
    c.step(1)
    good = c.get_state()
    bad = good.copy()
    bad.flat[7] = np.nan
    c.set_state(bad)
    with pytest.raises(hb.HBPCError) as ei:
        c.step(1)
    assert ei.value.status == hb.ERR_NONFINITE
    assert np.array_equal(c.get_state(), bad, equal_nan=True)
    c.set_state(good)
    c.step(1)
    assert np.isfinite(c.get_state()).all()
    c.close()
    c = hb.Context(2, (6, 5), (-1, -1), (1, 1), 3, law=hb.LAW_EULER, flux=hb.FLUX_RUSANOV, q=4, kmax=1, dt=0.04,
                   tol_newton_rel=1e-14, tol_newton_abs=0.0, tol_gmres_rel=1e-3, gmres_restart=12,
                   newton_max_iter=1, pc=hb.PC_BJEXT)
    c.set_step_graph(True)
    c.set_state(w)
    with pytest.raises(hb.HBPCError) as ei:
        c.step(1)
    assert ei.value.status == hb.ERR_NO_CONVERGENCE
    assert np.array_equal(c.get_state(), w)
    c.close()


def test_step_graph_recaptures_when_the_configuration_changes(hb):
    """advance_to's shorter last step and a new boundary: the graph follows
    (the same states as the host-driven runs)."""
    def go(graph):
        c = hb.Context(1, (10,), (-1.0,), (1.0,), 3, law=hb.LAW_EULER, flux=hb.FLUX_RUSANOV, q=4, kmax=1, dt=0.03,
                       tol_newton_rel=1e-12, tol_newton_abs=1e-13, tol_gmres_rel=1e-9, gmres_restart=30,
                       pc=hb.PC_BJEXT)
        if graph:
            c.set_step_graph(True)
        c.set_state(inputs.density_wave(c.node_coords()))
        c.advance_to(0.1)               # 3 steps and a 0.01 remainder
        st = inputs.euler_from_primitive(np.array([1.0]), [np.array([0.3])], np.array([1.0]))[0]
        c.set_boundary(0, st, "wall")
        c.step(2)
        w = c.get_state()
        s = c.stats()
        c.close()
        return w, s
    w0, s0 = go(False)
    w1, s1 = go(True)
    assert np.array_equal(w0, w1)
    assert s0["gmres_its"] == s1["gmres_its"] and s0["steps"] == s1["steps"]


def test_step_graph_argument_checks(hb):
    c = hb.Context(2, (4, 4), (0, 0), (1, 1), 3, law=hb.LAW_EULER, pc=hb.PC_BJEXT)
    with pytest.raises(hb.HBPCError) as ei:
        c._c(hb._lib.hbpc_set_step_graph(c._ctx, 2))
    assert ei.value.status == hb.ERR_INVALID_ARG
    c.set_schur(True)
    with pytest.raises(hb.HBPCError) as ei:
        c.set_step_graph(True)
    assert ei.value.status == hb.ERR_UNSUPPORTED
    c.close()


@pytest.mark.parametrize("graph", [False, True])
def test_preconditioner_built_once_per_solve(hb, graph):
    """hbpc_set_pc_rebuild(0): the blocks are built at every Newton solve's first
    iterate only; the answer is that of the rebuild-every-iteration run to the
    Newton tolerance, and the graph form equals the host-driven one."""
    make, init = CASES["euler_fp64_bjext"](hb)

    def go(every, g):
        c = make()
        c.set_pc_rebuild(every)
        if g:
            c.set_step_graph(True)
        c.set_state(init(c))
        c.step(2)
        w = c.get_state()
        s = c.stats()
        c.close()
        return w, s
    w_every, _ = go(True, False)
    w_once, s_once = go(False, graph)
    assert np.linalg.norm(w_once - w_every) <= 1e-10 * np.linalg.norm(w_every)
    if graph:
        w_host, s_host = go(False, False)
        assert np.array_equal(w_once, w_host)
        assert s_once["gmres_its"] == s_host["gmres_its"]
