"""The launch-shape autotuner: it picks shapes among its candidates and leaves
the answer unchanged (only the summation order of reductions may change)."""
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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_autotune_keeps_the_answer(hb, prec):
    kw = dict(law=hb.LAW_EULER, flux=hb.FLUX_RUSANOV, q=6, kmax=1, dt=0.04, tol_newton_rel=1e-13,
              tol_newton_abs=1e-13, tol_gmres_rel=1e-8 if prec == "fp64" else 1e-5, gmres_restart=60,
              pc=hb.PC_BJEXT, precision=hb.PREC_MIXED if prec == "mixed" else hb.PREC_FP64)
    out = []
    for tune in (False, True):
        c = hb.Context(2, (12, 10), (-1, -1), (1, 1), 3, **kw)
        w0 = inputs.density_wave(c.node_coords())
        c.set_state(w0)
        if tune:
            t = c.autotune()
            sms = torch.cuda.get_device_properties(0).multi_processor_count
            assert 1 <= t["krylov_blocks"] <= max(4 * sms, 4096)
            assert 1 <= t["pc_elems_per_block"] <= 16
            assert t["krylov_us"] > 0 and t["pc_us"] > 0
            assert t["krylov_us"] <= t["krylov_us_default"] * 1.0001 or t["krylov_us_default"] == 0
        c.step(2)
        out.append(c.get_state())
        c.close()
    assert np.linalg.norm(out[1] - out[0]) <= 1e-11 * np.linalg.norm(out[0])


def test_batch_autotune_per_group(hb):
    b = hb.Batch(2, [((6, 5), (0, 0), (1, 1)), ((4, 4), (0, 0), (1, 1)), ((5, 3), (0, 0), (1, 1))], [3, 4, 3],
                 nus=[0.01, 0.0, 0.005], law=hb.LAW_BURGERS, q=4, kmax=1, dt=0.01, tol_newton_rel=1e-12,
                 tol_newton_abs=1e-13,
                 tol_gmres_rel=1e-8, gmres_restart=40, pc=hb.PC_BJEXT)
    t = b.autotune()
    assert len(t) == b.groups() == 2
    for i in range(3):
        b.set_state(i, 0.5 + 0.2 * inputs.burgers_fourier(b.node_coords(i), seed=i, n_modes=3, kmax=2))
    b.step(1)
    assert b.stats()["steps"] == 1
    b.close()
