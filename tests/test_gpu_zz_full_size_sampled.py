"""Full-size configurations of the bench, on sampled elements against the
oracle: the Euler isentropic vortex of the learned-preconditioner line
(128^2 elements, N = 4, Rusanov, 1.64 M values; R1 of Eq. 12 and R2 of
Eq. 16) and the 256 viscous Burgers instances of the batch line (meshes 16^2
to 96^2, N = 3 to 7, BR2; 35 M values; R1 per instance).  An element's
operators depend only on it and its four face neighbours (the BR2 lifting is
face-local), so the oracle evaluates a periodic 3 x 3 patch of elements
centred on the sample and its centre element is compared."""
import os
import sys

import numpy as np
import pytest
import torch

from oracle import dgsem, laws
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


def test_vortex_full_size_sampled_parity(hb):
    n, N, lo, hi = 128, 4, -10.0, 10.0
    ctx = hb.Context(2, (n, n), (lo, lo), (hi, hi), N, law=hb.LAW_EULER, flux=hb.FLUX_RUSANOV, q=6, kmax=2,
                     dt=0.01, gmres_restart=2)
    w = inputs.isentropic_vortex(ctx.node_coords())
    rng = np.random.default_rng(71)
    w = w * (1.0 + 1e-3 * rng.standard_normal(w.shape))   # no element is a free stream (R1 = 0)
    s = rng.standard_normal(w.shape)
    wd = torch.from_numpy(np.ascontiguousarray(w)).cuda()
    sd = torch.from_numpy(np.ascontiguousarray(s)).cuda()
    out = torch.empty_like(wd)
    ctx.eval_R1(wd, out)
    r1 = out.cpu().numpy()
    ctx.eval_R2(wd, sd, out)
    r2 = out.cpu().numpy()
    ctx.close()
    del wd, sd, out
    h = (hi - lo) / n
    ph = laws.Physics(laws.EULER, 2, flux="rusanov")
    patch = dgsem.Disc(dgsem.Mesh(2, (3, 3), (0.0, 0.0), (3 * h, 3 * h)), N, ph, LOBATTO)
    centre = (n // 2) + n * (n // 2)                        # the vortex core, x = y = 0
    samples = [centre, centre - 1, centre + n] + [int(e) for e in rng.integers(0, n * n, size=6)]
    for e in samples:
        ex, ey = e % n, e // n
        idx = [((ex + a) % n) + n * ((ey + b) % n) for b in (-1, 0, 1) for a in (-1, 0, 1)]
        ref1 = dgsem.R1(patch, w[idx])[4]
        ref2 = dgsem.R2(patch, w[idx], s[idx])[4]
        assert np.abs(r1[e] - ref1).max() <= 1e-12 * np.abs(ref1).max(), e
        assert np.abs(r2[e] - ref2).max() <= 1e-12 * np.abs(ref2).max(), e


def test_burgers_batch_full_size_sampled_parity(hb):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import bench
    inst = bench.batch_instances(bench.BATCH["n_inst"])
    b = hb.Batch(2, [(n, (0.0, 0.0), (1.0, 1.0)) for n, _, _, _ in inst], [N for _, N, _, _ in inst],
                 nus=[nu for _, _, nu, _ in inst], law=hb.LAW_BURGERS, flux=hb.FLUX_GLOBAL_LF, q=6, kmax=2,
                 dt=1e-3, gmres_restart=2, pc=hb.PC_NONE, precision=hb.PREC_MIXED)
    states = []
    for i, (n, N, nu, seed) in enumerate(inst):
        w = inputs.burgers_fourier(b.node_coords(i), seed=seed)
        b.set_state(i, w)
        states.append(w)
    rng = np.random.default_rng(73)
    largest = max(range(len(inst)), key=lambda i: inst[i][0][0] ** 2 * (inst[i][1] + 1) ** 2)
    picks = [largest] + [int(i) for i in rng.choice(len(inst), size=5, replace=False)]
    for i in picks:
        (n, _), N, nu, _ = inst[i]
        r1 = b.eval_R1(i)
        w = states[i]
        h = 1.0 / n
        ph = laws.Physics(laws.BURGERS, 2, flux="lf", nu=nu)
        patch = dgsem.Disc(dgsem.Mesh(2, (3, 3), (0.0, 0.0), (3 * h, 3 * h)), N, ph, LOBATTO)
        for e in [0, n * n - 1] + [int(v) for v in rng.integers(0, n * n, size=3)]:
            ex, ey = e % n, e // n
            idx = [((ex + a) % n) + n * ((ey + c) % n) for c in (-1, 0, 1) for a in (-1, 0, 1)]
            ref = dgsem.R1(patch, w[idx])[4]
            assert np.abs(r1[e] - ref).max() <= 1e-12 * np.abs(ref).max(), (i, e)
    b.close()
