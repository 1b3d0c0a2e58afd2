"""The learned block preconditioner (BF16 network, GPU training) against the
FP64 oracle network (oracle/mlp.py), and its effect on the solver.

Tolerances: the GPU network multiplies BF16 operands (8-bit mantissa) with FP32
accumulation; a product of two BF16-rounded factors carries a relative error of
~2^-8 per factor, so loss and gradients are compared at 5e-2 relative (norm-wise
per parameter block) -- the error against the FP64 oracle is reported in the
assertion messages.  The preconditioner never changes the converged answer:
with it the Newton root equals the oracle's to 1e-11.
"""
import numpy as np
import pytest
import torch

from oracle import dgsem, laws, mlp, newton
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


def layout(info, p, din, classes=None):
    """oracle params (and optional stage classes [((c1, c2), mean minus I)])
    -> the library's flat FP32 parameter vector."""
    H, dinp, doutp = info["hidden"], info["d_in_padded"], info["d_out_padded"]
    W1 = np.zeros((H, dinp)); W1[:, :din] = p["W1"][:, :din]
    W3 = np.zeros((doutp, H)); W3[:p["W3"].shape[0]] = p["W3"]
    b3 = np.zeros(doutp); b3[:p["b3"].shape[0]] = p["b3"]
    mu, sd = np.zeros(dinp), np.ones(dinp)
    flat = np.concatenate([W1.ravel(), p["b1"], p["W2"].ravel(), p["b2"], W3.ravel(), b3, mu, sd])
    # stage-class keys (c1, c2 per class; c1 <= 0: unused) and class means (minus I)
    keys = np.full(2 * 4, -1.0)
    means = np.zeros((4, doutp))
    for k, (key, cm) in enumerate(classes or []):
        keys[2 * k:2 * k + 2] = key
        means[k, :cm.size] = cm
    flat = np.concatenate([flat, keys, means.ravel()])
    assert flat.size == info["n_params"]
    return flat.astype(np.float32)


def unlayout(info, g, din, dout):
    H, dinp, doutp = info["hidden"], info["d_in_padded"], info["d_out_padded"]
    o = 0
    out = {}
    for name, shape in (("W1", (H, dinp)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
                        ("W3", (doutp, H)), ("b3", (doutp,))):
        n = int(np.prod(shape))
        out[name] = g[o:o + n].reshape(shape).astype(np.float64)
        o += n
    out["W1"] = out["W1"][:, :din]
    out["W3"] = out["W3"][:dout]
    out["b3"] = out["b3"][:dout]
    return out


def test_learned_pc_loss_and_gradients_match_oracle(hb):
    # Euler 2-D, N = 2: n_b = 4 x 9 = 36, network 38(->48) -> 256 -> 256 -> 1296
    ctx = hb.Context(2, (4, 4), (-1, -1), (1, 1), 2, law=hb.LAW_EULER, flux=hb.FLUX_RUSANOV, dt=0.05,
                     pc=hb.PC_LEARNED)
    info = ctx.pc_model_info()
    nb = 36
    din, dout = nb + 2, nb * nb
    rng = np.random.default_rng(7)
    p = mlp.init_params(info["d_in_padded"], info["hidden"], dout, seed=3, out_scale=0.5)
    p["b1"] = 0.1 * rng.standard_normal(info["hidden"])
    p["b2"] = 0.1 * rng.standard_normal(info["hidden"])
    p["b3"] = 0.01 * rng.standard_normal(dout)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):   # values exactly representable in BF16
        p[k] = torch.from_numpy(p[k]).to(torch.bfloat16).to(torch.float64).numpy()
    p["W1"][:, din:] = 0.0
    ctx.pc_model_set(layout(info, p, info["d_in_padded"]))
    B, P = 16, 4
    F = np.zeros((B, info["d_in_padded"]))
    F[:, :din] = rng.standard_normal((B, din))
    F = torch.from_numpy(F).to(torch.bfloat16).to(torch.float64).numpy()
    J = 0.3 * rng.standard_normal((B, nb, nb))
    c12 = np.stack([rng.uniform(0.05, 0.3, B), rng.uniform(0.001, 0.02, B)], axis=1)
    X = np.sign(rng.standard_normal((B, P, nb)))
    S = (np.eye(nb)[None] - c12[:, 0, None, None] * J + c12[:, 1, None, None] * (J @ J))
    U = np.einsum("bij,bpj->bpi", S, X)
    act = mlp.forward(p, F)
    L_ref, dO = mlp.probe_loss(act["O"], U, X, nb)
    g_ref = mlp.backward(p, act, dO)
    L_gpu, g_flat = ctx.pc_loss_grad(F, J.transpose(0, 2, 1), c12, X)
    g_gpu = unlayout(info, g_flat, info["d_in_padded"], dout)
    assert abs(L_gpu - L_ref) <= 5e-2 * abs(L_ref), (L_gpu, L_ref)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        ref = g_ref[k] if k != "W1" else g_ref[k][:, :info["d_in_padded"]]
        err = np.linalg.norm(g_gpu[k] - ref) / np.linalg.norm(ref)
        assert err <= 5e-2, (k, err)
    ctx.close()


def test_learned_pc_inverse_loss_matches_oracle(hb):
    """The inverse-regression loss |M~ - T|_F^2 / B and its gradients against
    the FP64 oracle (same BF16-exact parameters as the probe-loss test)."""
    ctx = hb.Context(2, (4, 4), (-1, -1), (1, 1), 2, law=hb.LAW_EULER, flux=hb.FLUX_RUSANOV, dt=0.05,
                     pc=hb.PC_LEARNED)
    info = ctx.pc_model_info()
    nb = 36
    din, dout = nb + 2, nb * nb
    rng = np.random.default_rng(17)
    p = mlp.init_params(info["d_in_padded"], info["hidden"], dout, seed=4, out_scale=0.5)
    p["b1"] = 0.1 * rng.standard_normal(info["hidden"])
    p["b2"] = 0.1 * rng.standard_normal(info["hidden"])
    p["b3"] = 0.01 * rng.standard_normal(dout)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        p[k] = torch.from_numpy(p[k]).to(torch.bfloat16).to(torch.float64).numpy()
    p["W1"][:, din:] = 0.0
    ctx.pc_model_set(layout(info, p, info["d_in_padded"]))
    B = 16
    F = np.zeros((B, info["d_in_padded"]))
    F[:, :din] = rng.standard_normal((B, din))
    F = torch.from_numpy(F).to(torch.bfloat16).to(torch.float64).numpy()
    T = np.eye(nb)[None] + 0.2 * rng.standard_normal((B, nb, nb))
    c12 = np.zeros((B, 2))
    act = mlp.forward(p, F)
    L_ref, dO = mlp.inverse_loss(act["O"], T, nb)
    g_ref = mlp.backward(p, act, dO)
    L_gpu, g_flat = ctx.pc_loss_grad(F, T.transpose(0, 2, 1), c12, None, loss="inverse")
    g_gpu = unlayout(info, g_flat, info["d_in_padded"], dout)
    assert abs(L_gpu - L_ref) <= 5e-2 * abs(L_ref), (L_gpu, L_ref)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        ref = g_ref[k] if k != "W1" else g_ref[k][:, :info["d_in_padded"]]
        err = np.linalg.norm(g_gpu[k] - ref) / np.linalg.norm(ref)
        assert err <= 5e-2, (k, err)
    ctx.close()


def test_learned_pc_class_means_in_losses(hb):
    """Per-sample stage-class means C_k enter M~ = I + C_k + O in both losses."""
    ctx = hb.Context(2, (4, 4), (-1, -1), (1, 1), 2, law=hb.LAW_EULER, flux=hb.FLUX_RUSANOV, dt=0.05,
                     pc=hb.PC_LEARNED)
    info = ctx.pc_model_info()
    nb = 36
    din, dout = nb + 2, nb * nb
    rng = np.random.default_rng(27)
    p = mlp.init_params(info["d_in_padded"], info["hidden"], dout, seed=5, out_scale=0.5)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        p[k] = torch.from_numpy(p[k]).to(torch.bfloat16).to(torch.float64).numpy()
    p["W1"][:, din:] = 0.0
    keys = [(0.05, 0.002), (0.2, 0.015)]
    cms = [np.float32(0.1 * rng.standard_normal(dout)).astype(np.float64) for _ in keys]
    ctx.pc_model_set(layout(info, p, info["d_in_padded"], list(zip(keys, cms))))
    B, P = 16, 3
    F = np.zeros((B, info["d_in_padded"]))
    F[:, :din] = rng.standard_normal((B, din))
    F = torch.from_numpy(F).to(torch.bfloat16).to(torch.float64).numpy()
    cls = rng.integers(0, 2, B)
    c12 = np.array([keys[c] for c in cls], dtype=np.float32).astype(np.float64)
    C = np.stack([cms[c] for c in cls])
    act = mlp.forward(p, F)
    # inverse loss
    T = np.eye(nb)[None] + 0.2 * rng.standard_normal((B, nb, nb))
    L_ref, _ = mlp.inverse_loss(act["O"], T, nb, C)
    L_gpu, _ = ctx.pc_loss_grad(F, T.transpose(0, 2, 1), c12, None, loss="inverse")
    assert abs(L_gpu - L_ref) <= 5e-2 * abs(L_ref), (L_gpu, L_ref)
    # probe loss
    J = 0.3 * rng.standard_normal((B, nb, nb))
    X = np.sign(rng.standard_normal((B, P, nb)))
    S = np.eye(nb)[None] - c12[:, 0, None, None] * J + c12[:, 1, None, None] * (J @ J)
    U = np.einsum("bij,bpj->bpi", S, X)
    L_ref, dO = mlp.probe_loss(act["O"], U, X, nb, C)
    g_ref = mlp.backward(p, act, dO)
    L_gpu, g_flat = ctx.pc_loss_grad(F, J.transpose(0, 2, 1), c12, X)
    g_gpu = unlayout(info, g_flat, info["d_in_padded"], dout)
    assert abs(L_gpu - L_ref) <= 5e-2 * abs(L_ref), (L_gpu, L_ref)
    err = np.linalg.norm(g_gpu["W3"] - g_ref["W3"]) / np.linalg.norm(g_ref["W3"])
    assert err <= 5e-2, err
    ctx.close()


def euler_stage(hb, pc, precision, dt=0.08, n=(6, 5)):
    ctx = hb.Context(2, n, (-1, -1), (1, 1), 2, law=hb.LAW_EULER, flux=hb.FLUX_RUSANOV, dt=dt,
                     tol_newton_rel=1e-13, tol_newton_abs=1e-13, tol_gmres_rel=1e-6, gmres_restart=200,
                     pc=pc, precision=precision)
    return ctx


def test_learned_pc_training_cuts_gmres_iterations_same_answer(hb):
    """Train on (features, J_e) samples of the method's own Newton iterations
    (BJ_ext run), then solve a fresh stage system with no preconditioner and with
    the learned one: fewer GMRES iterations, the same root as the FP64 oracle."""
    dt = 0.08
    gen = euler_stage(hb, hb.PC_BJEXT, hb.PREC_FP64, dt)
    gen.pc_collect(samples_per_newton=30, capacity=4096)
    w0 = inputs.density_wave(gen.node_coords())
    gen.set_state(w0)
    # q = 6, kmax = 1 is not set here: the default HBPC(4,0) stage solves suffice for data
    gen.step(6)
    gen.pc_model_init(seed=1, out_scale=1e-2)
    l0, l1 = gen.pc_train(iters=400, batch=64, probes=4, lr=2e-3, seed=5)
    assert l1 < 0.5 * l0, (l0, l1)
    params = gen.pc_model_get()
    w_now = gen.get_state()
    gen.close()

    ph = laws.Physics(laws.EULER, 2, flux="rusanov")
    disc = dgsem.Disc(dgsem.Mesh(2, (6, 5), (-1, -1), (1, 1)), 2, ph, LOBATTO)
    b = w_now.copy()
    opts = newton.NewtonOptions(tol_rel=1e-13, tol_abs=1e-13, gmres_tol=1e-9, restart=200, jv="fd")
    Wr, _, _ = newton.newton_solve(disc, b, 1.0, 1.0, dt, w_now, opts)
    its = {}
    for pc in (hb.PC_NONE, hb.PC_LEARNED):
        ctx = euler_stage(hb, pc, hb.PREC_FP64, dt)
        if pc == hb.PC_LEARNED:
            ctx.pc_model_set(params)    # weights and feature standardisation
        Wd = torch.empty(disc.ndof, dtype=torch.float64, device="cuda")
        bt = torch.from_numpy(b.ravel().copy()).cuda()
        ctx.reset_stats()
        ctx.newton_solve(bt, 1.0, 1.0, torch.from_numpy(w_now.ravel().copy()).cuda(), Wd)
        its[pc] = ctx.stats()["gmres_its"]
        err = np.linalg.norm(Wd.cpu().numpy() - Wr.ravel()) / np.linalg.norm(Wr)
        assert err <= 1e-11, (pc, err)
        ctx.close()
    assert its[hb.PC_LEARNED] < its[hb.PC_NONE], its


def test_learned_blocks_failing_their_check_fall_back_to_exact(hb):
    """An untrained network (M~ close to I) fails the probe check on (nearly)
    every element at dt = 0.08, so those blocks get the exact inverse: the solve
    then takes about BJ_ext's iteration count, the counter reports the
    fallbacks, and the root is the same."""
    dt = 0.08
    n = (6, 5)
    ctx = euler_stage(hb, hb.PC_LEARNED, hb.PREC_FP64, dt, n)
    ctx.pc_model_init(seed=3, out_scale=1e-3)
    ref = euler_stage(hb, hb.PC_BJEXT, hb.PREC_FP64, dt, n)
    w0 = inputs.density_wave(ctx.node_coords())
    b = torch.from_numpy(w0.ravel().copy()).cuda()
    its = []
    outs = []
    for c in (ctx, ref):
        Wd = torch.empty_like(b)
        c.reset_stats()
        c.newton_solve(b, 1.0, 1.0, b, Wd)
        its.append(c.stats())
        outs.append(Wd.cpu().numpy())
    st = its[0]
    assert st["pc_exact_blocks"] >= 0.9 * 30 * st["newton_its"]    # (nearly) every element, every build
    assert st["gmres_its"] <= 1.5 * its[1]["gmres_its"] + 2
    assert np.linalg.norm(outs[0] - outs[1]) <= 1e-11 * np.linalg.norm(outs[1])
    ctx.close()
    ref.close()
