"""Element-wise parity of the learned preconditioner's network with the FP64
oracle (oracle/mlp.py): the forward map to the blocks M~ = I + C_k + reshape(O)
and one Adam step.

The GPU network multiplies BF16 operands with FP32 accumulation and keeps the
hidden activations in BF16.  The forward comparison feeds BF16-exact weights
and features and rounds the oracle's hidden activations to BF16 as the GPU
stores them; what remains is FP32 accumulation order and the BF16 rounding of
activations that the accumulation order moves across a rounding boundary, so
each output element is held to two BF16 units (2^-7) of the magnitude of its
own sum, sum_k |W3_ik| |h2_k| + |b3_i|.  Adam runs in FP32: each parameter is
held to 4e-7 of its size plus 1e-4 of the learning rate."""
import numpy as np
import pytest
import torch

from oracle import mlp
from tests.test_gpu_learned_pc import layout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    import __graft_entry__ as g
    g.build()
    from paper_2109_04804_gb300 import hbpc
    assert torch.cuda.is_available()
    return hbpc


def bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(torch.bfloat16).to(torch.float64).numpy()


def model(hb, seed):
    ctx = hb.Context(2, (4, 4), (-1, -1), (1, 1), 2, law=hb.LAW_EULER, flux=hb.FLUX_RUSANOV, dt=0.05,
                     pc=hb.PC_LEARNED)
    info = ctx.pc_model_info()
    nb = 36
    din, dout = nb + 2, nb * nb
    rng = np.random.default_rng(seed)
    p = mlp.init_params(info["d_in_padded"], info["hidden"], dout, seed=seed, out_scale=0.5)
    p["b1"] = 0.1 * rng.standard_normal(info["hidden"])
    p["b2"] = 0.1 * rng.standard_normal(info["hidden"])
    p["b3"] = 0.01 * rng.standard_normal(dout)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        p[k] = bf16(p[k])
    p["W1"][:, din:] = 0.0
    return ctx, info, p, rng, nb, din, dout


@pytest.mark.parametrize("B", [24, 296])
def test_forward_blocks_elementwise(hb, B):
    """B = 296 (a multiple of 8, as the entry point requires) spans three
    128-row tiles of the tensor-core GEMMs with a ragged last one (and
    n_b^2 = 1296 output columns, a ragged last 128-column tile)."""
    ctx, info, p, rng, nb, din, dout = model(hb, 41)
    keys = [(0.05, 0.002), (0.2, 0.015)]
    cms = [np.float32(0.1 * rng.standard_normal(dout)).astype(np.float64) for _ in keys]
    ctx.pc_model_set(layout(info, p, info["d_in_padded"], list(zip(keys, cms))))
    F = np.zeros((B, info["d_in_padded"]))
    F[:, :din] = rng.standard_normal((B, din))
    F = bf16(F)
    cls = rng.integers(0, 2, B)
    c12 = np.array([keys[c] for c in cls], dtype=np.float32).astype(np.float64)
    M_gpu = ctx.pc_model_forward(F, c12).astype(np.float64)
    # oracle forward with the activations stored in BF16 as on the GPU
    h1 = bf16(np.tanh(F @ p["W1"].T + p["b1"]))
    h2 = bf16(np.tanh(h1 @ p["W2"].T + p["b2"]))
    O = h2 @ p["W3"].T + p["b3"]
    C = np.stack([cms[c] for c in cls])
    M_ref = mlp.mtilde(O, nb, C)
    scale = (np.abs(h2) @ np.abs(p["W3"]).T + np.abs(p["b3"])).reshape(B, nb, nb)
    err = np.abs(M_gpu - M_ref)
    assert np.all(err <= 2.0 ** -7 * scale + 1e-6), float((err / (scale + 1e-30)).max())
    # the FP64 oracle without BF16 activations: the distance the reduced precision costs
    Mf = mlp.mtilde(mlp.forward(p, F)["O"], nb, C)
    rel = np.linalg.norm(M_gpu - Mf) / np.linalg.norm(Mf - np.eye(nb)[None])
    assert rel <= 2e-2, rel
    ctx.close()


def test_adam_steps_elementwise(hb):
    ctx, info, p, rng, nb, din, dout = model(hb, 43)
    flat0 = layout(info, p, info["d_in_padded"])
    ctx.pc_model_set(flat0)
    ntrain = info["n_params"] - 2 * info["d_in_padded"] - 2 * 4 - 4 * info["d_out_padded"]
    lr = 1e-3
    grads = [np.float32(rng.standard_normal(ntrain) * 10.0 ** rng.uniform(-3, 1, ntrain)) for _ in range(3)]
    for g in grads:
        ctx.pc_adam_step(g, lr)
    got = ctx.pc_model_get()[:ntrain].astype(np.float64)
    # oracle Adam on the flat parameter vector (one "parameter" holding them all)
    ref = {"p": flat0[:ntrain].astype(np.float64)}
    opt = mlp.Adam(ref, lr=lr)
    for g in grads:
        ref = opt.step(ref, {"p": g.astype(np.float64)})
    err = np.abs(got - ref["p"])
    tol = 4e-7 * np.abs(ref["p"]) + 1e-4 * lr
    assert np.all(err <= tol), float((err / tol).max())
    # the first step of Adam moves every parameter by about lr against its gradient
    ctx.pc_model_set(flat0)
    ctx.pc_model_init(seed=0)       # clears the Adam state
    ctx.pc_model_set(flat0)
    ctx.pc_adam_step(grads[0], lr)
    step = ctx.pc_model_get()[:ntrain].astype(np.float64) - flat0[:ntrain]
    big = np.abs(grads[0]) > 1e-4
    assert np.allclose(step[big], -lr * np.sign(grads[0][big]), rtol=1e-3, atol=2e-7)
    ctx.close()
