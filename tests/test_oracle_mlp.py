"""Pins of the oracle's learned-preconditioner network (oracle/mlp.py):
backward against central finite differences, the probe-loss gradient, and
Adam's first step (closed form: lr * sign(g))."""
import numpy as np
import pytest

from oracle import mlp


def small(seed=0, d_in=7, d_h=9, nb=3):
    p = mlp.init_params(d_in, d_h, nb * nb, seed=seed, out_scale=0.3)
    rng = np.random.default_rng(seed + 1)
    B, P = 5, 4
    F = rng.standard_normal((B, d_in))
    S = np.eye(nb)[None] + 0.3 * rng.standard_normal((B, nb, nb))
    X = rng.standard_normal((B, P, nb))
    U = np.einsum("bij,bpj->bpi", S, X)
    return p, F, U, X, nb


def loss_of(p, F, U, X, nb):
    act = mlp.forward(p, F)
    L, _ = mlp.probe_loss(act["O"], U, X, nb)
    return L


@pytest.mark.parametrize("name", ["W1", "b1", "W2", "b2", "W3", "b3"])
def test_backward_matches_central_differences(name):
    p, F, U, X, nb = small()
    act = mlp.forward(p, F)
    L, dO = mlp.probe_loss(act["O"], U, X, nb)
    g = mlp.backward(p, act, dO)
    rng = np.random.default_rng(3)
    h = 1e-6
    for _ in range(6):
        idx = tuple(rng.integers(0, s) for s in p[name].shape)
        pp = {k: v.copy() for k, v in p.items()}
        pm = {k: v.copy() for k, v in p.items()}
        pp[name][idx] += h
        pm[name][idx] -= h
        fd = (loss_of(pp, F, U, X, nb) - loss_of(pm, F, U, X, nb)) / (2 * h)
        assert abs(fd - g[name][idx]) <= 1e-7 * max(1.0, abs(fd))


def test_probe_loss_is_zero_for_exact_inverse():
    p, F, U, X, nb = small()
    S = np.einsum("bpi,bpj->bij", U, X)    # not used; build exact M = S^-1 below
    rng = np.random.default_rng(4)
    Sm = np.eye(nb)[None] + 0.2 * rng.standard_normal((3, nb, nb))
    Xp = rng.standard_normal((3, 5, nb))
    Up = np.einsum("bij,bpj->bpi", Sm, Xp)
    O = (np.linalg.inv(Sm) - np.eye(nb)[None]).reshape(3, nb * nb)
    L, dO = mlp.probe_loss(O, Up, Xp, nb)
    assert L < 1e-25 and np.abs(dO).max() < 1e-12


def test_adam_first_step_is_lr_sign():
    p = {"x": np.array([1.0, -2.0, 3.0])}
    g = {"x": np.array([0.5, -4.0, 1e-3])}
    opt = mlp.Adam(p, lr=0.01)
    q = opt.step({k: v.copy() for k, v in p.items()}, g)
    np.testing.assert_allclose(q["x"], p["x"] - 0.01 * np.sign(g["x"]), atol=1e-9)


def test_training_reduces_probe_loss():
    p, F, U, X, nb = small(seed=5)
    opt = mlp.Adam(p, lr=3e-3)
    L0 = loss_of(p, F, U, X, nb)
    for _ in range(300):
        act = mlp.forward(p, F)
        L, dO = mlp.probe_loss(act["O"], U, X, nb)
        p = opt.step(p, mlp.backward(p, act, dO))
    assert loss_of(p, F, U, X, nb) < 0.2 * L0


def test_inverse_loss_zero_at_target_and_fd_gradient():
    rng = np.random.default_rng(11)
    B, nb = 4, 3
    T = np.eye(nb)[None] + 0.4 * rng.standard_normal((B, nb, nb))
    L, dO = mlp.inverse_loss((T - np.eye(nb)[None]).reshape(B, nb * nb), T, nb)
    assert L < 1e-28 and np.abs(dO).max() < 1e-14
    O = rng.standard_normal((B, nb * nb))
    L, dO = mlp.inverse_loss(O, T, nb)
    h = 1e-6
    for _ in range(8):
        i, j = rng.integers(0, B), rng.integers(0, nb * nb)
        Op, Om = O.copy(), O.copy()
        Op[i, j] += h
        Om[i, j] -= h
        fd = (mlp.inverse_loss(Op, T, nb)[0] - mlp.inverse_loss(Om, T, nb)[0]) / (2 * h)
        assert abs(fd - dO[i, j]) <= 1e-7 * max(1.0, abs(fd))


def test_inverse_loss_equals_probe_loss_with_unit_probes():
    """With S = I the probe loss over the complete set of unit probes is
    |M~ - I|_F^2 / (B nb), the inverse loss against T = I divided by nb."""
    rng = np.random.default_rng(12)
    B, nb = 3, 4
    O = rng.standard_normal((B, nb * nb))
    X = np.broadcast_to(np.eye(nb)[None], (B, nb, nb)).copy()     # probes p = unit vectors
    Lp, _ = mlp.probe_loss(O, X, X, nb)
    Li, _ = mlp.inverse_loss(O, np.broadcast_to(np.eye(nb)[None], (B, nb, nb)), nb)
    assert abs(Lp * nb - Li) <= 1e-12 * Li
