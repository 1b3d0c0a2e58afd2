"""FP64 reference of the learned block preconditioner's network and its
training step.  Test infrastructure only (see ``oracle/__init__``).

The paper has no learned preconditioner; this is the oracle of the workload's
addition to the method: a per-element multilayer perceptron that maps the
element's features f (its state and the stage coefficients) to an approximate
inverse M~ = I + reshape(O) of the BJ_ext block S = I - c1 J + c2 J^2
(Sec. 3.2.3), trained with the probe loss

    L = sum_samples sum_p || M~ u_p - x_p ||^2 / (n_samples n_probes),   u_p = S x_p,

i.e. M~ S x_p should reproduce the probe x_p, or, to start training, with the
inverse regression L = sum_samples |M~ - S^-1|_F^2 / n_samples against exact
block inverses.

Network: two tanh hidden layers,
    z1 = W1 f + b1, h1 = tanh(z1), z2 = W2 h1 + b2, h2 = tanh(z2), O = W3 h2 + b3,
weights W (out x in); M~ = I + C_k + reshape(O) with C_k a fixed per-class
matrix (the mean block inverse minus I of the samples whose stage
coefficients (c1, c2) form class k; computed from the data, not trained).  Adam (Kingma & Ba 2015) updates every parameter with
m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, p -= lr m^/(sqrt(v^) + eps),
m^ = m / (1 - b1^t), v^ = v / (1 - b2^t).
"""
import numpy as np


def init_params(d_in, d_hidden, d_out, seed=0, out_scale=1e-3):
    rng = np.random.default_rng(seed)
    p = {
        "W1": rng.standard_normal((d_hidden, d_in)) / np.sqrt(d_in),
        "b1": np.zeros(d_hidden),
        "W2": rng.standard_normal((d_hidden, d_hidden)) / np.sqrt(d_hidden),
        "b2": np.zeros(d_hidden),
        "W3": out_scale * rng.standard_normal((d_out, d_hidden)) / np.sqrt(d_hidden),
        "b3": np.zeros(d_out),
    }
    return p


def forward(p, F):
    """F: (B, d_in) -> activations and O (B, d_out)."""
    z1 = F @ p["W1"].T + p["b1"]
    h1 = np.tanh(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.tanh(z2)
    O = h2 @ p["W3"].T + p["b3"]
    return {"F": F, "h1": h1, "h2": h2, "O": O}


def mtilde(O, nb, C=None):
    """M~ = I + C + reshape(O), row-major blocks (B, nb, nb); C (B, nb^2) is the
    fixed mean inverse (minus I) of each sample's stage class (None: 0)."""
    if C is not None:
        O = O + C
    return np.eye(nb)[None] + O.reshape(-1, nb, nb)


def probe_loss(O, U, X, nb, C=None):
    """L and dL/dO for probes X (B, P, nb) with U = S X (B, P, nb)."""
    B, P, _ = X.shape
    M = mtilde(O, nb, C)
    R = np.einsum("bij,bpj->bpi", M, U) - X          # residual M~ u_p - x_p
    L = np.sum(R * R) / (B * P)
    dM = 2.0 * np.einsum("bpi,bpj->bij", R, U) / (B * P)
    return L, dM.reshape(B, nb * nb)


def inverse_loss(O, T, nb, C=None):
    """Regression of M~ on the exact block inverses T (B, nb, nb):
    L = sum_s |M~_s - T_s|_F^2 / B and dL/dO (B, nb^2)."""
    B = T.shape[0]
    R = mtilde(O, nb, C) - T
    L = np.sum(R * R) / B
    return L, (2.0 * R / B).reshape(B, nb * nb)


def backward(p, act, dO):
    """Gradients of every parameter for the upstream gradient dO (B, d_out)."""
    h1, h2, F = act["h1"], act["h2"], act["F"]
    g = {}
    g["W3"] = dO.T @ h2
    g["b3"] = dO.sum(axis=0)
    dh2 = dO @ p["W3"]
    dz2 = dh2 * (1.0 - h2 * h2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (1.0 - h1 * h1)
    g["W1"] = dz1.T @ F
    g["b1"] = dz1.sum(axis=0)
    return g


class Adam:
    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = {k: np.zeros_like(v) for k, v in params.items()}
        self.v = {k: np.zeros_like(v) for k, v in params.items()}
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        for k in params:
            g = grads[k]
            self.m[k] = self.b1 * self.m[k] + (1.0 - self.b1) * g
            self.v[k] = self.b2 * self.v[k] + (1.0 - self.b2) * g * g
            mh = self.m[k] / (1.0 - self.b1 ** self.t)
            vh = self.v[k] / (1.0 - self.b2 ** self.t)
            params[k] = params[k] - self.lr * mh / (np.sqrt(vh) + self.eps)
        return params
