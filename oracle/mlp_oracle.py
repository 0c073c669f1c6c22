"""FP64 reference of the ELBM alpha surrogate: forward, backward, Adam.

TEST INFRASTRUCTURE ONLY.  The surrogate is not in the paper; it is an
8 -> 32 -> 32 -> 1 tanh network that maps eight lattice-symmetry invariants of
(f, f_eq - f) to a guess of the entropic over-relaxation alpha (Eq.
alpha_cond): it learns what the second-order small-deviation guess s2 misses,
alpha_guess = s2 + scale * out, with s2 written in the features
(t_3 = feature 0, t_4 = feature 1, eps = feature 4):
    s2 = 2 + (t_3 eps - 2 t_4 eps^2) / 3 + 4 t_3^2 eps^2 / 9.

Parameter vector layout (float64 here; the CUDA side keeps FP32 masters and a
BF16 copy of the weight matrices):
    [0:8]        feature mean            (fixed, from the training set)
    [8:16]       feature inverse std     (fixed)
    [16:272]     W1 [32][8]  row-major (out, in)
    [272:304]    b1 [32]
    [304:1328]   W2 [32][32]
    [1328:1360]  b2 [32]
    [1360:1392]  W3 [32]
    [1392]       b3
    [1393]       output scale            (fixed)
Trainable entries: [16:1393].  Loss: mean over the batch of (out - t)^2 with
t = (alpha* - s2) / scale.
Adam is Kingma & Ba (2015) with bias correction.
"""
from __future__ import annotations

import numpy as np

NIN, NH = 8, 32
O_MEAN, O_ISTD = 0, 8
O_W1 = 16
O_B1 = O_W1 + NH * NIN
O_W2 = O_B1 + NH
O_B2 = O_W2 + NH * NH
O_W3 = O_B2 + NH
O_B3 = O_W3 + NH
O_SCALE = O_B3 + 1
NPARAM = O_SCALE + 1
TRAIN_LO, TRAIN_HI = O_W1, O_SCALE


def unpack(P):
    P = np.asarray(P, dtype=np.float64)
    return dict(mean=P[O_MEAN:O_MEAN + NIN], istd=P[O_ISTD:O_ISTD + NIN],
                W1=P[O_W1:O_B1].reshape(NH, NIN), b1=P[O_B1:O_W2],
                W2=P[O_W2:O_B2].reshape(NH, NH), b2=P[O_B2:O_W3],
                W3=P[O_W3:O_B3], b3=P[O_B3], scale=P[O_SCALE])


def init_params(seed: int, mean, istd, scale: float) -> np.ndarray:
    """Glorot-uniform weights, zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    P = np.zeros(NPARAM)
    P[O_MEAN:O_MEAN + NIN] = mean
    P[O_ISTD:O_ISTD + NIN] = istd
    for lo, fan_in, fan_out in ((O_W1, NIN, NH), (O_W2, NH, NH), (O_W3, NH, 1)):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        P[lo:lo + fan_in * fan_out] = rng.uniform(-lim, lim, fan_in * fan_out)
    P[O_SCALE] = scale
    return P


def forward(P, X):
    """X [B, 8] features -> out [B] (and the activations for backward)."""
    p = unpack(P)
    Z = (np.asarray(X, dtype=np.float64) - p["mean"]) * p["istd"]
    H1 = np.tanh(Z @ p["W1"].T + p["b1"])
    H2 = np.tanh(H1 @ p["W2"].T + p["b2"])
    out = H2 @ p["W3"] + p["b3"]
    return out, (Z, H1, H2)


def series2(X):
    """Second-order small-deviation guess of alpha from the features: the
    expansion 2 + (a_3 - 2 a_4) / (3 a_2) + 4 a_3^2 / (9 a_2^2) with
    a_k = rho t_k eps^k."""
    X = np.asarray(X, dtype=np.float64)
    t3, t4, eps = X[:, 0], X[:, 1], X[:, 4]
    return 2.0 + (t3 * eps - 2.0 * t4 * eps * eps) / 3.0 + 4.0 * t3 * t3 * eps * eps / 9.0


def alpha_guess(P, X):
    out, _ = forward(P, X)
    return series2(X) + P[O_SCALE] * out


def target(P_or_scale, X, alpha):
    scale = P_or_scale if np.isscalar(P_or_scale) else P_or_scale[O_SCALE]
    return (np.asarray(alpha) - series2(X)) / scale


def loss_and_grad(P, X, t):
    """Mean-squared error and its gradient over the whole parameter vector
    (zeros at the fixed entries), by the chain rule layer by layer."""
    p = unpack(P)
    out, (Z, H1, H2) = forward(P, X)
    B = out.shape[0]
    r = out - np.asarray(t, dtype=np.float64)
    loss = float(np.mean(r * r))
    dout = 2.0 * r / B                              # dL/dout  [B]
    g = np.zeros(NPARAM)
    g[O_W3:O_B3] = dout @ H2
    g[O_B3] = dout.sum()
    dH2 = np.outer(dout, p["W3"])                   # [B, 32]
    dA2 = dH2 * (1.0 - H2 * H2)
    g[O_W2:O_B2] = (dA2.T @ H1).reshape(-1)
    g[O_B2:O_W3] = dA2.sum(axis=0)
    dH1 = dA2 @ p["W2"]
    dA1 = dH1 * (1.0 - H1 * H1)
    g[O_W1:O_B1] = (dA1.T @ Z).reshape(-1)
    g[O_B1:O_W2] = dA1.sum(axis=0)
    return loss, g


def adam_step(P, g, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update of the trainable entries; step counts from 1."""
    P = P.copy()
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    sl = slice(TRAIN_LO, TRAIN_HI)
    P[sl] -= lr * mh[sl] / (np.sqrt(vh[sl]) + eps)
    return P, m, v
