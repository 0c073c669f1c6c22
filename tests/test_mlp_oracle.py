"""Pins of the FP64 alpha-surrogate reference (CPU only).

- Backward pass against central finite differences of the loss.
- Adam's first step has the closed form  -lr * g / (|g| + eps)  (bias
  corrections cancel at step 1).
- The C oracle's forward pass (used inside its ELBM guarded mode) equals the
  NumPy forward pass.
"""
import numpy as np

import oracle.mlp_oracle as mo


def _setup(seed=0, B=64):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((B, 8)) * np.array([1, 2, 3, 4, 1e-2, 2, 2, 1.0])
    X[:, 4] = np.abs(X[:, 4]) + 1e-3
    P = mo.init_params(seed, X.mean(0), 1.0 / X.std(0), 0.5)
    P[mo.O_B1:mo.O_W2] = rng.standard_normal(mo.NH) * 0.1
    P[mo.O_B2:mo.O_W3] = rng.standard_normal(mo.NH) * 0.1
    t = rng.standard_normal(B)
    return P, X, t


def test_gradient_matches_finite_differences():
    P, X, t = _setup()
    _, g = mo.loss_and_grad(P, X, t)
    assert np.all(g[:mo.TRAIN_LO] == 0) and g[mo.O_SCALE] == 0
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(np.arange(lo, hi), 12, replace=False)
                          for lo, hi in ((mo.O_W1, mo.O_B1), (mo.O_B1, mo.O_W2),
                                         (mo.O_W2, mo.O_B2), (mo.O_B2, mo.O_W3),
                                         (mo.O_W3, mo.O_B3))] + [np.array([mo.O_B3])])
    h = 1e-6
    for i in idx:
        Pp = P.copy(); Pp[i] += h
        Pm = P.copy(); Pm[i] -= h
        fd = (mo.loss_and_grad(Pp, X, t)[0] - mo.loss_and_grad(Pm, X, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_adam_first_step_closed_form():
    P, X, t = _setup(2)
    _, g = mo.loss_and_grad(P, X, t)
    m = np.zeros_like(P)
    v = np.zeros_like(P)
    lr, eps = 1e-3, 1e-8
    P1, m1, v1 = mo.adam_step(P, g, m, v, 1, lr=lr, eps=eps)
    sl = slice(mo.TRAIN_LO, mo.TRAIN_HI)
    assert np.allclose(P1[sl] - P[sl], -lr * g[sl] / (np.abs(g[sl]) + eps), rtol=1e-12, atol=1e-18)
    assert np.array_equal(P1[:mo.TRAIN_LO], P[:mo.TRAIN_LO])
    # and the loss decreases for a small enough step
    P2, _, _ = mo.adam_step(P, g, m, v, 1, lr=1e-5)
    assert mo.loss_and_grad(P2, X, t)[0] < mo.loss_and_grad(P, X, t)[0]


def test_c_forward_equals_numpy_forward(oracle_lib):
    P, X, _ = _setup(3, B=16)
    ref = mo.alpha_guess(P, X)
    got = np.array([oracle_lib.mlp_guess(P, x) for x in X])
    assert np.abs(ref - got).max() < 1e-14


def test_training_reduces_loss_on_smooth_target():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((512, 8))
    X[:, 4] = np.abs(X[:, 4]) + 0.1
    t = np.tanh(X[:, 0]) * 0.5 + 0.2 * X[:, 1]
    P = mo.init_params(4, X.mean(0), 1.0 / X.std(0), 1.0)
    m = np.zeros_like(P)
    v = np.zeros_like(P)
    l0 = mo.loss_and_grad(P, X, t)[0]
    for step in range(1, 301):
        _, g = mo.loss_and_grad(P, X, t)
        P, m, v = mo.adam_step(P, g, m, v, step, lr=3e-3)
    assert mo.loss_and_grad(P, X, t)[0] < 0.05 * l0
