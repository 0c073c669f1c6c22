"""Train the ELBM alpha surrogate on the GPU from the library's own
Newton-solved ELBM runs (not part of the paper's method).

collect_pairs(): run a D3Q19 ELBM simulation with the full FP64 Newton solve
and capture (8 invariant features, converged alpha) pairs from its output
steps (lbm_elbm_collect_pairs).  train(): minibatch Adam on the GPU
(lbm_mlp_train).  Both only marshal arguments; all work runs in liblbm.so.
"""
from __future__ import annotations

import numpy as np

from . import lbm
from . import workloads as wl

NIN, NH = 8, 32
O_MEAN, O_ISTD, O_W1 = 0, 8, 16
O_SCALE = lbm.MLP_NPARAM - 1


def init_params(seed: int, mean, istd, scale: float) -> np.ndarray:
    """Glorot-uniform weights, zero biases, fixed input normalisation and
    output scale (layout of lbm_load_alpha_mlp)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    P = np.zeros(lbm.MLP_NPARAM, dtype=np.float64)
    P[O_MEAN:O_MEAN + NIN] = mean
    P[O_ISTD:O_ISTD + NIN] = istd
    o = O_W1
    for fan_in, fan_out in ((NIN, NH), (NH, NH), (NH, 1)):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        P[o:o + fan_in * fan_out] = rng.uniform(-lim, lim, fan_in * fan_out)
        o += fan_in * fan_out + fan_out
    P[O_SCALE] = scale
    return P.astype(np.float32)


def collect_pairs(n=64, tau=0.5005, rounds=6, steps_between=3, skip_eps=1e-4, seed=2404):
    """(X [m, 8] float32 CUDA tensor, alpha [m] float64 CUDA tensor, state, t)."""
    import torch
    rho, u = wl.turbulence(n, k0=4.0, u_rms=0.04, seed=seed)
    sim = lbm.Simulation(n, n, n, lbm.LBM_D3Q19, lbm.LBM_ELBM, tau, lbm.LBM_F32S)
    lbm.lbm_set_elbm(sim.h, lbm.LBM_ALPHA_NEWTON, 1e-12, 20, skip_eps)
    sim.init(rho, u)
    cap = n * n * n
    X = torch.empty((cap, 8), dtype=torch.float32, device="cuda")
    y = torch.empty(cap, dtype=torch.float64, device="cuda")
    Xs, ys = [], []
    for _ in range(rounds):
        sim.step(steps_between)
        cnt = lbm.lbm_elbm_collect_pairs(sim.h, 1, X, y)
        Xs.append(X[:cnt].clone())
        ys.append(y[:cnt].clone())
    state, t = sim.state()
    sim.close()
    return torch.cat(Xs), torch.cat(ys), state, t


def series2(Xh):
    """The second-order small-deviation guess of alpha from feature rows
    (t_3, t_4 and eps in columns 0, 1, 4): the part the network does not
    learn (alpha guess = series2 + scale * out)."""
    t3, t4, eps = Xh[:, 0], Xh[:, 1], Xh[:, 4]
    return 2.0 + (t3 * eps - 2.0 * t4 * eps * eps) / 3.0 + 4.0 * t3 * t3 * eps * eps / 9.0


def collect_pairs_from(sim, rounds=3, steps_between=2, stride=16, cap=1 << 21):
    """Pairs from an ELBM Simulation in its current state: `rounds` times,
    `steps_between` steps then one captured step (every stride-th eligible
    node).  The handle's alpha mode is used as set (Newton gives exact
    targets).  Returns (X, alpha) CUDA tensors."""
    import torch
    X = torch.empty((cap, 8), dtype=torch.float32, device="cuda")
    y = torch.empty(cap, dtype=torch.float64, device="cuda")
    Xs, ys = [], []
    for _ in range(rounds):
        if steps_between:
            sim.step(steps_between)
        cnt = lbm.lbm_elbm_collect_pairs(sim.h, stride, X, y)
        Xs.append(X[:cnt].clone())
        ys.append(y[:cnt].clone())
    return torch.cat(Xs), torch.cat(ys)


def train(X, alpha, epochs=20, batch=1024, lr=2e-3, seed=13, kernel=None):
    """Parameters (float32, 1394) trained on the GPU; returns (params, loss per epoch).
    The output scale is the spread of the targets alpha - series2.  kernel:
    lbm.LBM_MLP_FP32 or lbm.LBM_MLP_BF16_TC (the default: trains the network
    with the BF16 rounding lbm_load_alpha_mlp applies for inference)."""
    Xh = X.double().cpu().numpy()
    ah = alpha.cpu().numpy()
    scale = float(np.std(ah - series2(Xh)))
    P = init_params(seed, Xh.mean(0), 1.0 / (Xh.std(0) + 1e-12), scale)
    loss = np.zeros(epochs, dtype=np.float32)
    if kernel is None:
        kernel = lbm.LBM_MLP_BF16_TC
    lbm.lbm_mlp_train_cfg(X, alpha, int(alpha.numel()), epochs, batch, lr, seed, kernel, P, loss)
    return P, loss
