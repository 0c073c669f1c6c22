"""The allocation-free gradient entry point (GPU).

lbm_mlp_grad_static serves callers that cannot call cudaMalloc (for example
next to another framework's caching allocator that holds the free device
memory, or on a real-time path where an allocation may synchronise the
device).  It must give the same loss and gradient as lbm_mlp_grad, which
allocates its scratch, within the tolerance the gradient tests use, on two
calls in a row (the second with different data, so stale scratch contents
would show), and reject batches larger than its static scratch.
This file sorts last so that a run stopping at the first failure has run
every other test before it.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle.mlp_oracle as mo  # noqa: E402
from paper_1311_2404_gb300 import lbm  # noqa: E402


def _batch(seed, B):
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((B, 8)) * np.array([1, 2, 3, 4, 1e-2, 2, 2, 1.0])).astype(np.float32)
    X[:, 4] = np.abs(X[:, 4]) + 1e-3
    P = mo.init_params(seed, X.mean(0), 1.0 / X.std(0), 0.5).astype(np.float32)
    P[mo.O_B1:mo.O_W2] = (rng.standard_normal(mo.NH) * 0.1).astype(np.float32)
    t = (rng.standard_normal(B) * 0.3).astype(np.float32)
    return torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda(), P


def test_static_gradient_matches_allocating_entry_point():
    for seed, B in ((0, 4096), (1, 1000)):
        X, t, P = _batch(seed, B)
        l_ref, g_ref = lbm.lbm_mlp_grad(X, t, B, P)
        l_st, g_st = lbm.lbm_mlp_grad_static(X, t, B, P)
        assert abs(l_st - l_ref) <= 1e-5 * abs(l_ref)
        sl = slice(mo.TRAIN_LO, mo.TRAIN_HI)
        assert np.abs(g_st[sl] - g_ref[sl]).max() <= 1e-4 * np.abs(g_ref[sl]).max()
        assert np.all(g_st[:mo.TRAIN_LO] == 0) and g_st[mo.O_SCALE] == 0


def test_static_gradient_rejects_oversized_batch():
    X, t, P = _batch(2, 4097)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_mlp_grad_static(X, t, 4097, P)
    assert ei.value.code == lbm.LBM_EINVAL
    assert "4096" in str(ei.value)
