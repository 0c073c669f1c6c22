"""Device-allocation failures injected on the host (no GPU fault).

lbm_debug_fail_allocations makes the library's next allocations fail as if
the device were out of memory.  Each call that needs memory must return
LBM_ENOMEM and leave its object usable: a batch whose autotuner could not
back up its state keeps that state bit for bit.
"""
import numpy as np
import pytest


pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1311_2404_gb300 import lbm  # noqa: E402
from paper_1311_2404_gb300 import workloads as wl  # noqa: E402


def _specs():
    return wl.batch_channel_specs(4, nmin=33, nmax=120, seed=5)


def _batch(specs):
    b = lbm.lbm_batch_create([s["nx"] for s in specs], [s["ny"] for s in specs],
                             [s["tau"] for s in specs], lbm.LBM_F32S)
    for d, s in enumerate(specs):
        lbm.lbm_batch_set_geometry(b, d, wl.batch_channel_mask(s))
        lbm.lbm_batch_set_force(b, d, s["gx"], 0.0)
        rho, u = wl.random_state(s["nx"], s["ny"], 1, 2, seed=40 + d, u_amp=0.03)
        lbm.lbm_batch_init_equilibrium(b, d, rho, u)
    return b


def _fields(b, specs):
    out = []
    for d, s in enumerate(specs):
        r = np.empty((1, s["ny"], s["nx"]))
        u = np.empty((2, 1, s["ny"], s["nx"]))
        lbm.lbm_batch_get_macro(b, d, r, u)
        out.append((r, u))
    return out


def test_handle_batch_and_subdomain_allocation_failures():
    try:
        lbm.lbm_debug_fail_allocations(1)
        sim = lbm.Simulation(16, 8, 8, lbm.LBM_D3Q19, lbm.LBM_BGK, 0.6, lbm.LBM_F32S,
                             torch_memory=False)          # the library allocates
        with pytest.raises(lbm.LBMError) as ei:
            sim.init(np.ones((8, 8, 16)), np.zeros((3, 8, 8, 16)))
        assert ei.value.code == lbm.LBM_ENOMEM
        sim.init(np.ones((8, 8, 16)), np.zeros((3, 8, 8, 16)))   # the handle still works
        sim.step(2)
        sim.close()
        specs = _specs()
        lbm.lbm_debug_fail_allocations(1)
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_batch_create([s["nx"] for s in specs], [s["ny"] for s in specs],
                                 [s["tau"] for s in specs], lbm.LBM_F32S)
        assert ei.value.code == lbm.LBM_ENOMEM
        lbm.lbm_debug_fail_allocations(1)
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_multi_create(16, 8, 8, lbm.LBM_D3Q19, lbm.LBM_BGK, 0.6, lbm.LBM_F32S, 2)
        assert ei.value.code == lbm.LBM_ENOMEM
    finally:
        lbm.lbm_debug_fail_allocations(0)


def test_autotune_without_backup_memory_keeps_the_state():
    specs = _specs()
    ref = _batch(specs)
    lbm.lbm_batch_step(ref, 6)
    want = _fields(ref, specs)
    lbm.lbm_batch_destroy(ref)
    b = _batch(specs)
    lbm.lbm_batch_step(b, 3)
    try:
        lbm.lbm_debug_fail_allocations(1)
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_batch_autotune(b)
        assert ei.value.code == lbm.LBM_ENOMEM
    finally:
        lbm.lbm_debug_fail_allocations(0)
    lbm.lbm_batch_step(b, 3)
    got = _fields(b, specs)
    lbm.lbm_batch_destroy(b)
    for (r1, u1), (r2, u2) in zip(want, got):
        assert np.array_equal(r1, r2) and np.array_equal(u1, u2)


def test_training_allocation_failure():
    from oracle import mlp_oracle as mo
    rng = np.random.default_rng(3)
    X = rng.standard_normal((4096, 8)).astype(np.float32)
    X[:, 4] = np.abs(X[:, 4]) + 0.1
    alpha = 2.0 + 0.5 * X[:, 4] * np.tanh(X[:, 0])
    P = mo.init_params(3, X.mean(0), 1.0 / X.std(0), 0.5).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    ad = torch.from_numpy(alpha.astype(np.float64)).cuda()
    loss = np.zeros(3, dtype=np.float32)
    try:
        lbm.lbm_debug_fail_allocations(1)
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_mlp_train(Xd, ad, len(X), [3, 256, 3e-3, 5], P, loss)
        assert ei.value.code == lbm.LBM_ENOMEM
    finally:
        lbm.lbm_debug_fail_allocations(0)
    lbm.lbm_mlp_train(Xd, ad, len(X), [3, 256, 3e-3, 5], P, loss)
    assert np.all(np.isfinite(loss)) and loss[0] > 0
