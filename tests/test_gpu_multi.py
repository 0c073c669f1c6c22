"""Subdomain decomposition with ghost layers on one GPU (Sec. 3.6): slabs of
whole rows exchanging the direction-limited ghost rows after every step must
reproduce the single-domain run bit for bit, with walls crossing the slab
faces, forcing, every collision model and storage type, uneven slabs, slabs of
one and two rows, a single slab that is its own neighbour, with and without
the bulk/boundary overlap and under CUDA-graph replay.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1311_2404_gb300 import lbm  # noqa: E402
from paper_1311_2404_gb300 import workloads as wl  # noqa: E402


def _inputs(D, shape, seed):
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    mask = (rng.random(shape) < 0.12).astype(np.uint8)
    rho, u = wl.random_state(nx, ny, nz, D, seed=seed, u_amp=0.05, rho_amp=0.01)
    force = (1e-5, -2e-6, 0.0) if D == 2 else (1e-5, 2e-6, -3e-6)
    return mask, rho, u, force


def _single(D, model, dtype, shape, steps, mask, rho, u, force, tau):
    nz, ny, nx = shape
    lat = lbm.LBM_D2Q9 if D == 2 else lbm.LBM_D3Q19
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        sim = lbm.Simulation(nx, ny, nz, lat, model, tau, dtype, stream=s.cuda_stream)
        sim.set_geometry(mask)
        sim.set_force(*force)
        if model == lbm.LBM_SMAG:
            lbm.lbm_set_smagorinsky(sim.h, 0.15)
        if model == lbm.LBM_ELBM:
            lbm.lbm_set_elbm(sim.h, lbm.LBM_ALPHA_NEWTON, 1e-12, 20, 0.0)
        sim.init(rho, u)
        sim.step(steps)
        r, v = sim.macro()
        sim.close()
    return r, v


def _multi(D, model, dtype, shape, steps, mask, rho, u, force, tau, nsub, overlap, graph,
           split=1, direct=False):
    nz, ny, nx = shape
    lat = lbm.LBM_D2Q9 if D == 2 else lbm.LBM_D3Q19
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        m = lbm.lbm_multi_create(nx, ny, nz, lat, model, tau, dtype, nsub)
        lbm.lbm_multi_set_stream(m, s.cuda_stream)
        lbm.lbm_multi_set_overlap(m, overlap)
        lbm.lbm_multi_set_graph(m, graph)
        if direct:
            lbm.lbm_multi_set_transfer(m, lbm.LBM_TRANSFER_DIRECT)
        lbm.lbm_multi_set_geometry(m, mask)
        lbm.lbm_multi_set_force(m, *force)
        if model == lbm.LBM_SMAG:
            lbm.lbm_multi_set_smagorinsky(m, 0.15)
        if model == lbm.LBM_ELBM:
            lbm.lbm_multi_set_elbm(m, lbm.LBM_ALPHA_NEWTON, 1e-12, 20, 0.0)
        # device inputs for the fields
        lbm.lbm_multi_init_equilibrium(m, torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
        done = 0
        for k in range(split):
            n = steps // split + (1 if k < steps % split else 0)
            lbm.lbm_multi_step(m, n)
            done += n
        assert done == steps
        r = np.empty(rho.shape)
        v = np.empty(u.shape)
        lbm.lbm_multi_get_macro(m, r, v)
        hb = lbm.lbm_multi_halo_bytes(m)
        lbm.lbm_multi_destroy(m)
    return r, v, hb


CASES = [
    # D, model, dtype, shape (nz, ny, nx), nsub, overlap, graph
    (3, lbm.LBM_BGK, lbm.LBM_F32S, (13, 11, 37), 3, True, False),
    (3, lbm.LBM_BGK, lbm.LBM_F32S, (13, 11, 37), 3, False, False),
    (3, lbm.LBM_MRT, lbm.LBM_F16S, (10, 9, 33), 2, True, True),
    (3, lbm.LBM_ELBM, lbm.LBM_F64, (9, 7, 21), 3, True, False),
    (3, lbm.LBM_SMAG, lbm.LBM_BF16S, (12, 10, 40), 4, True, True),
    (3, lbm.LBM_REG, lbm.LBM_F32, (8, 9, 35), 4, False, True),     # 2-row slabs
    (3, lbm.LBM_BGK, lbm.LBM_F16S, (5, 9, 35), 5, True, False),    # 1-row slabs
    (3, lbm.LBM_BGK, lbm.LBM_F64, (6, 9, 35), 1, True, False),     # its own neighbour
    (2, lbm.LBM_BGK, lbm.LBM_F64, (1, 29, 45), 3, True, False),
    (2, lbm.LBM_REG, lbm.LBM_F16S, (1, 23, 70), 5, True, True),
    (2, lbm.LBM_ELBM, lbm.LBM_F32S, (1, 16, 40), 2, False, False),
    (2, lbm.LBM_SMAG, lbm.LBM_F32S, (1, 7, 40), 7, True, False),   # 1-row slabs
]


@pytest.mark.parametrize("case", CASES, ids=[f"D{c[0]}-m{c[1]}-t{c[2]}-S{c[4]}-o{int(c[5])}"
                                             f"-g{int(c[6])}" for c in CASES])
@pytest.mark.parametrize("steps", [6, 7])
def test_multi_equals_single_bitwise(case, steps):
    D, model, dtype, shape, nsub, overlap, graph = case
    mask, rho, u, force = _inputs(D, shape, seed=11 + nsub)
    tau = 0.52 if model == lbm.LBM_ELBM else 0.6
    r1, v1 = _single(D, model, dtype, shape, steps, mask, rho, u, force, tau)
    r2, v2, hb = _multi(D, model, dtype, shape, steps, mask, rho, u, force, tau, nsub, overlap,
                        graph, split=2)
    assert np.array_equal(r1, r2) and np.array_equal(v1, v2)
    r3, v3, _ = _multi(D, model, dtype, shape, steps, mask, rho, u, force, tau, nsub, overlap,
                       graph, split=1, direct=True)
    assert np.array_equal(r1, r3) and np.array_equal(v1, v3)
    nz, ny, nx = shape
    esize = {lbm.LBM_F64: 8, lbm.LBM_F32: 4, lbm.LBM_F32S: 4, lbm.LBM_F16S: 2,
             lbm.LBM_BF16S: 2}[dtype]
    ndir, row = (5, nx * ny) if D == 3 else (3, nx)
    assert hb == 2 * nsub * ndir * row * esize


def test_multi_rejects_bad_splits():
    with pytest.raises(lbm.LBMError):
        lbm.lbm_multi_create(16, 8, 4, lbm.LBM_D3Q19, lbm.LBM_BGK, 0.6, lbm.LBM_F32S, 5)
    with pytest.raises(lbm.LBMError):
        lbm.lbm_multi_create(16, 8, 1, lbm.LBM_D2Q9, lbm.LBM_BGK, 0.6, lbm.LBM_F32S, 0)
    m = lbm.lbm_multi_create(16, 8, 4, lbm.LBM_D3Q19, lbm.LBM_BGK, 0.6, lbm.LBM_F32S, 2)
    with pytest.raises(lbm.LBMError):
        lbm.lbm_multi_step(m, 1)                      # no initial state yet
    lbm.lbm_multi_destroy(m)
