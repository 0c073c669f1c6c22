"""Slab decomposition across processes (Sec. 3.6) on the GPU: one process
per slab, the faces moved between processes through torch.distributed
(gloo, staged through host memory), against the single-domain handle bit
for bit.

Every process of a test uses the one GPU of the machine, each with its own
context; the processes exchange faces on the host between launches, so no
kernel waits for another process.
"""
import os
import socket
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1311_2404_gb300 import lbm  # noqa: E402
from paper_1311_2404_gb300 import workloads as wl  # noqa: E402

SHAPE = (20, 18, 37)            # nz, ny, nx: ragged x, z split into 2 or 3 slabs
CASES = [(lbm.LBM_F32S, True, 7), (lbm.LBM_F32S, False, 6), (lbm.LBM_F16S, True, 8),
         (lbm.LBM_F16S, False, 5)]


def _inputs():
    nz, ny, nx = SHAPE
    mask = wl.channel_mask(nx, ny, nz)
    rng = np.random.default_rng(5)
    mask[(rng.random(SHAPE) < 0.05)] = 1
    rho, u = wl.random_state(nx, ny, nz, 3, seed=9, u_amp=0.04, rho_amp=0.01)
    return mask, rho, u


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    from paper_1311_2404_gb300 import slabs
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        nz, ny, nx = SHAPE
        mask, rho, u = _inputs()
        for k, (dtype, overlap, steps) in enumerate(CASES):
            sl = slabs.RankSlab(nx, ny, nz, lbm.LBM_D3Q19, lbm.LBM_BGK, 0.6, dtype, rank, world,
                                overlap=overlap)
            assert sl.host_staged
            sl.set_geometry(mask)
            sl.set_force(1e-5, 2e-6, 0.0)
            sl.init(rho, u)
            sl.step(steps)
            r, v = sl.macro()
            hb = sl.halo_bytes()
            sl.close()
            # each rank wrote only its rows; the sum over ranks assembles the fields
            rt, vt = torch.from_numpy(r), torch.from_numpy(v)
            dist.all_reduce(rt)
            dist.all_reduce(vt)
            if rank == 0:
                np.save(os.path.join(outdir, f"case{k}_rho.npy"), rt.numpy())
                np.save(os.path.join(outdir, f"case{k}_u.npy"), vt.numpy())
                np.save(os.path.join(outdir, f"case{k}_halo.npy"), np.array([hb]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_rank_slabs_equal_single_domain(world):
    nz, ny, nx = SHAPE
    mask, rho, u = _inputs()
    with tempfile.TemporaryDirectory() as outdir:
        mp.start_processes(_rank_main, args=(world, _free_port(), outdir), nprocs=world,
                           join=True, start_method="spawn")
        for k, (dtype, overlap, steps) in enumerate(CASES):
            sim = lbm.Simulation(nx, ny, nz, lbm.LBM_D3Q19, lbm.LBM_BGK, 0.6, dtype)
            sim.set_geometry(mask)
            sim.set_force(1e-5, 2e-6, 0.0)
            sim.init(rho, u)
            sim.step(steps)
            r1, v1 = sim.macro()
            sim.close()
            r2 = np.load(os.path.join(outdir, f"case{k}_rho.npy"))
            v2 = np.load(os.path.join(outdir, f"case{k}_u.npy"))
            assert np.array_equal(r1, r2) and np.array_equal(v1, v2), (world, k)
            # the rank sends its two faces: 5 directions of one padded row each
            hb = int(np.load(os.path.join(outdir, f"case{k}_halo.npy"))[0])
            es = 4 if dtype == lbm.LBM_F32S else 2
            assert hb == 2 * 5 * nx * ny * es


def test_rank_handle_refuses_plain_steps_and_bad_ranks():
    m = lbm.lbm_multi_create_rank(16, 8, 8, lbm.LBM_D3Q19, lbm.LBM_BGK, 0.6, lbm.LBM_F32S, 2, 1)
    try:
        assert lbm.lbm_multi_rows(m) == (4, 8)
        rho = np.ones((8, 8, 16))
        u = np.zeros((3, 8, 8, 16))
        lbm.lbm_multi_init_equilibrium(m, rho, u)
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_multi_step(m, 1)
        assert ei.value.code == lbm.LBM_ESTATE
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_multi_step_end(m)
        assert ei.value.code == lbm.LBM_ESTATE
    finally:
        lbm.lbm_multi_destroy(m)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_multi_create_rank(16, 8, 8, lbm.LBM_D3Q19, lbm.LBM_BGK, 0.6, lbm.LBM_F32S, 2, 2)
    assert ei.value.code == lbm.LBM_EINVAL
