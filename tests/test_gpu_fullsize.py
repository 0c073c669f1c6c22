"""Parity at the full workload sizes, in the launch configuration the
benchmark times, on sampled nodes.

After T steps a node's state depends only on the nodes within T links of it,
so the FP64 oracle reproduces a sampled node exactly by running T steps on the
(2T+1)^3 box around it, cut from the full initial fields and geometry with the
domain's periodic images (the box's own wrap-around only reaches the centre
after T + 1 steps).  Each GPU run is the full 512x256x256 duct, 256^3
turbulence, 254^3 cavity or 350^3 Kida vortex; the batched ensemble's 512
channels are compared whole, sampled by channel.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1311_2404_gb300 import lbm  # noqa: E402
from paper_1311_2404_gb300 import workloads as wl  # noqa: E402


def _box(a, c, r):
    """Periodic box of side 2r+1 around c = (z, y, x) from a [..., nz, ny, nx]."""
    nz, ny, nx = a.shape[-3:]
    iz = np.arange(c[0] - r, c[0] + r + 1) % nz
    iy = np.arange(c[1] - r, c[1] + r + 1) % ny
    ix = np.arange(c[2] - r, c[2] + r + 1) % nx
    return np.ascontiguousarray(a[..., iz[:, None, None], iy[None, :, None], ix[None, None, :]])


def _run_gpu(shape, lattice, model, tau, dtype, rho, u, T, mask=None, force=(0, 0, 0), bcs=(),
             setup=None):
    nz, ny, nx = shape
    sim = lbm.Simulation(nx, ny, nz, lattice, model, tau, dtype)
    for b in bcs:
        lbm.lbm_set_boundary(sim.h, *b)
    if setup:
        setup(sim)
    if mask is not None:
        sim.set_geometry(mask)
    if any(force):
        sim.set_force(*force)
    sim.init(torch.from_numpy(rho.astype(np.float32)).cuda(),
             torch.from_numpy(u.astype(np.float32)).cuda())
    sim.step(T)
    rg = torch.empty((nz, ny, nx), dtype=torch.float64, device="cuda")
    ug = torch.empty((3, nz, ny, nx), dtype=torch.float64, device="cuda")
    lbm.lbm_get_macro(sim.h, rg, ug)
    sim.close()
    return rg, ug


def _check_samples(rg, ug, rho, u, mask, T, pkw, samples, tol, bcs=()):
    r = T
    worst = 0.0
    for c in samples:
        rb = _box(rho.astype(np.float32).astype(np.float64), c, r)
        ub = _box(u.astype(np.float32).astype(np.float64), c, r)
        mb = _box(mask, c, r) if mask is not None else None
        s = 2 * r + 1
        p = oracle.make_params(s, s, s, **pkw)
        for b in bcs:
            oracle.set_bc(p, *b)
        F = oracle.init(p, rb, ub)
        ro, uo, _, _ = oracle.run(p, F, T, mb)
        go_r = float(rg[c].item())
        go_u = np.array([float(ug[(a,) + tuple(c)].item()) for a in range(3)])
        er = abs(go_r - ro[r, r, r])
        eu = np.abs(go_u - uo[:, r, r, r]).max() / max(np.abs(uo[:, r, r, r]).max(), 1e-3)
        worst = max(worst, eu)
        assert er < tol and eu < tol, (c, er, eu)
    return worst


def _samples(shape, mask, k, seed):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    out = []
    while len(out) < k:
        c = (int(rng.integers(nz)), int(rng.integers(ny)), int(rng.integers(nx)))
        if mask is None or mask[c] != 1:
            out.append(c)
    return out


def test_duct_full_size_sampled_parity():
    """512x256x256 sphere duct, MRT, FP32S (the benchmark's configuration),
    12 steps from rest with the body force; 6 sampled fluid nodes and the
    fluid neighbour of a sphere."""
    nx, ny, nz = 512, 256, 256
    mask, _ = wl.duct_with_spheres(nx, ny, nz)
    rho = np.ones((nz, ny, nx))
    u = np.zeros((3, nz, ny, nx))
    T, tau, F = 12, 0.55, (1e-5, 0.0, 0.0)
    rg, ug = _run_gpu((nz, ny, nx), lbm.LBM_D3Q19, lbm.LBM_MRT, tau, lbm.LBM_F32S, rho, u, T,
                      mask, F)
    samples = _samples((nz, ny, nx), mask, 6, 1)
    # a fluid node next to a solid one
    fl = np.argwhere((mask == 0) & (np.roll(mask, 1, axis=2) == 1))
    samples.append(tuple(int(v) for v in fl[len(fl) // 2]))
    w = _check_samples(rg, ug, rho, u, mask, T, dict(D=3, model=oracle.MRT, tau=tau, force=F),
                       samples, 1e-5)
    print(f"duct full size: worst relative velocity error {w:.2e}")


@pytest.mark.parametrize("alpha_mode", [lbm.LBM_ALPHA_NEWTON, lbm.LBM_ALPHA_SERIES_GUARDED])
def test_turbulence_elbm_full_size_sampled_parity(alpha_mode):
    """256^3 decaying turbulence, ELBM, FP32S, skip 1e-3 (the benchmark's
    configuration), 4 steps; 5 sampled nodes."""
    n, tau, T = 256, 0.5005, 4
    rho, u = wl.turbulence(n)
    rg, ug = _run_gpu((n, n, n), lbm.LBM_D3Q19, lbm.LBM_ELBM, tau, lbm.LBM_F32S, rho, u, T,
                      setup=lambda s: lbm.lbm_set_elbm(s.h, alpha_mode, 1e-12, 20, 1e-3))
    w = _check_samples(rg, ug, rho, u, None, T,
                       dict(D=3, model=oracle.ELBM, tau=tau, skip_eps=1e-3,
                            alpha_mode=oracle.NEWTON), _samples((n, n, n), None, 5, 2), 1e-5)
    print(f"turbulence full size: worst relative velocity error {w:.2e}")


def test_cavity_full_size_sampled_parity():
    """254^3 lid-driven cavity, LBGK, FP32S, regularized lid (the benchmark's
    configuration), 12 steps; samples under the lid, at a wall and inside."""
    n, T = 254, 12
    mask = wl.ldc_mask(n)
    tau = wl.ldc_tau(n)
    rho = np.ones(mask.shape)
    u = np.zeros((3,) + mask.shape)
    bcs = [(0, lbm.LBM_BC_VELOCITY, lbm.LBM_BC_REGULARIZED, -2, [0.05, 0.0, 0.0])]
    rg, ug = _run_gpu(mask.shape, lbm.LBM_D3Q19, lbm.LBM_BGK, tau, lbm.LBM_F32S, rho, u, T,
                      mask, bcs=bcs)
    samples = [(n // 2, n - 1, n // 2), (n // 2, n - 2, 5), (3, n - 1, n - 2), (n // 2, 1, n // 2),
               (100, 200, 150)]
    w = _check_samples(rg, ug, rho, u, mask, T, dict(D=3, model=oracle.BGK, tau=tau), samples,
                       1e-5, bcs=[(0, oracle.BC_VELOCITY, oracle.BC_REGULARIZED, -2,
                                   [0.05, 0.0, 0.0])])
    print(f"cavity full size: worst relative velocity error {w:.2e}")


def test_kida_full_size_sampled_parity():
    """350^3 Kida vortex, Smagorinsky, FP32S (the benchmark's configuration),
    8 steps; 5 sampled nodes."""
    n, T = 350, 8
    tau = 0.5 + 3 * n * 0.05 / 4000
    rho, u = wl.kida(n, 0.05)
    rg, ug = _run_gpu((n, n, n), lbm.LBM_D3Q19, lbm.LBM_SMAG, tau, lbm.LBM_F32S, rho, u, T)
    w = _check_samples(rg, ug, rho, u, None, T,
                       dict(D=3, model=oracle.SMAG, tau=tau, smag_cs=0.1),
                       _samples((n, n, n), None, 5, 3), 1e-5)
    print(f"Kida full size: worst relative velocity error {w:.2e}")


def test_batched_ensemble_full_size_sampled_parity():
    """The benchmark's ensemble: 512 D2Q9 channels of uneven sizes (64..1024 a
    side), each with a cylinder and its own tau and force, started from rest,
    autotuned and advanced in persistent launches (FP32S).  After 200 steps
    the three smallest channels and the median-sized one equal the FP64 oracle
    run on each channel alone (relative L2 1e-5); solid nodes report 0."""
    specs = wl.batch_channel_specs(512)
    T = 200
    b = lbm.lbm_batch_create([s["nx"] for s in specs], [s["ny"] for s in specs],
                             [s["tau"] for s in specs], lbm.LBM_F32S)
    masks = []
    for d, sp in enumerate(specs):
        m = wl.batch_channel_mask(sp)
        masks.append(m)
        lbm.lbm_batch_set_geometry(b, d, m)
        lbm.lbm_batch_set_force(b, d, sp["gx"], 0.0)
        lbm.lbm_batch_init_equilibrium(b, d, np.ones((1, sp["ny"], sp["nx"]), np.float32),
                                       np.zeros((2, 1, sp["ny"], sp["nx"]), np.float32))
    lbm.lbm_batch_autotune(b)
    lbm.lbm_batch_step(b, T // 2)
    lbm.lbm_batch_step(b, T - T // 2)
    sizes = np.array([s["nx"] * s["ny"] for s in specs])
    order = np.argsort(sizes, kind="stable")
    pick = list(order[:3]) + [order[len(order) // 2]]
    for d in pick:
        sp = specs[d]
        r = np.empty((1, sp["ny"], sp["nx"]))
        u = np.empty((2, 1, sp["ny"], sp["nx"]))
        lbm.lbm_batch_get_macro(b, int(d), r, u)
        p = oracle.make_params(sp["nx"], sp["ny"], 1, D=2, model=oracle.BGK, tau=sp["tau"],
                               force=(sp["gx"], 0.0, 0.0))
        F = oracle.init(p, np.ones((1, sp["ny"], sp["nx"])), np.zeros((2, 1, sp["ny"], sp["nx"])))
        ro, uo, _, _ = oracle.run(p, F, T, masks[d])
        fl = masks[d] == 0
        eu = np.sqrt(((u[:, fl] - uo[:, fl]) ** 2).sum() / (uo[:, fl] ** 2).sum())
        er = np.sqrt(((r[fl] - ro[fl]) ** 2).sum() / (ro[fl] ** 2).sum())
        assert eu < 1e-5 and er < 1e-5, (int(d), eu, er)
        assert np.all(r[~fl] == 0) and np.all(u[:, ~fl] == 0)
    lbm.lbm_batch_destroy(b)
