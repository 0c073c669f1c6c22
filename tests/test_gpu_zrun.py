"""Masked 3-D steps in z runs (the node word of the next layer loaded ahead).

The z-run kernel and the one-node kernel load the same populations (streamed
from x - e_i, or the node's own opposite population behind a solid link,
Sec. 2.3) and apply the same collision, so every field and the stored state
must agree bitwise, on every lattice, model and storage, with forcing, boundary
nodes and run lengths that do not divide the domain.  The geometry statistic
that picks the kernel is checked against a count made here from the mask.
"""
import numpy as np
import pytest

import analytic as an
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1311_2404_gb300 import lbm  # noqa: E402
from paper_1311_2404_gb300 import workloads as wl  # noqa: E402


def _mask(shape, solid=0.15, seed=8):
    rng = np.random.default_rng(seed)
    m = (rng.random(shape) < solid).astype(np.uint8)
    m[:, 0, :] = 1
    m[0, :, :] = 1
    return m


def _run(mode, lat, model, dtype, shape, steps, mask, force=(0, 0, 0), bcs=(), tau=0.7,
         seed=3):
    nz, ny, nx = shape
    rho, u = wl.random_state(nx, ny, nz, 3, seed=seed, u_amp=0.04, rho_amp=0.01)
    sim = lbm.Simulation(nx, ny, nz, lat, model, tau, dtype)
    lbm.lbm_set_masked_kernel(sim.h, mode)
    if model == lbm.LBM_SMAG:
        lbm.lbm_set_smagorinsky(sim.h, 0.15)
    for b in bcs:
        lbm.lbm_set_boundary(sim.h, *b)
    sim.set_geometry(mask)
    if any(force):
        sim.set_force(*force)
    sim.init(rho, u)
    sim.step(steps)
    r, v = sim.macro()
    st, t = sim.state()
    frac = lbm.lbm_get_nearwall_fraction(sim.h)
    sim.close()
    return r, v, st, frac, rho, u


@pytest.mark.parametrize("lat,model,dtype", [
    (lbm.LBM_D3Q19, lbm.LBM_BGK, lbm.LBM_F32S),
    (lbm.LBM_D3Q19, lbm.LBM_MRT, lbm.LBM_F32S),
    (lbm.LBM_D3Q19, lbm.LBM_MRT, lbm.LBM_F16S),
    (lbm.LBM_D3Q19, lbm.LBM_BGK, lbm.LBM_BF16S),
    (lbm.LBM_D3Q19, lbm.LBM_REG, lbm.LBM_F16S),
    (lbm.LBM_D3Q19, lbm.LBM_SMAG, lbm.LBM_F32S),
    (lbm.LBM_D3Q19, lbm.LBM_BGK, lbm.LBM_F64),
    (lbm.LBM_D3Q19, lbm.LBM_MRT, lbm.LBM_F32),
    (lbm.LBM_D3Q15, lbm.LBM_BGK, lbm.LBM_F32S),
    (lbm.LBM_D3Q27, lbm.LBM_REG, lbm.LBM_F16S)])
def test_zrun_equals_node_kernel_bitwise(lat, model, dtype):
    shape = (19, 13, 37)          # 19 layers: runs of 8, 8 and 3
    mask = _mask(shape)
    force = (1e-5, 2e-6, -3e-6)
    a = _run(lbm.LBM_MASKED_NODE, lat, model, dtype, shape, 9, mask, force)
    b = _run(lbm.LBM_MASKED_ZRUN, lat, model, dtype, shape, 9, mask, force)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(a[2], b[2])


def test_zrun_with_boundary_nodes_bitwise():
    # a regularized velocity plane and a Zou-He pressure plane between walls
    shape = (12, 10, 33)
    nz, ny, nx = shape
    mask = _mask(shape, solid=0.05)
    mask[:, :, 1] = 2
    mask[:, :, nx - 2] = 3
    mask[:, 0, :] = 1
    mask[0, :, :] = 1
    bcs = [(0, lbm.LBM_BC_VELOCITY, lbm.LBM_BC_REGULARIZED, 1, [0.02, 0.0, 0.0]),
           (1, lbm.LBM_BC_PRESSURE, lbm.LBM_BC_ZOUHE, -1, [1.0])]
    for dtype in (lbm.LBM_F32S, lbm.LBM_F16S):
        a = _run(lbm.LBM_MASKED_NODE, lbm.LBM_D3Q19, lbm.LBM_BGK, dtype, shape, 6, mask,
                 bcs=bcs)
        b = _run(lbm.LBM_MASKED_ZRUN, lbm.LBM_D3Q19, lbm.LBM_BGK, dtype, shape, 6, mask,
                 bcs=bcs)
        assert np.array_equal(a[0], b[0], equal_nan=True)
        assert np.array_equal(a[1], b[1], equal_nan=True)
        assert np.array_equal(a[2], b[2])


def test_zrun_vs_oracle_sphere_duct_copy():
    # a reduced sphere duct (walls on the y and z faces, spheres r 4..12),
    # MRT with the duct's force and tau, z-run kernel against the FP64 oracle
    mask, _ = wl.duct_with_spheres(48, 32, 32, seed=5)
    nz, ny, nx = mask.shape
    steps = 12
    r, v, _, frac, rho, u = _run(lbm.LBM_MASKED_ZRUN, lbm.LBM_D3Q19, lbm.LBM_MRT,
                                 lbm.LBM_F32S, mask.shape, steps, mask, (1e-5, 0, 0),
                                 tau=0.55)
    p = oracle.make_params(nx, ny, nz, D=3, model=oracle.MRT, tau=0.55, force=(1e-5, 0, 0))
    F = oracle.init(p, rho, u)
    ro, uo, _, _ = oracle.run(p, F, steps, mask)
    fl = mask == 0
    e_r, e_abs = an.rho_errors(r, ro, fl)
    print(f"z-run duct MRT FP32S: u {an.rel_l2(v[:, fl], uo[:, fl]):.2e} rho-1 {e_r:.2e} "
          f"max|drho| {e_abs:.2e}")
    assert an.rel_l2(v[:, fl], uo[:, fl]) < 1e-5
    assert e_r < 1e-5 and e_abs < 1e-7
    assert np.all(r[~fl] == 0) and np.all(v[:, ~fl] == 0)


def _nearwall_fraction(mask, E):
    """Share of x-aligned 32-node row segments holding a fluid node with a
    solid upstream neighbour (periodic), counted directly from the mask."""
    solid = mask == 1
    near = np.zeros_like(solid)
    for e in E:
        near |= np.roll(solid, shift=(e[2], e[1], e[0]), axis=(0, 1, 2))
    near &= ~solid
    nz, ny, nx = mask.shape
    segs = -(-nx // 32)
    pad = np.zeros((nz, ny, segs * 32), bool)
    pad[:, :, :nx] = near
    return pad.reshape(nz, ny, segs, 32).any(-1).mean()


def test_nearwall_statistic_and_choice():
    E19 = [(x, y, z) for z in (-1, 0, 1) for y in (-1, 0, 1) for x in (-1, 0, 1)
           if 0 < x * x + y * y + z * z <= 2]
    duct, _ = wl.duct_with_spheres(96, 48, 40, seed=2)
    chan = wl.channel_mask(256, 24, 10)        # walls at y = 0, 23 only
    for m in (duct, chan, wl.ldc_mask(70), _mask((9, 7, 70), solid=0.02)):
        nz, ny, nx = m.shape
        sim = lbm.Simulation(nx, ny, nz, lbm.LBM_D3Q19, lbm.LBM_BGK, 0.7, lbm.LBM_F32S)
        sim.set_geometry(m)
        got = lbm.lbm_get_nearwall_fraction(sim.h)
        sim.close()
        assert got == pytest.approx(_nearwall_fraction(m, E19), abs=1e-12)
    # spheres put a near-wall node into most segments, flat walls into few
    assert _nearwall_fraction(duct, E19) > 0.4 > _nearwall_fraction(chan, E19)
    sim = lbm.Simulation(40, 8, 8, lbm.LBM_D3Q19, lbm.LBM_BGK, 0.7, lbm.LBM_F32S)
    with pytest.raises(lbm.LBMError):
        lbm.lbm_get_nearwall_fraction(sim.h)
    with pytest.raises(lbm.LBMError):
        lbm.lbm_set_masked_kernel(sim.h, 3)
    sim.close()


@pytest.mark.parametrize("mode", [lbm.LBM_MASKED_NODE, lbm.LBM_MASKED_ZRUN])
@pytest.mark.parametrize("dtype,esize,ntype", [(lbm.LBM_F32S, 4, np.float32),
                                               (lbm.LBM_F16S, 2, np.float16)])
def test_solid_slots_rest_fill(mode, dtype, esize, ntype):
    """A solid node whose 32-byte sector holds a fluid node takes the rest
    state (shifted value 0) in every direction after a step, so sectors are
    written whole; other solid slots are never written."""
    nz, ny, nx = shape = (10, 12, 40)
    mask = _mask(shape, solid=0.3, seed=12)
    rho, u = wl.random_state(nx, ny, nz, 3, seed=2, u_amp=0.04, rho_amp=0.01)
    sim = lbm.Simulation(nx, ny, nz, lbm.LBM_D3Q19, lbm.LBM_BGK, 0.7, dtype)
    lbm.lbm_set_masked_kernel(sim.h, mode)
    sim.set_geometry(mask)
    sim.init(rho, u)
    s0, _ = sim.state()
    sim.step(2)                                # the state is back in the first array
    s2, _ = sim.state()
    sim.close()
    nxp = -(-nx // 32) * 32
    sq = -(-(nxp * ny * nz) // 128) * 128
    a0 = s0.view(ntype).reshape(19, sq)[:, :nz * ny * nxp].reshape(19, nz, ny, nxp)[..., :nx]
    a2 = s2.view(ntype).reshape(19, sq)[:, :nz * ny * nxp].reshape(19, nz, ny, nxp)[..., :nx]
    per = 32 // esize
    solid = mask == 1
    grp = np.zeros((nz, ny, nxp), bool)
    grp[..., :nx] = ~solid
    mixed = np.repeat(grp.reshape(nz, ny, nxp // per, per).any(-1), per, axis=-1)[..., :nx]
    fill = solid & mixed
    keep = solid & ~mixed
    assert fill.sum() > 0 and keep.sum() > 0
    assert np.all(a2[:, fill] == 0)
    assert np.array_equal(np.ascontiguousarray(a2[:, keep]).view(np.uint8),
                          np.ascontiguousarray(a0[:, keep]).view(np.uint8))
