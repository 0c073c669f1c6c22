"""The AA access pattern (one distribution array, Sec. 3.3) on the GPU.

AA and AB move the same populations through the same arithmetic, so their
fields must be bitwise equal after any number of steps (odd counts end on a
pull/push step, even counts on an in-place step), with walls, forcing, every
collision model and storage type; checkpoints at odd t resume exactly; the
footprint drops by one distribution array.
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


def _run(pattern, D, model, dtype, shape, steps, mask=None, force=(0, 0, 0), tau=0.7,
         graph=False, elbm_mode=None, seed=31):
    nz, ny, nx = shape
    rho, u = wl.random_state(nx, ny, nz, D, seed=seed, u_amp=0.04, rho_amp=0.01)
    lat = lbm.LBM_D2Q9 if D == 2 else lbm.LBM_D3Q19
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        sim = lbm.Simulation(nx, ny, nz, lat, model, tau, dtype, pattern=pattern)
        if mask is not None:
            sim.set_geometry(mask)
        if any(force):
            sim.set_force(*force)
        if elbm_mode is not None:
            lbm.lbm_set_elbm(sim.h, elbm_mode, 1e-12, 20, 0.0)
        lbm.lbm_set_graph(sim.h, graph)
        sim.init(rho, u)
        sim.step(steps)
        r, v = sim.macro()
        sim.close()
    return r, v, rho, u


@pytest.mark.parametrize("steps", [7, 8])
@pytest.mark.parametrize("D,model,dtype", [
    (3, lbm.LBM_BGK, lbm.LBM_F32S), (3, lbm.LBM_MRT, lbm.LBM_F16S),
    (2, lbm.LBM_BGK, lbm.LBM_F64), (3, lbm.LBM_BGK, lbm.LBM_BF16S),
    (3, lbm.LBM_ELBM, lbm.LBM_F64), (2, lbm.LBM_ELBM, lbm.LBM_F32S)])
def test_aa_equals_ab_bitwise(D, model, dtype, steps):
    shape = (1, 29, 45) if D == 2 else (9, 13, 37)
    rng = np.random.default_rng(4)
    mask = (rng.random(shape) < 0.1).astype(np.uint8)
    mask[:, 0, :] = 1
    force = (1e-5, -2e-6, 0.0) if D == 2 else (1e-5, 2e-6, -3e-6)
    em = lbm.LBM_ALPHA_NEWTON if model == lbm.LBM_ELBM else None
    tau = 0.52 if model == lbm.LBM_ELBM else 0.7
    ra, va, _, _ = _run(lbm.LBM_PATTERN_AB, D, model, dtype, shape, steps, mask, force, tau,
                        elbm_mode=em)
    rb, vb, _, _ = _run(lbm.LBM_PATTERN_AA, D, model, dtype, shape, steps, mask, force, tau,
                        elbm_mode=em)
    assert np.array_equal(ra, rb) and np.array_equal(va, vb)


def test_aa_vs_oracle_and_graph():
    shape = (8, 16, 40)
    mask = wl.channel_mask(40, 16, 8)
    r1, v1, rho, u = _run(lbm.LBM_PATTERN_AA, 3, lbm.LBM_BGK, lbm.LBM_F32S, shape, 25, mask,
                          (1e-5, 0, 0), graph=False)
    r2, v2, _, _ = _run(lbm.LBM_PATTERN_AA, 3, lbm.LBM_BGK, lbm.LBM_F32S, shape, 25, mask,
                        (1e-5, 0, 0), graph=True)
    assert np.array_equal(r1, r2) and np.array_equal(v1, v2)
    nz, ny, nx = shape
    p = oracle.make_params(nx, ny, nz, D=3, model=oracle.BGK, tau=0.7, force=(1e-5, 0, 0))
    F = oracle.init(p, rho, u)
    ro, uo, _, _ = oracle.run(p, F, 25, mask)
    fl = mask == 0
    e_r, e_abs = an.rho_errors(r1, ro, fl)
    print(f"AA FP32S vs oracle: u {an.rel_l2(v1, uo):.2e} rho-1 {e_r:.2e} max|drho| {e_abs:.2e}")
    assert an.rel_l2(v1, uo) < 1e-5 and e_r < 1e-5 and e_abs < 1e-7


def test_aa_checkpoint_at_odd_time_and_footprint():
    nx, ny, nz = 32, 24, 16
    rho, u = wl.random_state(nx, ny, nz, 3, seed=33)
    hab = lbm.lbm_create(nx, ny, nz, lbm.LBM_D3Q19, lbm.LBM_BGK, 0.6, lbm.LBM_F32S)
    bab = lbm.lbm_required_bytes(hab)
    lbm.lbm_destroy(hab)
    sim = lbm.Simulation(nx, ny, nz, lbm.LBM_D3Q19, lbm.LBM_BGK, 0.6, lbm.LBM_F32S,
                         pattern=lbm.LBM_PATTERN_AA)
    baa = lbm.lbm_required_bytes(sim.h)
    assert bab - baa >= lbm.lbm_state_bytes(sim.h)      # one distribution array less
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_set_access_pattern(sim.h, lbm.LBM_PATTERN_AB)   # memory already bound
    assert ei.value.code == lbm.LBM_ESTATE
    sim.init(rho, u)
    sim.step(5)
    buf, t = sim.state()
    assert t == 5
    sim.step(6)
    r1, v1 = sim.macro()
    sim.set_state(buf, t)
    sim.step(6)
    r2, v2 = sim.macro()
    sim.close()
    assert np.array_equal(r1, r2) and np.array_equal(v1, v2)


@pytest.mark.parametrize("lat,model,dtype,nx", [
    (lbm.LBM_D3Q19, lbm.LBM_BGK, lbm.LBM_F16S, 40),
    (lbm.LBM_D3Q19, lbm.LBM_BGK, lbm.LBM_BF16S, 36),
    (lbm.LBM_D3Q19, lbm.LBM_SMAG, lbm.LBM_F16S, 44),
    (lbm.LBM_D3Q27, lbm.LBM_REG, lbm.LBM_BF16S, 40),
    (lbm.LBM_D3Q15, lbm.LBM_BGK, lbm.LBM_F16S, 64),
    (lbm.LBM_D2Q9, lbm.LBM_BGK, lbm.LBM_F16S, 68),
    (lbm.LBM_D3Q19, lbm.LBM_BGK, lbm.LBM_F16S, 43),     # odd nx: a half-empty last pair
    (lbm.LBM_D3Q19, lbm.LBM_MRT, lbm.LBM_F16S, 40)])
def test_unmasked_half_width_kernels_equal_aa_bitwise(lat, model, dtype, nx):
    """Unmasked half-width AB steps take the two-node kernel (pair loads and
    pair stores with stochastic rounding); the AA pattern takes the one-node
    kernel.  Forced, 7 steps, every lattice: fields bitwise equal."""
    D = 2 if lat == lbm.LBM_D2Q9 else 3
    nz, ny = (1, 21) if D == 2 else (6, 11)
    rho, u = wl.random_state(nx, ny, nz, D, seed=9, u_amp=0.04, rho_amp=0.01)
    force = (1e-5, -2e-6, 3e-6 if D == 3 else 0.0)
    out = []
    for pattern in (lbm.LBM_PATTERN_AB, lbm.LBM_PATTERN_AA):
        sim = lbm.Simulation(nx, ny, nz, lat, model, 0.7, dtype, pattern=pattern)
        if model == lbm.LBM_SMAG:
            lbm.lbm_set_smagorinsky(sim.h, 0.15)
        sim.set_force(*force)
        sim.init(rho, u)
        sim.step(7)
        out.append(sim.macro())
        sim.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
