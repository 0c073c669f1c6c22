"""Regularized LBGK (Sec. 2.1.1), Smagorinsky LBGK (Sec. 2.1.4) and the
kinetic-energy / enstrophy diagnostics (Sec. 5.2) on the GPU against the FP64
oracle: element-wise fields after several steps on ragged domains with walls
and forcing, the Kida vortex with its FP64 diagnostics, and the AA pattern.
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

OMODEL = {lbm.LBM_REG: oracle.REG, lbm.LBM_SMAG: oracle.SMAG}
# FP64 agrees to rounding; the FP32-arithmetic storages to their resolution
# of the deviations (Sec. 3.7): plain FP32 keeps f itself.
TOL = {lbm.LBM_F64: 1e-11, lbm.LBM_F32S: 1e-5, lbm.LBM_F32: 2e-4, lbm.LBM_F16S: 5e-3,
       lbm.LBM_BF16S: 5e-2}
# largest absolute density error (density units)
RHO_ABS = {lbm.LBM_F64: 1e-13, lbm.LBM_F32S: 1e-7, lbm.LBM_F32: 1e-6, lbm.LBM_F16S: 2e-4,
           lbm.LBM_BF16S: 2e-3}


def _gpu(model, D, dtype, shape, steps, rho, u, mask=None, force=(0, 0, 0), tau=0.6, cs=0.1,
         pattern=lbm.LBM_PATTERN_AB):
    nz, ny, nx = shape
    lat = lbm.LBM_D2Q9 if D == 2 else lbm.LBM_D3Q19
    sim = lbm.Simulation(nx, ny, nz, lat, model, tau, dtype, pattern=pattern)
    if model == lbm.LBM_SMAG:
        lbm.lbm_set_smagorinsky(sim.h, cs)
    if mask is not None:
        sim.set_geometry(mask)
    if any(force):
        sim.set_force(*force)
    sim.init(rho, u)
    sim.step(steps)
    r, v = sim.macro()
    return sim, r, v


def _oracle(model, D, shape, steps, rho, u, mask=None, force=(0, 0, 0), tau=0.6, cs=0.1):
    nz, ny, nx = shape
    p = oracle.make_params(nx, ny, nz, D=D, model=OMODEL[model], tau=tau, force=force,
                           smag_cs=cs)
    F = oracle.init(p, rho, u)
    ro, uo, _, _ = oracle.run(p, F, steps, mask)
    return ro, uo


@pytest.mark.parametrize("model", [lbm.LBM_REG, lbm.LBM_SMAG])
@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("dtype", [lbm.LBM_F64, lbm.LBM_F32S, lbm.LBM_F32, lbm.LBM_F16S,
                                   lbm.LBM_BF16S])
def test_les_models_vs_oracle(model, D, dtype):
    """Ragged domain (x not a multiple of the 32-wide rows), 10 % random
    solid nodes plus a wall plane, body force, strong shear (u 0.08) so the
    Smagorinsky tau_t is far from zero; 12 steps."""
    shape = (1, 37, 75) if D == 2 else (11, 19, 45)
    nz, ny, nx = shape
    rng = np.random.default_rng(40 + D)
    mask = (rng.random(shape) < 0.1).astype(np.uint8)
    mask[:, 0, :] = 1
    rho, u = wl.random_state(nx, ny, nz, D, seed=7 + D, u_amp=0.08, rho_amp=0.01)
    force = (2e-5, -1e-5, 0.0) if D == 2 else (2e-5, -1e-5, 3e-6)
    tau = 0.52
    sim, rg, ug = _gpu(model, D, dtype, shape, 12, rho, u, mask, force, tau, cs=0.15)
    sim.close()
    ro, uo = _oracle(model, D, shape, 12, rho, u, mask, force, tau, cs=0.15)
    fluid = mask == 0
    eu = an.rel_l2(ug[:, fluid], uo[:, fluid])
    e_r, er = an.rho_errors(rg, ro, fluid)
    print(f"model {model} D{D} dtype {dtype}: rel-L2 u {eu:.3e}, rho-1 {e_r:.3e}, "
          f"max |drho| {er:.3e}")
    assert eu < TOL[dtype]
    assert e_r < TOL[dtype] and er < RHO_ABS[dtype]


def test_smagorinsky_cs0_matches_lbgk_oracle():
    shape = (8, 16, 40)
    nz, ny, nx = shape
    rho, u = wl.random_state(nx, ny, nz, 3, seed=3, u_amp=0.05, rho_amp=0.01)
    sim, rg, ug = _gpu(lbm.LBM_SMAG, 3, lbm.LBM_F64, shape, 10, rho, u, tau=0.7, cs=0.0)
    sim.close()
    p = oracle.make_params(nx, ny, nz, D=3, model=oracle.BGK, tau=0.7)
    F = oracle.init(p, rho, u)
    ro, uo, _, _ = oracle.run(p, F, 10)
    assert an.rel_l2(ug, uo) < 1e-12


@pytest.mark.parametrize("model", [lbm.LBM_REG, lbm.LBM_SMAG])
@pytest.mark.parametrize("dtype", [lbm.LBM_F64, lbm.LBM_F32S])
def test_kida_vortex_and_diagnostics(model, dtype):
    """40^3 Kida vortex (u0 0.05, tau 0.5015: Re = N u0 / nu of a few
    hundred), 30 steps.  The GPU's FP64 E and Omega of its own velocity
    field equal the oracle's diagnostics of the same field to rounding;
    the fields match the oracle's run; E(0) = 3 u0^2 / 8."""
    n, u0, tau, T = 40, 0.05, 0.5015, 30
    rho, u = wl.kida(n, u0)
    sim, rg, ug = _gpu(model, 3, dtype, (n, n, n), T, rho, u, tau=tau, cs=0.1)
    E, Om = lbm.lbm_kinetic_energy_enstrophy(sim.h)
    sim.close()
    Eo, Omo = oracle.kinetic_energy_enstrophy(ug)
    assert abs(E - Eo) < 1e-12 * Eo and abs(Om - Omo) < 1e-12 * Omo
    ro, uo = _oracle(model, 3, (n, n, n), T, rho, u, tau=tau, cs=0.1)
    e_r, e_abs = an.rho_errors(rg, ro)
    print(f"Kida model {model} dtype {dtype}: u {an.rel_l2(ug, uo):.2e} rho-1 {e_r:.2e} "
          f"max|drho| {e_abs:.2e}")
    assert an.rel_l2(ug, uo) < TOL[dtype]
    assert e_abs < RHO_ABS[dtype]
    Er, Omr = oracle.kinetic_energy_enstrophy(uo)
    assert abs(E - Er) < 10 * TOL[dtype] * Er and abs(Om - Omr) < 10 * TOL[dtype] * Omr
    E0, _ = oracle.kinetic_energy_enstrophy(u)
    assert abs(E0 - 3 * u0 ** 2 / 8) < 1e-15
    assert E < E0                                  # free decay
    print(f"Kida model {model} dtype {dtype}: E/E0 {E / E0:.6f}, Omega {Om:.6e}")


def test_diagnostics_d2q9_and_errors():
    """The 2-D diagnostics (vorticity z only) against the oracle; a masked
    handle and a handle without output are refused."""
    shape = (1, 24, 36)
    rho, u = wl.random_state(36, 24, 1, 2, seed=5, u_amp=0.05, rho_amp=0.01)
    sim, rg, ug = _gpu(lbm.LBM_BGK, 2, lbm.LBM_F64, shape, 3, rho, u, tau=0.8)
    E, Om = lbm.lbm_kinetic_energy_enstrophy(sim.h)
    sim.close()
    Eo, Omo = oracle.kinetic_energy_enstrophy(ug)
    assert abs(E - Eo) < 1e-13 * Eo and abs(Om - Omo) < 1e-12 * Omo
    sim = lbm.Simulation(36, 24, 1, lbm.LBM_D2Q9, lbm.LBM_BGK, 0.8, lbm.LBM_F32S)
    sim.init(rho, u)
    with pytest.raises(lbm.LBMError):
        lbm.lbm_kinetic_energy_enstrophy(sim.h)      # no output step yet
    sim.close()
    sim = lbm.Simulation(36, 24, 1, lbm.LBM_D2Q9, lbm.LBM_BGK, 0.8, lbm.LBM_F32S)
    sim.set_geometry(wl.channel_mask(36, 24, 1))
    sim.init(rho, u)
    sim.step(1)
    with pytest.raises(lbm.LBMError):
        lbm.lbm_kinetic_energy_enstrophy(sim.h)      # not a periodic domain
    sim.close()


@pytest.mark.parametrize("model", [lbm.LBM_REG, lbm.LBM_SMAG])
@pytest.mark.parametrize("dtype", [lbm.LBM_F32S, lbm.LBM_F16S])
def test_les_aa_equals_ab(model, dtype):
    shape = (9, 13, 37)
    nz, ny, nx = shape
    rng = np.random.default_rng(8)
    mask = (rng.random(shape) < 0.1).astype(np.uint8)
    rho, u = wl.random_state(nx, ny, nz, 3, seed=9, u_amp=0.06, rho_amp=0.01)
    force = (1e-5, 2e-6, -3e-6)
    for steps in (7, 8):
        sa, ra, va = _gpu(model, 3, dtype, shape, steps, rho, u, mask, force, 0.53)
        sa.close()
        sb, rb, vb = _gpu(model, 3, dtype, shape, steps, rho, u, mask, force, 0.53,
                          pattern=lbm.LBM_PATTERN_AA)
        sb.close()
        assert np.array_equal(ra, rb) and np.array_equal(va, vb)
