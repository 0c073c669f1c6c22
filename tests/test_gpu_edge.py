"""Degenerate states every kernel must keep exactly (GPU).

Only the slots of fluid nodes are compared: row and plane padding and the
slots of solid nodes outside any fluid node's memory sector are never
written by the kernels and never read.

- Rest: rho = 1, u = 0 and no force is a fixed point of every collision
  (LBGK, MRT, ELBM; Eqs. lbgk, mrt_collision, elbm) and of pull streaming.
  In the shifted storage of Sec. 3.7 every stored deviation f_i - w_i is then
  exactly 0, and stochastic rounding of 0 is 0, so after any number of steps
  every fluid node's slots hold zeros bit for bit and the fields read rho = 1,
  u = 0, on open, masked (one-node and z-run kernels) and batched domains.
  ELBM forms f_i = w_i + d_i in FP64 for its alpha solve, and the FP64
  weights sum to 1 only up to an ulp: its rest state gains about
  alpha beta 1.1e-16 of density a step, which is bounded here.
- All solid: a domain without fluid nodes updates nothing; the fields read
  rho = 0, u = 0 (the solid-node convention) and the stored state is left as
  it was.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1311_2404_gb300 import lbm  # noqa: E402
from paper_1311_2404_gb300 import workloads as wl  # noqa: E402

SHIFTED = [lbm.LBM_F32S, lbm.LBM_F16S, lbm.LBM_BF16S]


def _rest_run(D, model, dtype, shape, mask=None, masked_kernel=None, steps=7):
    nz, ny, nx = shape
    lat = lbm.LBM_D2Q9 if D == 2 else lbm.LBM_D3Q19
    sim = lbm.Simulation(nx, ny, nz, lat, model, 0.6, dtype)
    if masked_kernel is not None:
        lbm.lbm_set_masked_kernel(sim.h, masked_kernel)
    if mask is not None:
        sim.set_geometry(mask)
    sim.init(np.ones((nz, ny, nx)), np.zeros((D, nz, ny, nx)))
    sim.step(steps)
    r, u = sim.macro()
    st, _ = sim.state()
    sim.close()
    st = np.frombuffer(bytes(st), dtype=np.uint8)
    # the slots of the fluid nodes: [q][sq] planes, x padded to 32, planes to
    # 128 elements (the padding is never written)
    nxp = -(-nx // 32) * 32
    q = 19 if D == 3 else 9
    esize = st.size // q // (-(-(nxp * ny * nz) // 128) * 128)
    planes = st.reshape(q, -1)
    fluid = np.ones(shape, bool) if mask is None else mask == 0
    z, y, x = np.nonzero(fluid)
    cols = ((z * ny + y) * nxp + x) * esize
    keep = (cols[:, None] + np.arange(esize)[None, :]).ravel()
    return r, u, np.ascontiguousarray(planes[:, keep])


_EL = {lbm.LBM_F32S: np.float32, lbm.LBM_F16S: np.float16, lbm.LBM_BF16S: None}


def _values(st, dtype):
    """Stored elements as float64 (BF16: the high half of an FP32)."""
    if dtype == lbm.LBM_BF16S:
        bits = st.view(np.uint16).astype(np.uint32) << 16
        return bits.view(np.float32).astype(np.float64)
    return st.view(_EL[dtype]).astype(np.float64)


@pytest.mark.parametrize("dtype", SHIFTED)
@pytest.mark.parametrize("model", [lbm.LBM_BGK, lbm.LBM_MRT])
def test_rest_is_a_fixed_point_open_domain(model, dtype):
    r, u, st = _rest_run(3, model, dtype, (6, 9, 40))
    assert np.all(r == 1.0) and np.all(u == 0.0)
    assert np.all(_values(st, dtype) == 0.0)


@pytest.mark.parametrize("dtype", SHIFTED)
@pytest.mark.parametrize("kernel", [lbm.LBM_MASKED_NODE, lbm.LBM_MASKED_ZRUN])
def test_rest_is_a_fixed_point_masked(kernel, dtype):
    mask, _ = wl.duct_with_spheres(40, 24, 20, seed=7)
    r, u, st = _rest_run(3, lbm.LBM_MRT, dtype, mask.shape, mask, kernel)
    fl = mask == 0
    assert np.all(r[fl] == 1.0) and np.all(r[~fl] == 0.0) and np.all(u == 0.0)
    assert np.all(_values(st, dtype) == 0.0)


def test_rest_is_a_fixed_point_elbm_and_d2q9():
    for dt, steps in ((lbm.LBM_F32S, 7), (lbm.LBM_F64, 20)):
        r, u, _ = _rest_run(3, lbm.LBM_ELBM, dt, (5, 6, 33), steps=steps)
        drift = np.abs(r - 1.0).max()
        print(f"ELBM rest, storage {dt}: |rho - 1| {drift:.2e} after {steps} steps")
        assert drift <= 3e-16 * (steps + 1) and np.abs(u).max() <= 1e-15, dt
    r, u, st = _rest_run(2, lbm.LBM_BGK, lbm.LBM_F16S, (1, 17, 45))
    assert np.all(r == 1.0) and np.all(u == 0.0) and np.all(_values(st, lbm.LBM_F16S) == 0.0)


@pytest.mark.parametrize("dtype", [lbm.LBM_F32S, lbm.LBM_F16S])
def test_rest_is_a_fixed_point_batched(dtype):
    specs = wl.batch_channel_specs(5, nmin=33, nmax=150, seed=3)
    b = lbm.lbm_batch_create([s["nx"] for s in specs], [s["ny"] for s in specs],
                             [s["tau"] for s in specs], dtype)
    for d, s in enumerate(specs):
        lbm.lbm_batch_set_geometry(b, d, wl.batch_channel_mask(s))
        lbm.lbm_batch_init_equilibrium(b, d, np.ones((1, s["ny"], s["nx"])),
                                       np.zeros((2, 1, s["ny"], s["nx"])))
    lbm.lbm_batch_step(b, 9)
    for d, s in enumerate(specs):
        r = np.empty((1, s["ny"], s["nx"]))
        u = np.empty((2, 1, s["ny"], s["nx"]))
        lbm.lbm_batch_get_macro(b, d, r, u)
        fl = wl.batch_channel_mask(s) == 0
        assert np.all(r[fl] == 1.0) and np.all(r[~fl] == 0.0) and np.all(u == 0.0), d
    lbm.lbm_batch_destroy(b)


@pytest.mark.parametrize("dtype", [lbm.LBM_F32S, lbm.LBM_F16S])
@pytest.mark.parametrize("kernel", [lbm.LBM_MASKED_NODE, lbm.LBM_MASKED_ZRUN])
def test_all_solid_domain(kernel, dtype):
    """No fluid node: nothing is updated, the fields read rho = 0, u = 0 and
    the stored state keeps its initial values."""
    nz, ny, nx = shape = (9, 7, 35)
    rho, u = wl.random_state(nx, ny, nz, 3, seed=41)
    sim = lbm.Simulation(nx, ny, nz, lbm.LBM_D3Q19, lbm.LBM_BGK, 0.7, dtype)
    lbm.lbm_set_masked_kernel(sim.h, kernel)
    sim.set_geometry(np.ones(shape, dtype=np.uint8))
    sim.init(rho, u)
    s0, _ = sim.state()
    sim.step(4)
    r, v = sim.macro()
    s4, _ = sim.state()
    sim.close()
    assert np.all(r == 0.0) and np.all(v == 0.0)
    assert bytes(s0) == bytes(s4)
