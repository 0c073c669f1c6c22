"""Host and device buffers at the ABI boundary: initial fields and readback
through pinned host memory (accessed in place by the kernels), pageable host
memory (staged) and device memory give bitwise identical results."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1311_2404_gb300 import lbm  # noqa: E402
from paper_1311_2404_gb300 import workloads as wl  # noqa: E402


@pytest.mark.parametrize("fdt", [np.float32, np.float64])
def test_pinned_pageable_device_buffers_agree(fdt):
    nx, ny, nz = 45, 17, 11
    rho, u = wl.random_state(nx, ny, nz, 3, seed=21, u_amp=0.05, rho_amp=0.01)
    rho, u = rho.astype(fdt), u.astype(fdt)
    tdt = torch.float32 if fdt == np.float32 else torch.float64
    outs = []
    for kind in ("pageable", "pinned", "device"):
        sim = lbm.Simulation(nx, ny, nz, lbm.LBM_D3Q19, lbm.LBM_BGK, 0.7, lbm.LBM_F32S)
        if kind == "pageable":
            r_in, u_in = rho, u
        elif kind == "pinned":
            r_in = torch.from_numpy(rho.copy()).pin_memory()
            u_in = torch.from_numpy(u.copy()).pin_memory()
        else:
            r_in = torch.from_numpy(rho).cuda()
            u_in = torch.from_numpy(u).cuda()
        lbm.lbm_init_equilibrium(sim.h, r_in, u_in)
        if kind == "pinned":        # the call has returned: the buffers are free again
            r_in.zero_()
            u_in.zero_()
        sim.step(5)
        if kind == "pageable":
            r_out = np.empty(rho.shape, dtype=fdt)
            u_out = np.empty(u.shape, dtype=fdt)
            lbm.lbm_get_macro(sim.h, r_out, u_out)
        else:
            dev = kind == "device"
            r_out = torch.empty(rho.shape, dtype=tdt, device="cuda" if dev else "cpu")
            u_out = torch.empty(u.shape, dtype=tdt, device="cuda" if dev else "cpu")
            if not dev:
                r_out, u_out = r_out.pin_memory(), u_out.pin_memory()
            lbm.lbm_get_macro(sim.h, r_out, u_out)
            r_out, u_out = r_out.cpu().numpy(), u_out.cpu().numpy()
        sim.close()
        outs.append((r_out, u_out))
    for r2, u2 in outs[1:]:
        assert np.array_equal(outs[0][0], r2) and np.array_equal(outs[0][1], u2)
