"""Out-of-bounds writes, checked with canaries (no sanitizer needed).

The handle's arena is bound inside a larger buffer filled with a canary byte,
and every padding slot of the distribution array (x >= nx in each row, and
the tail of each direction plane) is set to the canary through
lbm_set_state.  No kernel may write there: after odd and even step counts,
with every kernel family (one node, two nodes, z runs, the AA pattern,
masked and unmasked, every storage width), the padding of the state and the
bytes past the arena are still the canary.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1311_2404_gb300 import lbm  # noqa: E402
from paper_1311_2404_gb300 import workloads as wl  # noqa: E402

CANARY = 0xA5
ESIZE = {lbm.LBM_F64: 8, lbm.LBM_F32: 4, lbm.LBM_F32S: 4, lbm.LBM_F16S: 2, lbm.LBM_BF16S: 2}
Q = {lbm.LBM_D2Q9: 9, lbm.LBM_D3Q19: 19, lbm.LBM_D3Q15: 15, lbm.LBM_D3Q27: 27}


def _padding_mask(nx, ny, nz, q, esize):
    """Bytes of the state that belong to no node: x >= nx and plane tails."""
    nxp = -(-nx // 32) * 32
    sq = -(-(nxp * ny * nz) // 128) * 128
    pad = np.ones((q, sq), bool)
    body = np.zeros((nz, ny, nxp), bool)
    body[..., :nx] = True
    pad[:, :nz * ny * nxp] = ~body.reshape(-1)
    return np.repeat(pad.reshape(-1), esize)


CASES = [
    # lattice, model, dtype, (nz, ny, nx), masked, pattern
    (lbm.LBM_D3Q19, lbm.LBM_BGK, lbm.LBM_F32S, (6, 9, 37), False, lbm.LBM_PATTERN_AB),
    (lbm.LBM_D3Q19, lbm.LBM_BGK, lbm.LBM_F16S, (6, 9, 37), False, lbm.LBM_PATTERN_AB),  # odd nx
    (lbm.LBM_D3Q19, lbm.LBM_MRT, lbm.LBM_BF16S, (6, 9, 45), False, lbm.LBM_PATTERN_AB),
    (lbm.LBM_D3Q19, lbm.LBM_MRT, lbm.LBM_F32S, (19, 9, 37), True, lbm.LBM_PATTERN_AB),
    (lbm.LBM_D3Q19, lbm.LBM_BGK, lbm.LBM_F16S, (19, 9, 37), True, lbm.LBM_PATTERN_AB),
    (lbm.LBM_D3Q19, lbm.LBM_BGK, lbm.LBM_F16S, (6, 9, 37), True, lbm.LBM_PATTERN_AB),
    (lbm.LBM_D3Q19, lbm.LBM_BGK, lbm.LBM_F32S, (6, 9, 37), True, lbm.LBM_PATTERN_AA),
    (lbm.LBM_D3Q27, lbm.LBM_SMAG, lbm.LBM_F16S, (5, 7, 33), True, lbm.LBM_PATTERN_AB),
    (lbm.LBM_D2Q9, lbm.LBM_BGK, lbm.LBM_F64, (1, 13, 41), True, lbm.LBM_PATTERN_AB),
    (lbm.LBM_D2Q9, lbm.LBM_BGK, lbm.LBM_F16S, (1, 13, 41), False, lbm.LBM_PATTERN_AA),
]


@pytest.mark.parametrize("case", CASES)
def test_no_writes_outside_the_nodes(case):
    lat, model, dtype, (nz, ny, nx), masked, pattern = case
    D = 2 if lat == lbm.LBM_D2Q9 else 3
    h = lbm.lbm_create(nx, ny, nz, lat, model, 0.7, dtype)
    try:
        lbm.lbm_set_access_pattern(h, pattern)
        nb = lbm.lbm_required_bytes(h)
        buf = torch.full((nb + 65536,), CANARY, dtype=torch.uint8, device="cuda")
        lbm.lbm_bind_memory(h, buf.data_ptr(), nb)   # torch buffers are 256-byte aligned
        if model == lbm.LBM_SMAG:
            lbm.lbm_set_smagorinsky(h, 0.15)
        if masked:
            m = (np.random.default_rng(3).random((nz, ny, nx)) < 0.2).astype(np.uint8)
            m[:, 0, :] = 1
            lbm.lbm_set_geometry(h, m)
        lbm.lbm_set_force(h, 1e-5, 2e-6, 3e-6 if D == 3 else 0.0)
        rho, u = wl.random_state(nx, ny, nz, D, seed=4, u_amp=0.03, rho_amp=0.01)
        lbm.lbm_init_equilibrium(h, rho, u)
        st = np.empty(lbm.lbm_state_bytes(h), dtype=np.uint8)
        t = lbm.lbm_get_state(h, st)
        pad = _padding_mask(nx, ny, nz, Q[lat], ESIZE[dtype])
        assert pad.size == st.size
        st[pad] = CANARY
        lbm.lbm_set_state(h, st, t)
        for steps in (3, 2):                          # the state in either array
            lbm.lbm_step(h, steps)
            lbm.lbm_get_state(h, st)
            assert np.all(st[pad] == CANARY), steps
        lbm.lbm_sync(h)
        tail = buf[nb:].cpu().numpy()
        assert np.all(tail == CANARY)
    finally:
        lbm.lbm_destroy(h)
