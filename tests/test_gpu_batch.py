"""Batched ensemble of uneven D2Q9 channels in one persistent launch (GPU).

- every domain equals the same domain run alone through the single-domain
  path, bitwise (same per-node arithmetic, FP32S and FP16S storage);
- sampled domains match the FP64 oracle within 1e-5 (FP32S);
- the autotuner leaves the state untouched and returns a valid configuration;
- graph replay equals direct launches; one launch per lbm_batch_step call;
- a withheld barrier arrival makes the bounded wait run out and the next
  synchronising call report LBM_ETIMEOUT, with the context still usable.
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


def _specs(k=6, seed=99):
    specs = wl.batch_channel_specs(k, nmin=33, nmax=200, seed=seed)
    return specs


def _init_state(spec, seed):
    rho, u = wl.random_state(spec["nx"], spec["ny"], 1, 2, seed=seed, u_amp=0.03, rho_amp=0.01)
    return rho, u


def _make_batch(specs, dtype, stream=None):
    b = lbm.lbm_batch_create([s["nx"] for s in specs], [s["ny"] for s in specs],
                             [s["tau"] for s in specs], dtype)
    if stream is not None:
        lbm.lbm_batch_set_stream(b, stream)
    for d, s in enumerate(specs):
        lbm.lbm_batch_set_geometry(b, d, wl.batch_channel_mask(s))
        lbm.lbm_batch_set_force(b, d, s["gx"], 0.0)
        rho, u = _init_state(s, 100 + d)
        lbm.lbm_batch_init_equilibrium(b, d, rho, u)
    return b


def _batch_fields(b, specs):
    out = []
    for d, s in enumerate(specs):
        r = np.empty((1, s["ny"], s["nx"]))
        u = np.empty((2, 1, s["ny"], s["nx"]))
        lbm.lbm_batch_get_macro(b, d, r, u)
        out.append((r, u))
    return out


@pytest.mark.parametrize("dtype", [lbm.LBM_F32S, lbm.LBM_F16S])
def test_batch_equals_single_domains_bitwise(dtype):
    specs = _specs()
    steps = 25
    s = torch.cuda.Stream()
    b = _make_batch(specs, dtype, s.cuda_stream)
    lbm.lbm_batch_step(b, steps)
    got = _batch_fields(b, specs)
    assert lbm.lbm_batch_launch_count(b) >= 1
    lbm.lbm_batch_destroy(b)
    for d, sp in enumerate(specs):
        sim = lbm.Simulation(sp["nx"], sp["ny"], 1, lbm.LBM_D2Q9, lbm.LBM_BGK, sp["tau"], dtype)
        sim.set_geometry(wl.batch_channel_mask(sp))
        sim.set_force(sp["gx"], 0.0)
        rho, u = _init_state(sp, 100 + d)
        sim.init(rho, u)
        sim.step(steps)
        r, v = sim.macro()
        sim.close()
        assert np.array_equal(r, got[d][0]) and np.array_equal(v, got[d][1]), d


def test_batch_vs_oracle_sampled():
    specs = _specs()
    steps = 30
    b = _make_batch(specs, lbm.LBM_F32S)
    lbm.lbm_batch_step(b, steps)
    got = _batch_fields(b, specs)
    lbm.lbm_batch_destroy(b)
    for d in (0, 3):
        sp = specs[d]
        mask = wl.batch_channel_mask(sp)
        rho, u = _init_state(sp, 100 + d)
        p = oracle.make_params(sp["nx"], sp["ny"], 1, D=2, model=oracle.BGK, tau=sp["tau"],
                               force=(sp["gx"], 0, 0))
        F = oracle.init(p, rho, u)
        ro, uo, _, _ = oracle.run(p, F, steps, mask)
        fl = mask == 0
        e_r, e_abs = an.rho_errors(got[d][0], ro, fl)
        print(f"batch domain {d}: u {an.rel_l2(got[d][1], uo):.2e} rho-1 {e_r:.2e} "
              f"max|drho| {e_abs:.2e}")
        assert an.rel_l2(got[d][1], uo) < 1e-5 and e_r < 1e-5 and e_abs < 1e-7


def test_autotune_keeps_state_and_graph_equals_direct():
    specs = _specs(5, seed=7)
    s = torch.cuda.Stream()
    b1 = _make_batch(specs, lbm.LBM_F32S, s.cuda_stream)
    lbm.lbm_batch_autotune(b1)
    cfg = lbm.lbm_batch_get_config(b1)
    assert cfg[0] in (128, 256, 512) and cfg[1] >= 1 and cfg[2] in (64, 128, 256)
    lbm.lbm_batch_step(b1, 7)
    lbm.lbm_batch_step(b1, 7)
    a = _batch_fields(b1, specs)
    lbm.lbm_batch_destroy(b1)
    b2 = _make_batch(specs, lbm.LBM_F32S)          # legacy stream: direct launches
    lbm.lbm_batch_step(b2, 14)
    c = _batch_fields(b2, specs)
    lbm.lbm_batch_destroy(b2)
    for (r1, u1), (r2, u2) in zip(a, c):
        assert np.array_equal(r1, r2) and np.array_equal(u1, u2)


def test_barrier_timeout_reports_and_context_survives():
    specs = _specs(4, seed=8)
    b = _make_batch(specs, lbm.LBM_F32S)
    lbm.lbm_batch_set_wait_limit(b, 20000)        # a few ms of bounded spinning
    lbm.lbm_batch_inject_missing_arrival(b, 1)
    lbm.lbm_batch_step(b, 3)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_batch_sync(b)
    assert ei.value.code == lbm.LBM_ETIMEOUT
    lbm.lbm_batch_destroy(b)
    # the context is intact: a fresh batch runs normally
    b = _make_batch(specs, lbm.LBM_F32S)
    lbm.lbm_batch_step(b, 3)
    lbm.lbm_batch_sync(b)
    lbm.lbm_batch_destroy(b)
    x = torch.ones(4, device="cuda") * 2
    assert float(x.sum()) == 8.0


def test_batch_errors():
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_batch_create([10, 0], [10, 10], [0.6, 0.6], lbm.LBM_F32S)
    assert ei.value.code == lbm.LBM_EINVAL
    with pytest.raises(lbm.LBMError):
        lbm.lbm_batch_create([10], [10], [0.6], lbm.LBM_F64)
    with pytest.raises(lbm.LBMError):
        lbm.lbm_batch_create([10], [10], [0.6], lbm.LBM_F32S, lattice=lbm.LBM_D3Q19)
    b = lbm.lbm_batch_create([40, 50], [30, 20], [0.6, 0.7], lbm.LBM_F32S)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_batch_step(b, 1)                  # domains not initialised
    assert ei.value.code == lbm.LBM_ESTATE
    lbm.lbm_batch_destroy(b)


def _single(spec, rho, u, steps, dtype):
    sim = lbm.Simulation(spec["nx"], spec["ny"], 1, lbm.LBM_D2Q9, lbm.LBM_BGK, spec["tau"], dtype)
    sim.set_geometry(wl.batch_channel_mask(spec))
    sim.set_force(spec["gx"], 0.0)
    sim.init(rho, u)
    sim.step(steps)
    r, v = sim.macro()
    sim.close()
    return r, v


@pytest.mark.parametrize("t_reinit", [5, 6])
def test_batch_reinit_one_domain_mid_run(t_reinit):
    """Re-initialising domain 1 after t steps (odd and even t: the state is in
    either buffer) restarts that domain only: after 4 more steps it equals a
    fresh single-domain run of 4 steps, and the other domains equal
    uninterrupted runs of t + 4 steps (bitwise)."""
    specs = _specs(3, seed=7)
    b = _make_batch(specs, lbm.LBM_F32S)
    lbm.lbm_batch_step(b, t_reinit)
    rho1, u1 = _init_state(specs[1], 555)
    lbm.lbm_batch_init_equilibrium(b, 1, rho1, u1)
    lbm.lbm_batch_step(b, 4)
    got = _batch_fields(b, specs)
    lbm.lbm_batch_destroy(b)
    r, v = _single(specs[1], rho1, u1, 4, lbm.LBM_F32S)
    assert np.array_equal(got[1][0], r) and np.array_equal(got[1][1], v)
    for d in (0, 2):
        rho, u = _init_state(specs[d], 100 + d)
        r, v = _single(specs[d], rho, u, t_reinit + 4, lbm.LBM_F32S)
        assert np.array_equal(got[d][0], r) and np.array_equal(got[d][1], v)


CONFIGS = [
    # threads, ctas, tile width, tile rows, rows per thread and pass
    (256, 7, 128, 8, 1),
    (64, 1, 32, 3, 1),        # one CTA walks every tile of every domain
    (128, 3, 64, 5, 2),       # tile rows not a multiple of the rows per pass
    (512, 2, 128, 64, 4),
    (96, 5, 32, 1, 4),        # one-row tiles: only the first row of a pass exists
    (256, 11, 256, 16, 2),
    # the staged kernel (bulk copies into double-buffered shared memory)
    (256, 7, 128, 8, 0),
    (64, 1, 32, 3, 0),
    (128, 3, 64, 5, 0),
    (256, 2, 64, 16, 0),
    (96, 5, 32, 1, 0),
    # the register kernel with two x-adjacent nodes per thread
    (128, 3, 64, 5, -1),
    (64, 1, 64, 3, -1),       # one CTA walks every tile of every domain
    (256, 7, 128, 8, -2),
    (512, 2, 128, 64, -2),
    (256, 11, 256, 16, -2),
    (128, 5, 64, 1, -2),      # one-row tiles
]


@pytest.mark.parametrize("dtype", [lbm.LBM_F32S, lbm.LBM_F16S])
def test_every_launch_configuration_gives_the_same_bits(dtype):
    """The persistent kernel walks its tile range arithmetically across
    domain boundaries; every tile shape, CTA count and rows-per-pass
    choice must reproduce the same fields bit for bit."""
    specs = _specs(7, seed=21)
    ref = None
    for cfg in CONFIGS:
        b = _make_batch(specs, dtype)
        lbm.lbm_batch_set_config(b, cfg)
        assert list(lbm.lbm_batch_get_config(b)) == list(cfg)
        lbm.lbm_batch_step(b, 5)
        lbm.lbm_batch_step(b, 4)
        got = _batch_fields(b, specs)
        lbm.lbm_batch_destroy(b)
        if ref is None:
            ref = got
            continue
        for (r1, u1), (r2, u2) in zip(ref, got):
            assert np.array_equal(r1, r2) and np.array_equal(u1, u2), cfg


@pytest.mark.parametrize("hook,cfg", [(1, (256, 4, 128, 8, 0)), (2, (256, 4, 128, 8, 0)),
                                      (2, (64, 1, 32, 2, 0))])
def test_staged_kernel_bounded_waits(hook, cfg):
    """Hook 1: a withheld grid-barrier arrival; hook 2: a stage whose copies
    deliver fewer bytes than it expects.  Either wait runs out, the next
    synchronising call reports LBM_ETIMEOUT, and the context stays usable."""
    specs = _specs(4, seed=23)
    b = _make_batch(specs, lbm.LBM_F32S)
    lbm.lbm_batch_set_config(b, cfg)
    lbm.lbm_batch_set_wait_limit(b, 20000)
    lbm.lbm_batch_inject_missing_arrival(b, hook)
    lbm.lbm_batch_step(b, 3)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_batch_sync(b)
    assert ei.value.code == lbm.LBM_ETIMEOUT
    lbm.lbm_batch_destroy(b)
    b = _make_batch(specs, lbm.LBM_F32S)
    lbm.lbm_batch_set_config(b, cfg)
    lbm.lbm_batch_step(b, 3)
    lbm.lbm_batch_sync(b)
    lbm.lbm_batch_destroy(b)
    x = torch.ones(4, device="cuda") * 2
    assert float(x.sum()) == 8.0


def test_set_config_rejects_bad_values():
    specs = _specs(3, seed=22)
    b = _make_batch(specs, lbm.LBM_F32S)
    before = list(lbm.lbm_batch_get_config(b))
    for bad in [(256, 4, 48, 8, 1), (256, 4, 128, 8, 3), (1024, 4, 128, 8, 1),
                (256, 0, 128, 8, 1), (256, 10 ** 6, 128, 8, 1), (192, 4, 128, 8, 1),
                (256, 4, 128, 0, 1), (512, 4, 256, 32, 0)]:
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_batch_set_config(b, bad)
        assert ei.value.code == lbm.LBM_EINVAL
        assert list(lbm.lbm_batch_get_config(b)) == before
    lbm.lbm_batch_destroy(b)


@pytest.mark.parametrize("dtype", [lbm.LBM_F32S, lbm.LBM_F16S])
def test_host_buffer_kinds_agree(dtype):
    """Initial fields and read-back through pageable (staged), pinned (read
    and written in place by the kernels) and device buffers give the same
    bits, for FP32 and FP64 fields."""
    specs = _specs(4, seed=17)
    results = []
    for kind in ("pageable", "pinned", "device"):
        b = lbm.lbm_batch_create([s["nx"] for s in specs], [s["ny"] for s in specs],
                                 [s["tau"] for s in specs], dtype)
        for d, s in enumerate(specs):
            lbm.lbm_batch_set_geometry(b, d, wl.batch_channel_mask(s))
            lbm.lbm_batch_set_force(b, d, s["gx"], 0.0)
            rho, u = _init_state(s, 100 + d)
            r = torch.from_numpy(np.ascontiguousarray(rho, dtype=np.float32))
            v = torch.from_numpy(np.ascontiguousarray(u, dtype=np.float32))
            if kind == "pinned":
                r, v = r.pin_memory(), v.pin_memory()
            elif kind == "device":
                r, v = r.cuda(), v.cuda()
            lbm.lbm_batch_init_equilibrium(b, d, r, v)
        lbm.lbm_batch_step(b, 6)
        out = []
        for d, s in enumerate(specs):
            for fdt in (torch.float32, torch.float64):
                ro = torch.empty((1, s["ny"], s["nx"]), dtype=fdt)
                uo = torch.empty((2, 1, s["ny"], s["nx"]), dtype=fdt)
                if kind == "pinned":
                    ro, uo = ro.pin_memory(), uo.pin_memory()
                elif kind == "device":
                    ro, uo = ro.cuda(), uo.cuda()
                lbm.lbm_batch_get_macro(b, d, ro, uo)
                out.append((ro.cpu().numpy(), uo.cpu().numpy()))
        lbm.lbm_batch_destroy(b)
        results.append(out)
    for other in results[1:]:
        for (r1, u1), (r2, u2) in zip(results[0], other):
            assert np.array_equal(r1, r2) and np.array_equal(u1, u2)
