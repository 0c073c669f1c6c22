"""The C-ABI library without a GPU: it loads, exports every function that
include/*.h declares, and validates arguments on the host (lbm_create touches
no device memory)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lbm():
    import __graft_entry__ as g
    g.build()
    from paper_1311_2404_gb300 import lbm as m
    return m


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names |= set(re.findall(r"LBM_API\s+[\w\s\*]+?\b(lbm_\w+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lbm):
    decl = _declared()
    assert len(decl) >= 40
    lib = ctypes.CDLL(lbm.LIB_PATH)
    for name in sorted(decl):
        assert hasattr(lib, name), name
    assert decl == set(lbm.exported_symbols())


def test_create_validates_on_host(lbm):
    h = lbm.lbm_create(64, 32, 1, lbm.LBM_D2Q9, lbm.LBM_BGK, 0.8, lbm.LBM_F64)
    try:
        nb = lbm.lbm_required_bytes(h)
        # two FP64 D2Q9 copies of 64x32 (padded plane 2048) at least
        assert nb >= 2 * 9 * 2048 * 8
        assert lbm.lbm_state_bytes(h) == 9 * 2048 * 8
        assert lbm.lbm_launch_count(h) == 0
    finally:
        lbm.lbm_destroy(h)
    bad = [
        (0, 4, 4, lbm.LBM_D3Q19, lbm.LBM_BGK, 0.6, lbm.LBM_F32S),      # size 0
        (4, 4, 2, lbm.LBM_D2Q9, lbm.LBM_BGK, 0.6, lbm.LBM_F32S),       # D2Q9 with nz != 1
        (4, 4, 4, lbm.LBM_D3Q19, lbm.LBM_BGK, 0.5, lbm.LBM_F32S),      # tau = 1/2
        (4, 4, 4, lbm.LBM_D3Q19, lbm.LBM_BGK, float("nan"), lbm.LBM_F32S),
        (4, 4, 1, lbm.LBM_D2Q9, lbm.LBM_MRT, 0.6, lbm.LBM_F32S),       # MRT on D2Q9
        (4, 4, 4, 7, lbm.LBM_BGK, 0.6, lbm.LBM_F32S),                  # unknown lattice
        (4, 4, 4, lbm.LBM_D3Q19, 9, 0.6, lbm.LBM_F32S),                # unknown model
        (4, 4, 4, lbm.LBM_D3Q19, lbm.LBM_BGK, 0.6, 11),                # unknown dtype
        (4096, 4096, 4096, lbm.LBM_D3Q19, lbm.LBM_BGK, 0.6, lbm.LBM_F32S),  # > 2^31 nodes
    ]
    for args in bad:
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_create(*args)
        assert ei.value.code == lbm.LBM_EINVAL, args
        assert lbm.lbm_last_error(None)


def test_setters_validate_on_host(lbm):
    h = lbm.lbm_create(8, 8, 8, lbm.LBM_D3Q19, lbm.LBM_MRT, 0.6, lbm.LBM_F32S)
    try:
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_set_mrt_rates(h, np.ones(18))
        assert ei.value.code == lbm.LBM_EINVAL
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_set_elbm(h, lbm.LBM_ALPHA_NEWTON)       # not an ELBM handle
        assert ei.value.code == lbm.LBM_EINVAL
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_step(h, 1)                               # before init
        assert ei.value.code == lbm.LBM_ESTATE
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_set_force(h, float("inf"), 0, 0)
        assert ei.value.code == lbm.LBM_EINVAL
        lbm.lbm_set_force(h, 1e-5, 0, 0)
        lbm.lbm_set_mrt_rates(h, np.full(19, 1.0 / 0.6))
    finally:
        lbm.lbm_destroy(h)
    h = lbm.lbm_create(8, 8, 1, lbm.LBM_D2Q9, lbm.LBM_ELBM, 0.51, lbm.LBM_F32S)
    try:
        with pytest.raises(lbm.LBMError):
            lbm.lbm_set_force(h, 0, 0, 1e-3)                 # z force on D2Q9
        with pytest.raises(lbm.LBMError):
            lbm.lbm_set_elbm_guard(h, 0, 1e-6)
        lbm.lbm_set_elbm(h, lbm.LBM_ALPHA_SERIES_GUARDED, 1e-12, 20, 1e-3)
        lbm.lbm_set_elbm_guard(h, 2, 1e-6)
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_step(h, 1)
        assert ei.value.code == lbm.LBM_ESTATE
    finally:
        lbm.lbm_destroy(h)


def test_workload_generators_are_seeded():
    from paper_1311_2404_gb300 import workloads as wl
    m1, n1 = wl.duct_with_spheres(64, 32, 32)
    m2, n2 = wl.duct_with_spheres(64, 32, 32)
    assert np.array_equal(m1, m2) and n1 == n2
    assert 0.20 <= m1.mean() < 0.30          # one sphere can overshoot on a small box
    assert m1[:, 0, :].all() and m1[0].all()
    r, u = wl.turbulence(32)
    assert abs(np.sqrt((u * u).sum(0).mean() / 3) - 0.04) < 1e-12
    # solenoidal: spectral divergence vanishes
    k = np.fft.fftfreq(32) * 2 * np.pi
    div = (np.fft.fftn(u[0]) * k[None, None, :] + np.fft.fftn(u[1]) * k[None, :, None] +
           np.fft.fftn(u[2]) * k[:, None, None])
    assert np.abs(div).max() < 1e-10 * np.abs(np.fft.fftn(u[0])).max()
    specs = wl.batch_channel_specs(512)
    assert len(specs) == 512
    assert all(64 <= s["nx"] <= 1024 and 64 <= s["ny"] <= 1024 for s in specs)
    assert all(0.52 <= s["tau"] <= 0.9 for s in specs)
    m = wl.batch_channel_mask(specs[0])
    assert m.shape == (1, specs[0]["ny"], specs[0]["nx"]) and m[0, 0].all()


def test_injected_allocation_failure_on_host(lbm):
    """An allocation failure injected on the host: the call that needs the
    arena returns LBM_ENOMEM (no cudaMalloc is attempted) and the handle
    stays valid."""
    h = lbm.lbm_create(16, 8, 8, lbm.LBM_D3Q19, lbm.LBM_BGK, 0.6, lbm.LBM_F32S)
    try:
        lbm.lbm_debug_fail_allocations(1)
        with pytest.raises(lbm.LBMError) as ei:
            lbm.lbm_set_geometry(h, np.zeros((8, 8, 16), dtype=np.uint8))
        assert ei.value.code == lbm.LBM_ENOMEM
        assert "out of memory" in lbm.lbm_last_error(h)
        assert lbm.lbm_required_bytes(h) > 0
    finally:
        lbm.lbm_debug_fail_allocations(0)
        lbm.lbm_destroy(h)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_debug_fail_allocations(-1)
    assert ei.value.code == lbm.LBM_EINVAL


def test_header_is_plain_c(lbm, tmp_path):
    """The ABI header compiles as C99 (no C++ in the interface) and a C
    program links against the library and calls it."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    lib = os.path.join(root, "paper_1311_2404_gb300", "_lib", "liblbm.so")
    if not os.path.exists(lib):
        pytest.skip("library not built")
    src = tmp_path / "abi.c"
    src.write_text(
        '#include "lbm.h"\n'
        "int main(void) {\n"
        "    lbm_handle h = 0;\n"
        "    if (lbm_create(8, 8, 8, LBM_D3Q19, LBM_BGK, 0.6, LBM_F32S, &h) != LBM_OK) return 1;\n"
        "    if (lbm_required_bytes(h) == 0) return 2;\n"
        "    if (lbm_create(0, 8, 8, LBM_D3Q19, LBM_BGK, 0.6, LBM_F32S, &h) != LBM_EINVAL) return 3;\n"
        "    return lbm_destroy(h);\n"
        "}\n")
    exe = tmp_path / "abi"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(root, "include"), str(src), "-o", str(exe), lib,
                        "-Wl,-rpath," + os.path.dirname(lib)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert subprocess.run([str(exe)]).returncode == 0


def test_python_constants_match_the_header(tmp_path):
    """abi.py (imported by the benchmark's CPU arm, which must load no CUDA
    library) holds the same values as the header's enums: a C program
    compiled against include/lbm.h prints them."""
    import subprocess
    from paper_1311_2404_gb300 import abi
    src = tmp_path / "consts.c"
    src.write_text('#include <stdio.h>\n#include "lbm.h"\nint main(void) {\n' + "".join(
        f'    printf("{n} %d\\n", (int)({n}));\n' for n in abi.NAMES) + "    return 0;\n}\n")
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = dict((k, int(v)) for k, v in (ln.split() for ln in out.splitlines()))
    assert got == {n: getattr(abi, n) for n in abi.NAMES}
    assert len(got) >= 40


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of lbm_mlp_cfg and lbm_train_stats have the C
    structs' sizes and field offsets (a C program compiled against the
    header prints them)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_1311_2404_gb300 import lbm as m
    pairs = (("lbm_mlp_cfg", m.MlpCfg), ("lbm_train_stats", m.TrainStats))
    lines = []
    for cname, cls in pairs:
        lines.append(f'    printf("{cname} sizeof %d\\n", (int)sizeof({cname}));\n')
        for f, _ in cls._fields_:
            lines.append(f'    printf("{cname} {f} %d\\n", (int)offsetof({cname}, {f}));\n')
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbm.h"\n'
                   "int main(void) {\n" + "".join(lines) + "    return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = dict(line.rsplit(" ", 1) for line in
               subprocess.run([str(exe)], capture_output=True, text=True, check=True)
               .stdout.splitlines())
    for cname, cls in pairs:
        assert int(got[f"{cname} sizeof"]) == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got[f"{cname} {f}"]) == getattr(cls, f).offset, (cname, f)


def test_batch_create_validates_on_host(lbm):
    """The batched ensemble is D2Q9 with FP32S / FP16S storage: other
    lattices and storage types are refused before any device work."""
    for lat, dt in ((lbm.LBM_D3Q19, lbm.LBM_F32S), (7, lbm.LBM_F32S), (lbm.LBM_D2Q9, lbm.LBM_F64)):
        with pytest.raises(lbm.LBMError):
            lbm.lbm_batch_create([8], [8], [0.6], dt, lattice=lat)
