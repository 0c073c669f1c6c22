"""The committed profiler records that bench.py reports beside its timings
(CPU): a record holds for the kernel sources it was captured on and for the
workload's node count only, so a changed kernel or another grid size reports
no figure rather than a stale one."""
import json
import os

import pytest

pytest.importorskip("torch")
import bench  # noqa: E402

N256 = 256 ** 3


def test_records_are_current_for_the_benchmark_workloads():
    # the committed records were captured on the committed sources
    assert bench.fp64_inst_for("root", "f32s", N256) is not None
    assert bench.traffic_for("tg256", "f32s", 0, 1, N256) is not None


def test_records_do_not_apply_to_other_sizes():
    assert bench.fp64_inst_for("root", "f32s", 128 ** 3) is None
    assert bench.traffic_for("tg256", "f32s", 0, 1, 128 ** 3) is None


def test_records_do_not_apply_to_changed_sources(tmp_path, monkeypatch):
    # the same records under a copy of the sources with one byte changed
    csrc = os.path.join(bench.ROOT, "paper_1311_2404_gb300", "csrc")
    root = tmp_path
    (root / "profiles").mkdir()
    (root / "paper_1311_2404_gb300" / "csrc").mkdir(parents=True)
    for name in set(bench.KERNEL_SOURCES) | set(bench.ELBM_SOURCES):
        data = open(os.path.join(csrc, name), "rb").read()
        if name == "collide.cuh":
            data += b"\n"
        (root / "paper_1311_2404_gb300" / "csrc" / name).write_bytes(data)
    for name in ("fp64_elbm.json", "traffic.json"):
        with open(os.path.join(bench.ROOT, "profiles", name)) as fh:
            (root / "profiles" / name).write_text(json.dumps(json.load(fh)))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.fp64_inst_for("root", "f32s", N256) is None
    assert bench.traffic_for("tg256", "f32s", 0, 1, N256) is None
