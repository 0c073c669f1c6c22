"""The N > 1 bench path on CPU: two gloo ranks (127.0.0.1) take the maximum
of their timings, the whole-job throughput counts every rank's updates over
that time, and the reference arm does its work on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.dist_env()
        assert (r, w, lr) == (rank, world, rank)
        vals = bench.max_over_ranks([10.0 + rank, 5.0 - rank], w, "cpu")
        out[rank] = vals
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    assert out[0] == [11.0, 5.0] and out[1] == [11.0, 5.0]
    # 2 ranks x 1e6 nodes x 100 steps in the slowest rank's 11 ms
    assert abs(bench.job_glups(1_000_000, 100, world, 11.0) - 2e8 / 11e-3 / 1e9) < 1e-9


def test_reference_arm_runs_on_rank0_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    import argparse
    ns = argparse.Namespace(workload="tg256", dtype="f32s", size=0, model="", steps=1, warmup=0,
                            impl="reference", gpus=2)
    bench.run_reference(ns)
    assert capsys.readouterr().out == ""


def test_algorithmic_bytes_count_solid_nodes_by_their_geometry_word():
    """A fluid node moves its q values in and out plus its geometry word; a
    solid node only the word (D3Q19 FP32S: 156 B and 4 B)."""
    assert bench.bytes_per_node("f32s", 1) == 152
    assert bench.bytes_per_node("f16s", 0) == 36
    assert bench.algorithmic_bytes(100, 80, 156, 4) == 80 * 156 + 20 * 4
    assert bench.algorithmic_bytes(10, 10, 152, 0) == 1520


def _faces_main(rank, world, port, out):
    """Each rank sends faces tagged with its own number; checks what arrives."""
    from paper_1311_2404_gb300 import slabs
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        nb = 48
        send_up = torch.full((nb,), 10 + rank, dtype=torch.uint8)
        send_down = torch.full((nb,), 100 + rank, dtype=torch.uint8)
        recv_below = torch.zeros(nb, dtype=torch.uint8)
        recv_above = torch.zeros(nb, dtype=torch.uint8)
        for _ in range(3):                      # repeated steps reuse the buffers
            slabs.exchange_faces(send_up, send_down, recv_below, recv_above, rank, world)
        out[rank] = (int(recv_below.min()), int(recv_below.max()),
                     int(recv_above.min()), int(recv_above.max()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [1, 2, 3])
def test_slab_face_exchange_gloo(world):
    """The transport of the slab decomposition across processes: rank r's
    upper face arrives in rank r + 1's lower receive buffer and its lower
    face in rank r - 1's upper one, periodically; with two ranks both faces
    go to the same peer and still land in the right buffers."""
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_faces_main, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        below, above = (r - 1) % world, (r + 1) % world
        assert out[r] == (10 + below, 10 + below, 100 + above, 100 + above), (r, out[r])
