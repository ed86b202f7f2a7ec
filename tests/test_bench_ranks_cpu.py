"""The multi-rank host logic of bench.py on CPU: two gloo ranks, each with
its own replica timing; the job's time is the slowest rank's and the
throughput counts the cells of every rank (weak scaling)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = bench.max_over_ranks(times[rank], "cpu")
        out[rank] = (m, bench.aggregate_glups(1000, 10, m, world))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    times = [2.0, 5.0]
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        m, g = out[r]
        assert m == 5.0
        # 2 ranks x 1000 cells x 10 steps in 5 ms
        assert g == pytest.approx(2 * 1000 * 10 / 5e-3 / 1e9)


def test_one_rank_without_a_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.aggregate_glups(16777216, 1000, 500.0, 1) == pytest.approx(16777216 * 1000 / 0.5 / 1e9)


def test_sequential_server_queueing():
    """The sequential FP32 baseline's latencies at a given rate follow from
    its measured per-request times by first-come-first-served queueing: a
    request starts when it has arrived and the previous one has finished."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    lat, makespan = bench._fifo([0.0, 0.5, 0.6, 5.0], [1.0, 1.0, 0.2, 0.3])
    # starts 0, 1, 2, 5; finishes 1, 2, 2.2, 5.3
    assert lat == pytest.approx([1.0, 1.5, 1.6, 0.3])
    assert makespan == pytest.approx(5.3)
    # arrivals out of order are served in arrival order
    lat2, m2 = bench._fifo([0.6, 0.0, 5.0, 0.5], [0.2, 1.0, 0.3, 1.0])
    assert sorted(lat2) == sorted(lat) and m2 == pytest.approx(makespan)


def test_kernel_fingerprint_ignores_comments_not_code(tmp_path, monkeypatch):
    """The source fingerprint that keeps a committed ncu summary valid
    changes with the kernel's code, not with its comments."""
    import shutil
    import sys
    sys.path.insert(0, ROOT)
    import bench
    src = os.path.join(ROOT, "paper_2208_09267_gb300", "csrc")
    dst = tmp_path / "paper_2208_09267_gb300" / "csrc"
    shutil.copytree(src, dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    p = dst / "step_row.cuh"
    text = p.read_text()
    p.write_text(text.replace("#pragma once", "// a comment\n/* another\n   one */\n#pragma once", 1))
    assert bench.kernel_source_hash() == h0
    p.write_text(text.replace("kMaxTileRows = 8", "kMaxTileRows = 4", 1))
    assert bench.kernel_source_hash() != h0
