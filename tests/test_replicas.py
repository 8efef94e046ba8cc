"""The multi-GPU form of the benchmark is replicas (independent plans per
rank, no collective on the data path): the host logic that turns the ranks'
timings into one whole-job number, run as two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        assert bench._dist() == (ws, rank, rank)
        ms, value = bench._aggregate(times[rank], ws, 3, 180, "cpu")
        out[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ws, times = 2, [1500.0, 1900.0]
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_rank, args=(ws, _free_port(), times, out), nprocs=ws, start_method="spawn")
    assert out[0] == out[1]
    ms, value = out[0]
    assert ms == max(times)
    assert value == pytest.approx(ws * 3 * 180 / (max(times) / 1e3))


def test_single_rank_needs_no_process_group():
    import bench
    ms, value = bench._aggregate(2000.0, 1, 3, 180, "cpu")
    assert ms == 2000.0 and value == pytest.approx(270.0)
