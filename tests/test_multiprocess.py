"""The multi-process path of bench.py on CPU: two gloo ranks, each timing its own
independent system (weak scaling, no data-path collective), combine their step
times as the maximum over ranks; the whole-job value is all ranks' chain-steps
over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, ws: int, port: int, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    t_max = bench.slowest_rank_time(times[rank], ws)
    out[rank] = (t_max, bench.job_value(ws, 900, t_max), bench.rank_seed(rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ws, port = 2, _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    times = [0.25, 0.40]
    mp.start_processes(_worker, args=(ws, port, times, out), nprocs=ws, start_method="spawn", join=True)
    assert out[0][0] == out[1][0] == 0.40
    assert out[0][1] == out[1][1] == pytest.approx(2 * 900 / 0.40)
    assert {out[0][2], out[1][2]} == {2, 3}          # every rank runs its own seeded system


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.slowest_rank_time(0.5, 1) == 0.5
    assert bench.job_value(1, 900, 0.5) == 1800.0
