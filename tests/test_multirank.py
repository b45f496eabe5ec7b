"""The N > 1 path of bench.py on CPU: two gloo ranks, each an independent
replica, combined as total units / slowest rank's time (no data-path
collective; only the timing reduction)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms = [120.0, 200.0][rank]      # rank 1 is the slow one
    units = [1.0e9, 3.0e9][rank]   # ranks may process different amounts
    rate, ms_max = bench.whole_job_rate(ms, units)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, rate, ms_max))


def test_two_rank_rate_is_total_units_over_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for _, rate, ms_max in res:
        assert ms_max == 200.0
        assert abs(rate - 4.0e9 / 0.2) < 1e-6 * rate


def test_single_process_rate():
    import bench
    rate, ms = bench.whole_job_rate(50.0, 1.0e9)
    assert ms == 50.0 and abs(rate - 2.0e10) < 1.0
