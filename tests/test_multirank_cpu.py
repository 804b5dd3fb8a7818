"""The multi-rank aggregation of bench.py on CPU: world_size 2 over gloo
(127.0.0.1), each rank with its own time; the job rate is all ranks' units
over the slowest rank's time."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 10.0 * (rank + 1)             # rank 1 is the slow one
    value, ms = bench.job_throughput(dist, 1.0e9, ms_local, world, device="cpu")
    q.put((rank, value, ms))
    dist.destroy_process_group()


def test_job_throughput_two_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms in res:
        assert ms == pytest.approx(20.0)
        assert value == pytest.approx(2 * 1.0e9 / 0.020)


def test_cpu_baseline_single_and_all_cores():
    """The bench's oracle baseline: a single-thread rate, and every host core running the same bounded
    sample in its own spawned process."""
    import os

    import bench
    from paper_2601_14476_gb300 import inputs

    b = bench.cpu_baseline(inputs.plain_er800(), budget_s=0.2, kind="plain")
    assert b["kind"] == "oracle" and b["cores"] == 1 and b["value"] > 0
    if (os.cpu_count() or 1) > 1:
        assert b["all_cores"]["cores"] == os.cpu_count() and b["all_cores"]["value"] > 0
