"""The multi-rank path of the bench on CPU: two gloo ranks (127.0.0.1), one volume per rank, no
collective on the data path; the timing is the max over ranks and the value the whole-job rate."""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank-dependent timings: rank 1 is the slow one on the first entry, rank 0 on the second
        vals = [10.0 + 5.0 * rank, 7.0 - 2.0 * rank]
        red = bench.max_over_ranks(vals, dist, "cpu")
        q.put((rank, red, bench.job_throughput(world, 1_000_000, 4, red[0])))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_max_and_report_the_whole_job():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, red, value in out:
        assert red == [15.0, 7.0]
        # 2 ranks x 1 M voxels x 4 steps in 15 ms
        assert value == pytest.approx(2 * 1_000_000 * 4 / 0.015 / 1e6)


def test_reference_arm_prints_only_on_rank_zero(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup, gpus = 1, 0, 2
    bench.run_reference(A(), bench.WORKLOADS["fault48"])
    assert capsys.readouterr().out == ""
