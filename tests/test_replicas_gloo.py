"""The benchmark's multi-process path on CPU (gloo, world size 2): each rank
runs its own replica (weak scaling), the only collectives are the timing
barrier and the max / sum of the timing scalars, and the reference arm runs
on rank 0 alone."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        cpu = torch.device("cpu")
        bench.barrier(world)
        # rank r processed (r + 1) * 1e9 units in (100 + 50 r) ms
        value, ms_max = bench.job_value((rank + 1) * 1e9, 100.0 + 50.0 * rank, world, cpu)
        mx = bench.max_over_ranks(float(rank), world, cpu)
        sm = bench.sum_over_ranks(float(rank + 1), world, cpu)
        bench.barrier(world)
        out.put((rank, value, ms_max, mx, sm))
    finally:
        dist.destroy_process_group()


def test_two_replicas_reduce_timing_scalars_only():
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
    for rank, value, ms_max, mx, sm in res:
        assert ms_max == 150.0                      # the slowest rank's time
        assert value == pytest.approx(3e9 / 0.150)  # all ranks' units / that time
        assert mx == 1.0 and sm == 3.0


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        gpus, steps, warmup = 2, 1, 1
    bench.run_reference(Args())
    assert capsys.readouterr().out == ""
