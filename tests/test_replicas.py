"""The N > 1 path of bench.py on the CPU: two gloo ranks, each timing its own
replica, must agree on the slowest rank's step time (all_reduce MAX) and on
the whole-job throughput (world solves per step); without a process group the
helpers return the local values.  Runs on CPU (no GPU, no NCCL)."""
import multiprocessing as mp
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    from paper_1611_02045_gb300.replicas import dist_env, job_throughput, max_over_ranks
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, loc = dist_env()
        ms = max_over_ranks(times[rank])
        q.put((r, w, loc, ms, job_throughput(ms, w)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_step():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [310.0, 297.5]
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 and o[2] == o[0] for o in out)
    assert all(o[3] == max(times) for o in out)
    assert all(abs(o[4] - 2 * 1000.0 / max(times)) < 1e-12 for o in out)


def test_single_process_helpers_without_a_group(monkeypatch):
    from paper_1611_02045_gb300.replicas import dist_env, job_throughput, max_over_ranks
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert dist_env() == (0, 1, 0)
    assert max_over_ranks(12.5) == 12.5
    assert job_throughput(250.0, 1) == 4.0
