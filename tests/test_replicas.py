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


def _share_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    from paper_1611_02045_gb300.replicas import instance_share, sum_over_ranks
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = instance_share(96, rank, world)
        shares = [None] * world
        dist.all_gather_object(shares, mine)  # host-side gather of small reports, no field data
        totals = sum_over_ranks([len(mine), sum(mine)])
        q.put((rank, mine, shares, totals))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_the_sweep_instances():
    """bench.py --gpus N splits the 96 independent sweep instances by index:
    two gloo ranks get disjoint shares whose union is all 96, and the host-side
    sum of their report counts is the whole batch's."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_share_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=120) for _ in procs), key=lambda o: o[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    a, b = out[0][1], out[1][1]
    assert not set(a) & set(b)
    assert sorted(a + b) == list(range(96))
    assert abs(len(a) - len(b)) <= 1
    assert out[0][2] == out[1][2] == [a, b]
    assert out[0][3] == out[1][3] == [96.0, float(sum(range(96)))]


def test_single_process_helpers_without_a_group(monkeypatch):
    from paper_1611_02045_gb300.replicas import dist_env, job_throughput, max_over_ranks
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert dist_env() == (0, 1, 0)
    assert max_over_ranks(12.5) == 12.5
    assert job_throughput(250.0, 1) == 4.0
    from paper_1611_02045_gb300.replicas import instance_share, sum_over_ranks
    assert instance_share(5, 0, 1) == [0, 1, 2, 3, 4]
    assert instance_share(5, 1, 2) == [1, 3]
    assert sum_over_ranks([1, 2.5]) == [1.0, 2.5]
    with pytest.raises(ValueError):
        instance_share(4, 2, 2)
