"""The multi-GPU path of the benchmark is replicas only (independent
instances per rank, no collective on the data path); its host logic -- the
max-over-ranks time of the timed region and the whole-job throughput -- is
checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as tdist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank          # rank 1 is the slower replica
    t = bench.reduce_max_ms(ms, device="cpu")
    q.put((rank, t, bench.whole_job_mlups(1_000_000, 100, t, world)))
    tdist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == 15.0
        # 2 replicas x 1e6 cells x 100 steps in 15 ms
        assert v == pytest.approx(2 * 1e6 * 100 / 15e-3 / 1e6)


def test_single_rank_is_unchanged():
    assert bench.reduce_max_ms(7.5) == 7.5
    assert bench.whole_job_mlups(1000, 10, 2.0, 1) == pytest.approx(5.0)
