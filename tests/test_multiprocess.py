"""The multi-process path of bench.py on CPU: two gloo ranks shard the
instances without overlap or gaps and agree on the slowest rank's time."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2606_17971_b300 import workloads as W
    w = W.WORKLOADS["diff3d_128"]
    insts = W.draw_instances(w, count=10)
    mine = bench.shard(insts, rank, world)
    t = bench.max_over_ranks(1.5 + rank, "cpu", world)
    q.put((rank, [i.a for i in mine], t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_instances_and_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from paper_2606_17971_b300 import workloads as W
    allv = [i.a for i in W.draw_instances(W.WORKLOADS["diff3d_128"], count=10)]
    got = res[0][1] + res[1][1]
    assert sorted(got) == sorted(allv) and len(got) == len(allv)
    assert not set(res[0][1]) & set(res[1][1])
    assert res[0][2] == res[1][2] == 2.5
