"""Multi-rank logic of the benchmark on CPU (gloo, world size 2): every rank gets its own view of
the room (weak scaling, no data-path collective) and the timing is the maximum over ranks."""
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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2605_10760_gb300 import scenes as S
    wl = S.workload("room500k", scale=0.01)
    views = bench.rank_views(S, wl, rank, world)
    t = bench.max_over_ranks(10.0 + rank, dist, "cpu")
    cam = wl.cameras[views[0]]
    out.put((rank, views, t, cam.t.tolist(), len(wl.cameras)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_and_max_timing():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, v0, t0, c0, n0), (r1, v1, t1, c1, n1) = res
    assert v0 == [0] and v1 == [1] and n0 == n1 == world
    assert t0 == t1 == 11.0
    assert c0 != c1

