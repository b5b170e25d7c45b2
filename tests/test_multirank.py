"""bench.py's multi-process host logic with two gloo ranks on CPU: frames are
sharded without overlap (weak scaling, no data-path collective), the step
time is the maximum over ranks, and the barrier releases both ranks."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    import bench
    r, w, local = bench.dist_env()
    seeds = bench.frame_seeds(4, r)
    t = bench.max_over_ranks(1.5 * (r + 1), w)
    bench.barrier(w)
    q.put((r, w, local, seeds, t))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, s0, t0), (r1, w1, l1, s1, t1) = out
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert not set(s0) & set(s1) and len(s0) == len(s1) == 4
    assert t0 == t1 == 3.0


def test_single_rank_defaults(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (0, 1, 0)
    assert bench.max_over_ranks(2.5, 1) == 2.5
    bench.barrier(1)
