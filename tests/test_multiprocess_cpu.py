"""The N-replica benchmark path on CPU with torch.distributed gloo,
world_size 2: max-over-ranks timing and whole-job frames/s, and the
reference arm's behaviour on non-zero ranks."""
import os
import socket
import sys

import torch.multiprocessing as mp

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
    red = bench.make_max_reduce(dist, "cpu")
    fps, ms = bench.replica_rate(100, [10.0, 14.0][rank], world, red)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, fps, ms))


def test_two_gloo_ranks_report_the_slowest_rank():
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
    for rank, fps, ms in out:
        assert abs(ms - 0.14) < 1e-12  # 14 ms / 100 frames on the slower rank
        assert abs(fps - 2 * 100 / 0.014) < 1e-6


def test_reference_arm_is_silent_on_other_ranks(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    bench.run_reference(bench.parse())
    assert capsys.readouterr().out == ""
