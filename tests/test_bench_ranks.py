"""The multi-process path of bench.py on the CPU: two gloo ranks combine their
timings (max over ranks) and effective samples (sum), and draw disjoint chain
seeds (independent replicas, no collective on the data path)."""
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, w, e = bench.combine_over_ranks(dist, 1.0 + rank, 10.0 - rank, 2.5 * (rank + 1), "cpu")
    out[rank] = (t, w, e, tuple(int(x) for x in bench.replica_seeds(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_like_the_bench():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in (0, 1):
        t, w, e, _ = res[r]
        assert t == 2.0 and w == 10.0 and e == 7.5
    assert not set(res[0][3]) & set(res[1][3])


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_over_ranks(None, 1.5, 2.0, 3.0, "cpu") == (1.5, 2.0, 3.0)
    assert np.array_equal(bench.replica_seeds(0), np.arange(8))


def test_whole_slice_schedule(monkeypatch):
    """--langevin-every n: a Langevin sweep at steps n-1, 2n-1, ...; 0 never
    (the default), 1 always."""
    import bench
    for n, want in ((0, []), (1, list(range(8))), (4, [3, 7]), (3, [2, 5])):
        monkeypatch.setattr(bench, "LANGEVIN_EVERY", n)
        assert [k for k in range(8) if bench.langevin_step(k)] == want
    monkeypatch.setattr(bench, "LANGEVIN_EVERY", 0)
    assert "only" in bench.schedule_text("prior")
