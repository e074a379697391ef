"""The multi-rank path of bench.py on CPU: two gloo ranks of independent
replicas combine into whole-job figures (slowest rank's time, summed
particle-steps), as the torchrun launch does on GPUs with NCCL."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, e2e_ms, ps, e2e_ps = bench.reduce_over_ranks(10.0 + rank, 20.0 - rank, 1000 * (rank + 1),
                                                     7 * (rank + 1), "cpu")
    out[rank] = (ms, e2e_ms, ps, e2e_ps)
    torch.distributed.barrier()
    torch.distributed.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench():
    mp = torch.multiprocessing.get_context("spawn")
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        procs = [mp.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(2):
            assert out[r] == (11.0, 20.0, 3000, 21)
