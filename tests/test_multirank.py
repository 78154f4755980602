"""The N > 1 path of bench.py on the CPU: two ranks over gloo (127.0.0.1).
Every rank decodes its own shard of the workload (weak scaling, no
collective on the data path); the slowest rank's time is taken with one
all-reduce MAX; the whole-job throughput counts every rank's frames.  The
ranks decode their shards with the oracle here (the GPU path is the same
host logic around gfbp_decode)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import oracle as O
    from paper_cs_0605069_gb300 import workload as W
    F = 6
    first = bench.shard_first_frame(rank, F)
    b = W.make_batch("gf4_n96_bsc005", frames=F, first_frame=first)
    r = O.decode(b.code, b.obs, "bsc", b.param, "sus", max_iter=30, threads=1)
    ms = 10.0 * (rank + 1)          # a stand-in for the rank's measured time
    slowest = bench.max_over_ranks(ms, world, "cpu")
    value = bench.job_frames_per_s(F, world, slowest)
    dist.barrier()
    out[rank] = (first, b.obs.copy(), np.asarray(r["iters"]).copy(), slowest, value)
    dist.destroy_process_group()


def test_two_ranks_shard_frames_and_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    (f0, obs0, it0, s0, v0), (f1, obs1, it1, s1, v1) = res[0], res[1]
    assert (f0, f1) == (0, 6)                       # disjoint shards
    assert not np.array_equal(obs0, obs1)           # different frames
    from paper_cs_0605069_gb300 import workload as W
    both = W.make_batch("gf4_n96_bsc005", frames=12)
    np.testing.assert_array_equal(np.concatenate([obs0, obs1]), both.obs)   # the shards tile the workload
    assert s0 == s1 == 20.0                         # max over ranks
    assert v0 == v1 == pytest.approx(12 / 0.020)    # all ranks' frames / slowest time
    assert (it0 >= 1).all() and (it1 >= 1).all()
