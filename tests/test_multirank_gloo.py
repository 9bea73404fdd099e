"""The multi-rank path on CPU: two gloo ranks (processes) each run a disjoint history range, sum
their exact int64 fixed-point tallies and their event counters with one all_reduce, and take
the max of their run times as the job time, which is how the work shards across GPUs (history
ranges, no collective on the data path; tallies combine exactly and in any order).  The result
must equal one run over the whole range, bit for bit."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2305_07636_gb300 import problems as P

N_PER_RANK = 300
SEED = 21


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = P.config3()
        r = oracle.run(prob, N_PER_RANK, seed=SEED, threads=1, first=rank * N_PER_RANK)
        t = torch.from_numpy(np.ascontiguousarray(r.fixed, dtype=np.int64).ravel())
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        names = sorted(r.counters)
        c = torch.tensor([r.counters[k] for k in names], dtype=torch.int64)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
        dt = torch.tensor([float(rank + 1)], dtype=torch.float64)  # stand-in run times
        dist.all_reduce(dt, op=dist.ReduceOp.MAX)
        if rank == 0:
            np.save(os.path.join(out_dir, "tally.npy"), t.numpy())
            np.save(os.path.join(out_dir, "counters.npy"), c.numpy())
            np.save(os.path.join(out_dir, "time.npy"), dt.numpy())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_to_the_single_run(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    one = oracle.run(P.config3(), 2 * N_PER_RANK, seed=SEED, threads=2)
    tally = np.load(tmp_path / "tally.npy")
    assert np.array_equal(tally, np.ascontiguousarray(one.fixed, dtype=np.int64).ravel())
    names = sorted(one.counters)
    assert np.array_equal(np.load(tmp_path / "counters.npy"), [one.counters[k] for k in names])
    assert np.load(tmp_path / "time.npy")[0] == 2.0
    assert torch.distributed.is_available()
