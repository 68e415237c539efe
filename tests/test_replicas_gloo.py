"""Replica (data-parallel) host logic of bench.py on two gloo ranks on the CPU: disjoint seeded
slice ranges per rank, the job time as the max over ranks, and the whole-job throughput.  The path
shards over independent slices, so no data-path collective exists to test."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    import synth
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        cfg = synth.CONFIGS[1]
        off = bench.replica_slice_offset(rank, 2)
        d = synth.make_slices(cfg, range(off, off + 2))
        t_local = 10.0 + 5.0 * rank           # this rank's timed region (ms)
        t = bench.max_over_ranks(t_local, dist, torch.device("cpu"))
        v = bench.whole_job_value(2, world, 3, t)
        out[rank] = (off, float(np.abs(d["x_gt"]).sum()), t, v)
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_replicas():
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    (o0, s0, t0, v0), (o1, s1, t1, v1) = out[0], out[1]
    assert (o0, o1) == (0, 2)                 # disjoint, contiguous slice ranges
    assert s0 != s1                           # different seeded phantoms per rank
    assert t0 == t1 == 15.0                   # both ranks see the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 2 * 3 / 15e-3)
