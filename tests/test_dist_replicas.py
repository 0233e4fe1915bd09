"""The multi-process (replicas only) plumbing of bench.py on CPU: two gloo
ranks on 127.0.0.1 join, take the slowest rank's time, shard the field-levels
without overlap, and report the whole-job throughput."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_1711_11296_gb300 import workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    r, w, local = bench.dist_env()
    dist = bench.dist_init(w, "gloo")
    try:
        bench.barrier(dist)
        # each rank "took" a different time; the job's time is the maximum
        ms = bench.max_over_ranks(dist, 10.0 + 5.0 * r, "cpu")
        wl = W.WORKLOADS["T31"]
        shard = W.workload_spectrum(wl, F=3, field0=r * 3)
        out[r] = (r, w, local, ms, bench.job_throughput(w, 3, 4, ms), shard)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in (0, 1):
        rank, world, local, ms, thr, _ = res[r]
        assert (rank, world, local) == (r, 2, r)
        assert ms == 15.0                      # the slower rank's time on both
        assert abs(thr - 2 * 3 * 4 / 0.015) < 1e-6
    # the two shards are disjoint columns of the 6-field spectrum
    full = W.workload_spectrum(W.WORKLOADS["T31"], F=6)
    np.testing.assert_array_equal(np.concatenate([res[0][5], res[1][5]], axis=1), full)


def test_single_process_needs_no_group():
    import bench
    assert bench.dist_init(1, "gloo") is None
    assert bench.max_over_ranks(None, 3.5, "cpu") == 3.5
    assert bench.job_throughput(1, 256, 100, 600.0) == 256 * 100 / 0.6
