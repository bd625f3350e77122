"""The benchmark's multi-rank path on CPU: two gloo ranks (one process per
GPU in a real run; the path has no data collective, only the reduction of
the timings and the posterior counts).  Each rank draws its own seeded batch;
the whole-job value is the posteriors of all ranks over the slowest rank's
step time."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "SPS_BENCH_GLOO": "1"})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r = bench._dist()
    wl = bench._hmc_workload(r, n_gal=8)
    post = 10.0 + r                         # posteriors counted on this rank
    ms = 1000.0 * (1 + r)                   # this rank's step time
    value, ms_max = bench.job_value(post, ms, w)
    bench._barrier(w)
    out[r] = (w, float(wl.z[0]), float(wl.extra["theta0_unb"][0, 0]), value, ms_max)
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ws = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(ws, _free_port(), out), nprocs=ws, start_method="spawn", join=True)
    res = dict(out)
    assert sorted(res) == [0, 1]
    assert all(v[0] == ws for v in res.values())
    assert res[0][1] != res[1][1] and res[0][2] != res[1][2]      # per-rank seeded batches
    for v in res.values():                                        # (10 + 11) / (2 s / 60)
        assert v[4] == pytest.approx(2000.0)
        assert v[3] == pytest.approx(21.0 / (2000.0 / 60000.0))


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    v, ms = bench.job_value(5.0, 3000.0, 1)
    assert ms == 3000.0 and v == pytest.approx(5.0 / 0.05)
