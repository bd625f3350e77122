"""Splitting a galaxy catalogue over processes (host only): the native
partition against brute force over every contiguous split, its edge cases,
and a two-rank gloo run of partition -> per-rank work -> host gather."""
import itertools
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def shard():
    from paper_2506_19919_gb300 import build as b
    b.build()
    from paper_2506_19919_gb300 import shard as S
    return S


def _weights(mask, base):
    w = np.array([base + bin(int(m)).count("1") for m in mask], np.int64)
    return np.ones_like(w) if w.sum() == 0 else w


def _best_max_load(w, parts):
    """Smallest possible heaviest block over every split into `parts`
    contiguous (possibly empty) blocks: brute force over the cut positions."""
    n = len(w)
    c = np.concatenate([[0], np.cumsum(w)])
    best = None
    for cuts in itertools.combinations_with_replacement(range(n + 1), parts - 1):
        edges = (0,) + cuts + (n,)
        m = max(c[edges[i + 1]] - c[edges[i]] for i in range(parts))
        best = m if best is None else min(best, m)
    return best


def test_partition_is_optimal_against_brute_force(shard):
    rng = np.random.default_rng(4)
    for _ in range(300):
        n = int(rng.integers(0, 10))
        parts = int(rng.integers(1, 5))
        base = int(rng.integers(0, 4))
        mask = rng.integers(0, 1 << 6, n).astype(np.uint32)
        mask[rng.random(n) < 0.2] = 0
        s = shard.partition_galaxies(mask, parts, base)
        assert s.shape == (parts + 1,) and s[0] == 0 and s[-1] == n
        assert np.all(np.diff(s) >= 0)
        w = _weights(mask, base)
        c = np.concatenate([[0], np.cumsum(w)])
        heaviest = max(c[s[p + 1]] - c[s[p]] for p in range(parts))
        assert heaviest == _best_max_load(w, parts), (mask, base, parts, s)
        sizes = np.diff(s)
        if n >= parts:
            assert np.all(sizes >= 1)                  # nobody idles
        else:
            assert np.all(sizes[:n] == 1) and np.all(sizes[n:] == 0)


def test_partition_balances_a_catalogue(shard):
    """Config-style masks of 3-12 observed bands over 4,096 galaxies split
    eight ways within one galaxy's weight of the ideal share."""
    rng = np.random.default_rng(0)
    nb = rng.integers(3, 13, 4096)
    mask = np.array([(1 << int(k)) - 1 for k in nb], np.uint32)
    for base in (0, 10):
        s = shard.partition_galaxies(mask, 8, base)
        w = nb + base
        loads = [w[s[p]:s[p + 1]].sum() for p in range(8)]
        assert max(loads) - w.sum() / 8 <= w.max()


def test_partition_errors(shard):
    from paper_2506_19919_gb300 import SpsError
    with pytest.raises(SpsError):
        shard.partition_galaxies(np.ones(4, np.uint32), 0)
    with pytest.raises(SpsError):
        shard.partition_galaxies(np.ones(4, np.uint32), 2, base_weight=-1)
    assert list(shard.partition_galaxies(np.zeros(0, np.uint32), 3)) == [0, 0, 0, 0]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(ws), "MASTER_ADDR": "127.0.0.1",
                       "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import sps_workloads as W
    from paper_2506_19919_gb300 import shard as S
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    wl = W.config(3, n_gal=37)                     # the same seeded catalogue on every rank
    a, b = S.block_of(wl.mask, rank, ws, base_weight=10)
    local = np.stack([wl.z[a:b], np.arange(a, b, dtype=np.float64)], axis=1)   # per-galaxy "results"
    full = S.gather_blocks(local)
    out[rank] = (a, b, None if full is None else full.tolist())
    dist.destroy_process_group()


def test_two_ranks_partition_and_gather():
    ws = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(ws, _free_port(), out), nprocs=ws, start_method="spawn", join=True)
    res = dict(out)
    assert res[0][0] == 0 and res[0][1] == res[1][0] and res[1][1] == 37 and res[0][1] > 0
    assert res[1][2] is None
    sys.path.insert(0, ROOT)
    import sps_workloads as W
    wl = W.config(3, n_gal=37)
    full = np.array(res[0][2])
    np.testing.assert_array_equal(full[:, 0], wl.z)            # catalogue order restored
    np.testing.assert_array_equal(full[:, 1], np.arange(37))
