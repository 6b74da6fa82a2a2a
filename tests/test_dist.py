"""The multi-process path on CPU: two gloo ranks, no GPU.

Each rank scores its own slice of one deck's poses (the oracle stands in for
the GPU kernel here); the slices cover every pose once, the gathered result
equals the single-process one, and the timing aggregation takes the slowest
rank.  The benchmark's weak-scaling mode (one deck per rank) uses the same
helpers.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as tdist
import torch.multiprocessing as mp

from paper_2509_21039_gb300 import dist as bdist
from paper_2509_21039_gb300 import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n_poses, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        r, _, w = bdist.world()
        assert (r, w) == (rank, world)
        D = synth.make_deck(5, 6, 120, 8, n_poses)
        lo, hi = bdist.shard_range(n_poses, r, w)
        E = oracle.energies(D, D["poses"][:, lo:hi])
        # gather the slices (a test-side check only: the path itself needs none)
        sizes = [None] * w
        tdist.all_gather_object(sizes, (lo, hi, E.tolist()))
        fake_ms = 10.0 + 5.0 * r
        slowest = bdist.max_over_ranks(fake_ms)
        rate = bdist.aggregate_rate(hi - lo, slowest, w)
        q.put((r, sizes, slowest, rate))
    finally:
        tdist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_gloo_ranks_shard_poses_without_exchange(world):
    n = 37
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle
    D = synth.make_deck(5, 6, 120, 8, n)
    full = oracle.energies(D, D["poses"])
    for r, slices, slowest, rate in out:
        assert slowest == 10.0 + 5.0 * (world - 1)
        got = np.zeros(n)
        seen = np.zeros(n, int)
        for lo, hi, E in slices:
            got[lo:hi] = E
            seen[lo:hi] += 1
        assert np.all(seen == 1)
        np.testing.assert_array_equal(got, full)
        lo, hi = bdist.shard_range(n, r, world)
        assert rate == pytest.approx(world * (hi - lo) / (slowest / 1e3))


def test_shard_range_partitions():
    for n in (0, 1, 5, 64, 65537):
        for w in (1, 2, 3, 8):
            parts = [bdist.shard_range(n, r, w) for r in range(w)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            sizes = [hi - lo for lo, hi in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        bdist.shard_range(5, 2, 2)


def test_single_process_helpers():
    assert bdist.max_over_ranks(3.5) == 3.5
    assert bdist.aggregate_rate(1000, 2.0, 4) == pytest.approx(2e6)
    assert bdist.rank_seed(1, 3) == 4
