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


def _best_makespan(costs, m):
    """Brute force over every assignment of the items to m ranks."""
    import itertools
    best = float("inf")
    for assign in itertools.product(range(m), repeat=len(costs)):
        loads = [0.0] * m
        for c, r in zip(costs, assign):
            loads[r] += c
        best = min(best, max(loads))
    return best


def test_lpt_partition_covers_every_deck_once_within_grahams_bound():
    rng = np.random.default_rng(8)
    for trial in range(40):
        n = int(rng.integers(1, 9))
        m = int(rng.integers(1, 4))
        costs = [float(x) for x in rng.integers(1, 100, n)]
        parts = bdist.lpt_partition(costs, m)
        assert len(parts) == m
        assert sorted(i for p in parts for i in p) == list(range(n))
        assert parts == bdist.lpt_partition(costs, m)          # deterministic
        makespan = max(sum(costs[i] for i in p) for p in parts)
        assert makespan <= (4 / 3 - 1 / (3 * m)) * _best_makespan(costs, m) + 1e-9
    # the textbook instance where LPT is off the optimum by exactly Graham's
    # factor: 2 ranks, costs 3, 3, 2, 2, 2 (LPT 7, best 6)
    parts = bdist.lpt_partition([3, 3, 2, 2, 2], 2)
    assert max(sum([3, 3, 2, 2, 2][i] for i in p) for p in parts) == 7
    assert _best_makespan([3, 3, 2, 2, 2], 2) == 6
    # equal costs: counts differ by at most one; more ranks than decks: empty ranks
    parts = bdist.lpt_partition([5.0] * 7, 3)
    assert sorted(len(p) for p in parts) == [2, 2, 3]
    assert bdist.lpt_partition([1.0], 3) == [[0], [], []]
    with pytest.raises(ValueError):
        bdist.lpt_partition([1.0, -1.0], 2)


def test_lpt_partition_of_the_batched_workload():
    # the 64 uneven decks of the batched benchmark, costed by pair count
    shapes = synth.batched_shapes(3, 64)
    costs = [bdist.deck_cost(*s) for s in shapes]
    for m in (2, 4, 8):
        parts = bdist.lpt_partition(costs, m)
        loads = [sum(costs[i] for i in p) for p in parts]
        # greedy list scheduling's bound: total / m + (1 - 1/m) of the largest deck
        assert max(loads) <= sum(costs) / m + (1 - 1 / m) * max(costs)
        assert sorted(i for p in parts for i in p) == list(range(64))


def _lpt_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        decks = [synth.make_deck([6, i], 3 + i, 40 + 15 * i, 8, 5 + 3 * i) for i in range(5)]
        costs = [bdist.deck_cost(len(d["lig_type"]), len(d["pro_type"]), d["poses"].shape[1])
                 for d in decks]
        mine = bdist.lpt_partition(costs, world)[rank]   # every rank computes the same split
        out = {i: oracle.energies(decks[i], decks[i]["poses"]).tolist() for i in mine}
        gathered = [None] * world
        tdist.all_gather_object(gathered, out)           # test-side check only
        q.put((rank, gathered))
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks_split_uneven_decks_by_lpt():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_lpt_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle
    decks = [synth.make_deck([6, i], 3 + i, 40 + 15 * i, 8, 5 + 3 * i) for i in range(5)]
    for _, gathered in out:
        seen = {}
        for part in gathered:
            for i, E in part.items():
                assert i not in seen
                seen[i] = E
        assert sorted(seen) == list(range(5))
        for i, E in seen.items():
            np.testing.assert_array_equal(np.array(E), oracle.energies(decks[i], decks[i]["poses"]))


def test_split_and_partition_balances_the_batched_workload():
    shapes = synth.batched_shapes(3, 64)
    total = sum(bdist.deck_cost(*s) for s in shapes)
    for m in (1, 2, 4, 8, 16):
        work = bdist.split_and_partition(shapes, m)
        assert len(work) == m
        # every pose of every deck exactly once
        seen = {d: np.zeros(s[2], int) for d, s in enumerate(shapes)}
        for part in work:
            for d, lo, hi in part:
                assert 0 <= lo < hi <= shapes[d][2]
                seen[d][lo:hi] += 1
        assert all(np.all(v == 1) for v in seen.values())
        loads = [sum(bdist.deck_cost(shapes[d][0], shapes[d][1], hi - lo) for d, lo, hi in p)
                 for p in work]
        assert sum(loads) == total
        # no piece exceeds the average, so greedy list scheduling stays within
        # (2 - 1/m) of the average load; in practice far closer
        assert max(loads) <= (2 - 1 / m) * total / m + 1e-6
        assert max(loads) <= 1.1 * total / m
    assert bdist.split_and_partition([], 3) == [[], [], []]
    # one deck, several ranks: pose slices of near-equal size
    work = bdist.split_and_partition([(10, 100, 1000)], 4)
    assert sorted(hi - lo for p in work for _, lo, hi in p) == [250, 250, 250, 250]


# --- the bench's shard modes -------------------------------------------------
#
# bench.py --shard {decks,poses,batch} takes each rank's work from
# dist.shard_pieces.  Two gloo ranks drive the same function here, with the
# oracle standing in for the GPU kernel: every pose is evaluated exactly once,
# the pieces' energies equal the single-process ones, the whole-job rate is
# total poses over the slowest rank's time, and nothing but the test's own
# check is exchanged.

def _shard_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        out = {}
        batch = [synth.make_deck([9, i], 2 + i, 20 + 7 * i, 6, 3 + 5 * i) for i in range(6)]
        shapes = [(len(d["lig_type"]), len(d["pro_type"]), d["poses"].shape[1]) for d in batch]
        for mode in bdist.SHARD_MODES:
            pieces, total, scaling = bdist.shard_pieces(mode, rank, world, n_poses=11,
                                                        batch_shapes=shapes)
            res = []
            for d, lo, hi in pieces:
                if mode == "decks":
                    D = synth.make_deck(bdist.rank_seed(1, rank), 3, 30, 6, 11)
                elif mode == "poses":
                    D = synth.make_deck(1, 3, 30, 6, 11)
                else:
                    D = batch[d]
                res.append((d, lo, hi, oracle.energies(D, D["poses"][:, lo:hi]).tolist()))
            fake_ms = 4.0 + rank
            slowest = bdist.max_over_ranks(fake_ms)
            out[mode] = (res, total, scaling, total / (slowest / 1e3))
        gathered = [None] * world
        tdist.all_gather_object(gathered, out)           # test-side check only
        q.put((rank, gathered))
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks_drive_every_shard_mode():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle
    batch = [synth.make_deck([9, i], 2 + i, 20 + 7 * i, 6, 3 + 5 * i) for i in range(6)]
    _, gathered = out[0]
    # decks: each rank all 11 poses of its own deck; weak scaling
    for r in range(world):
        res, total, scaling, rate = gathered[r]["decks"]
        assert scaling == "weak" and total == world * 11
        (d, lo, hi, E), = res
        D = synth.make_deck(bdist.rank_seed(1, r), 3, 30, 6, 11)
        assert (d, lo, hi) == (r, 0, 11)
        np.testing.assert_array_equal(np.array(E), oracle.energies(D, D["poses"]))
        assert rate == pytest.approx(total / (4.0 + world - 1) * 1e3)
    # poses: one deck's poses, each exactly once over the ranks; strong scaling
    D = synth.make_deck(1, 3, 30, 6, 11)
    got, seen = np.zeros(11), np.zeros(11, int)
    for r in range(world):
        res, total, scaling, _ = gathered[r]["poses"]
        assert scaling == "strong" and total == 11
        for d, lo, hi, E in res:
            got[lo:hi] = E
            seen[lo:hi] += 1
    assert np.all(seen == 1)
    np.testing.assert_array_equal(got, oracle.energies(D, D["poses"]))
    # batch: every pose of every deck exactly once; strong scaling
    seen = {i: np.zeros(b["poses"].shape[1], int) for i, b in enumerate(batch)}
    for r in range(world):
        res, total, scaling, _ = gathered[r]["batch"]
        assert scaling == "strong" and total == sum(b["poses"].shape[1] for b in batch)
        for d, lo, hi, E in res:
            seen[d][lo:hi] += 1
            B = batch[d]
            np.testing.assert_array_equal(np.array(E), oracle.energies(B, B["poses"][:, lo:hi]))
    assert all(np.all(v == 1) for v in seen.values())


def test_shard_pieces_rejects_bad_arguments():
    with pytest.raises(ValueError):
        bdist.shard_pieces("rows", 0, 1, n_poses=4)
    with pytest.raises(ValueError):
        bdist.shard_pieces("batch", 0, 2)
    with pytest.raises(ValueError):
        bdist.shard_pieces("poses", 2, 2, n_poses=4)
    assert bdist.shard_pieces("poses", 0, 1, n_poses=4) == ([(0, 0, 4)], 4, "strong")
