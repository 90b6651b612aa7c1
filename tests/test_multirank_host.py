"""Host logic of the multi-GPU benchmark path on CPU: two gloo ranks.

The one sweep is split across the ranks by cell count (strong scaling; the instances exchange
nothing inside a step); the collectives are the max over ranks of the timed region and the
sums of per-rank parts of sweep-wide totals.  Here the ranks use the gloo backend and the
oracle-free host pieces of bench.py.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # a rank-dependent "elapsed time": the reported value must be the slowest rank's
        ms = 10.0 + 5.0 * rank
        got = bench.max_over_ranks(torch, dist, world, ms, device="cpu")
        from paper_1812_00394_gb300 import meshgen as mg
        sweep = mg.batched_sweep(seed=5, scale=0.02, n_cavity=4, n_bfs=1, n_naca=1)
        mine = [c.name for c in bench.shard_of(sweep, world, rank)]
        names = [None] * world
        dist.all_gather_object(names, mine)
        cells = bench.sum_over_ranks(torch, dist, world, 1000 + 10 * rank, device="cpu")
        parts = bench.sum_over_ranks(torch, dist, world, [1.0 * rank, 2.0], device="cpu")
        out[rank] = (got, names, cells, list(parts), [c.name for c in sweep])
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_sweep_split():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:  # no fork of a process that may run threads
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0            # max over ranks, seen by every rank
    shares = res[0][1]
    assert shares == res[1][1]                        # every rank computes the same split
    assert sorted(shares[0] + shares[1]) == sorted(res[0][4])  # a partition of the one sweep
    assert not set(shares[0]) & set(shares[1])
    assert res[0][2] == res[1][2] == 2010.0           # sums of per-rank parts
    assert res[0][3] == res[1][3] == [1.0, 4.0]


def test_single_rank_is_identity_and_rate():
    assert bench.max_over_ranks(torch, None, 1, 3.5) == 3.5
    # 2000 cells over all ranks, 10 steps in 2 ms -> 10 Mcell-steps/s
    assert abs(bench.aggregate_rate(2000, 10, 2.0) - 10.0) < 1e-12
    assert bench.sum_over_ranks(torch, None, 1, 7.0) == 7.0


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_sweep_shares_partition_and_balance(world):
    """The full benchmark sweep (48 instances) split over 1-8 ranks: a partition, no rank more
    than the largest instance above the mean."""
    from paper_1812_00394_gb300 import meshgen as mg
    sweep = mg.batched_sweep(seed=5, scale=0.05)
    shares = [bench.shard_of(sweep, world, r) for r in range(world)]
    names = sorted(c.name for sh in shares for c in sh)
    assert names == sorted(c.name for c in sweep)
    loads = [sum(c.mesh.n_cells for c in sh) for sh in shares]
    cells = [c.mesh.n_cells for c in sweep]
    assert max(loads) <= sum(cells) / world + max(cells)
    if world == 1:
        assert [c.name for c in shares[0]] == [c.name for c in sweep]


def test_bench_entry_points_exist():
    """Every mode main() dispatches to is defined (the ncu profile mode included)."""
    for name in ("run_ours", "run_reference", "run_profile_mode", "run_adjoint_mode"):
        assert callable(getattr(bench, name)), name


def test_ncu_traffic_lookup_follows_the_kernel_source():
    """roofline.traffic comes from the committed ncu summary only for the default workload and
    only while the recorded hash matches the kernel source; otherwise it is None."""
    assert bench._ncu_traffic("fused_stage2", "cavity64", 1)[0] is None
    assert bench._ncu_traffic("no_such_kernel", "sweep", 1)[0] is None
    for fv in (False, True):
        got, src = bench._ncu_traffic("fused_stage2", "sweep", 1, fv)
        assert (got is None) or (got > 1e8 and "profiles/" in src), src
