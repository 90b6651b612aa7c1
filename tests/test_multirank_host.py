"""Host logic of the multi-GPU benchmark path on CPU: two gloo ranks.

Each rank advances its own seeded copy of the sweep (weak scaling, no data exchange); the only
collective is the max over ranks of the timed region.  Here the ranks use the gloo backend and
the oracle-free host pieces of bench.py.
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
        seed = bench.rank_seed(rank)
        seeds = [None] * world
        dist.all_gather_object(seeds, seed)
        cells = bench.sum_over_ranks(torch, dist, world, 1000 + 10 * rank, device="cpu")
        out[rank] = (got, seeds, cells)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_distinct_seeds():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:  # no fork of a process that may run threads
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0            # max over ranks, seen by every rank
    assert len(set(res[0][1])) == world               # every rank its own sweep
    assert res[0][2] == res[1][2] == 2010.0           # cells summed over the ranks' own sweeps


def test_single_rank_is_identity_and_rate():
    assert bench.max_over_ranks(torch, None, 1, 3.5) == 3.5
    # 2000 cells over all ranks, 10 steps in 2 ms -> 10 Mcell-steps/s
    assert abs(bench.aggregate_rate(2000, 10, 2.0) - 10.0) < 1e-12
    assert bench.sum_over_ranks(torch, None, 1, 7.0) == 7.0


@pytest.mark.parametrize("rank", [0, 1, 3])
def test_rank_workloads_differ_but_are_seeded(rank):
    from paper_1812_00394_gb300 import meshgen as mg
    a = mg.batched_sweep(seed=bench.rank_seed(rank), scale=0.02, n_cavity=2, n_bfs=0, n_naca=0)
    b = mg.batched_sweep(seed=bench.rank_seed(rank), scale=0.02, n_cavity=2, n_bfs=0, n_naca=0)
    assert [c.mesh.n_cells for c in a] == [c.mesh.n_cells for c in b]
    assert all((x.mesh.xy == y.mesh.xy).all() for x, y in zip(a, b))


def test_bench_entry_points_exist():
    """Every mode main() dispatches to is defined (the ncu profile mode included)."""
    for name in ("run_ours", "run_reference", "run_profile_mode", "run_adjoint_mode"):
        assert callable(getattr(bench, name)), name


def test_ncu_traffic_lookup_follows_the_kernel_source():
    """roofline.traffic comes from the committed ncu summary only for the default workload and
    only while the recorded hash matches the kernel source; otherwise it is None."""
    assert bench._ncu_traffic("fused_stage2", "cavity64", 1) is None
    assert bench._ncu_traffic("no_such_kernel", "sweep", 1) is None
    got = bench._ncu_traffic("fused_stage2", "sweep", 1)
    assert got is None or got > 1e8
