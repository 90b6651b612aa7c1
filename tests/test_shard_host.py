"""Sharding one sweep across ranks (paper_1812_00394_gb300/shard.py) on CPU gloo ranks.

The per-rank solver here is the FP64 oracle (test infrastructure) behind the interface the
library's batched handle offers, so that the host logic -- the cell-balanced assignment, one
handle per rank for its share, the FP64 combination of statistics and the gather of
per-instance results -- runs without a GPU.  Checks, on 2 and 3 ranks:
  - the assignment is a partition of the instances, balanced to within the largest instance;
  - the union of the ranks' results equals a single process stepping every instance, bitwise
    (fields and forces of every instance);
  - the combined residual is the largest instance residual, the combined mass the total mass
    (to FP64 summation order), and every rank sees the same combined values.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1812_00394_gb300 import meshgen as mg
from paper_1812_00394_gb300.shard import ShardedSweep, assign_instances


def _cases():
    cs = [mg.cavity_quad(n, re=400.0) for n in (6, 9, 12, 7)]
    cs.append(mg.naca0012_cmesh(n_target=700, re_c=1e4, alpha_deg=4.0))
    cs.append(mg.bfs_hybrid(n_target=500))
    cs.append(mg.Case(mg.couette_channel(6, 5, kind="tri", jitter=0.2, seed=2), nu=0.01, cfl=0.5))
    return cs


class _OracleBatch:
    """The batched-handle interface (step with stats, fields, forces) over FP64 oracles."""

    def __init__(self, cases):
        from oracle.oracle import Oracle
        self.cases = list(cases)
        self.o = [Oracle(c) for c in cases]
        self.steps = 0

    def step(self, n, stats=False):
        for o in self.o:
            o.step(n)
        self.steps += n
        if not stats:
            return None
        return {"steps": self.steps, "residual": max(o.residual() for o in self.o),
                "mass": float(sum(o.mass() for o in self.o)), "diverged": 0}

    def fields(self, i):
        return self.o[i].fields()

    def forces(self, i):
        return self.o[i].forces()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sw = ShardedSweep(_cases(), _OracleBatch, dist=dist, device="cpu")
        sw.step(3)
        st = sw.step(2, stats=True)
        out[rank] = {"mine": sw.mine, "stats": st, "forces": sw.gather_forces(),
                     "fields": sw.gather_fields(("rho", "u", "v"))}
    finally:
        dist.destroy_process_group()


def _run(world):
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:  # no fork of a process that may run threads
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
        return dict(out)


def test_assignment_is_a_balanced_partition():
    cells = [c.mesh.n_cells for c in _cases()]
    for world in (1, 2, 3, 5, 9):
        parts = assign_instances(cells, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(cells)))
        loads = [sum(cells[i] for i in p) for p in parts]
        # greedy longest-first: no rank exceeds the mean by more than the largest instance
        assert max(loads) <= sum(cells) / world + max(cells)
    assert assign_instances([5, 5, 5, 5], 2) == [[0, 2], [1, 3]]
    with pytest.raises(ValueError):
        assign_instances(cells, 0)


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_sweep_equals_one_process(world):
    res = _run(world)
    cases = _cases()
    ref = _OracleBatch(cases)
    ref.step(3)
    st = ref.step(2, stats=True)
    mine = sorted(i for r in res.values() for i in r["mine"])
    assert mine == list(range(len(cases)))
    for r in range(world):
        got = res[r]
        assert got["stats"]["residual"] == st["residual"]          # max: exact
        assert got["stats"]["steps"] == 5 and got["stats"]["diverged"] == 0
        assert abs(got["stats"]["mass"] - st["mass"]) <= 1e-14 * st["mass"]
        assert got["stats"] == res[0]["stats"]                      # the same on every rank
        for g, c in enumerate(cases):
            fr = ref.forces(g)
            assert np.array_equal(got["forces"][g], [fr["fx"], fr["fy"], fr["cd"], fr["cl"]])
            fl = ref.fields(g)
            for key in ("rho", "u", "v"):
                assert np.array_equal(got["fields"][g][key], fl[key]), (g, key)


def test_one_rank_needs_no_process_group():
    cases = _cases()[:3]
    sw = ShardedSweep(cases, _OracleBatch)
    assert sw.mine == [0, 1, 2]
    sw.step(2)
    st = sw.step(1, stats=True)
    ref = _OracleBatch(cases)
    ref.step(2)
    assert st == ref.step(1, stats=True)
