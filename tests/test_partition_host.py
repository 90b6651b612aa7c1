"""One mesh split into parts with ghost rings (paper_1812_00394_gb300/partition.py), on CPU.

The per-part solver is the FP64 oracle (test infrastructure) behind the interface the library
handle offers for a part (get/set of a cell list, the wall distance, per-edge wall forces), so
that the host logic runs without a GPU.  The whole-mesh oracle is the reference.

Checks:
  - the split: owned sets partition the cells, the ghosts are exactly the cells within the
    given number of face rings, send and receive lists match, every part's mesh passes the
    library's host validation;
  - with 8 ghost rings the owned cells of every part step exactly like the whole mesh (to FP64
    summation order) on SST and laminar meshes, with walls, inlet / outlet, far field and
    periodic faces, and the owned wall edges add up to the whole wall force;
  - the depth is what the step needs: without SST 6 rings are exact and 5 are not; ring by
    ring, the SST update reaches 2 rings and the stages carry the error further;
  - on 2 and 3 gloo ranks (point-to-point ghost exchange, FP64 sums) every rank sees the
    whole-mesh fields, forces, residual and mass.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle.oracle import Oracle
from paper_1812_00394_gb300 import fvlbm, meshgen as mg
from paper_1812_00394_gb300.partition import (DEPTH, LocalPartitionedRun, MeshPartition,
                                              PartitionedRank, adjacency, face_neighbours, rings)


class _OraclePart:
    """A part's solver: the oracle with the handle's cell-list interface."""

    def __init__(self, case):
        self.o = Oracle(case)

    def step(self, n=1, stats=False):
        self.o.step(n)

    def get_cells(self, lids):
        f = self.o.get_f()[lids]
        fl = self.o.fields()
        return f, fl["k"][lids], fl["omega"][lids], fl["nut"][lids]

    def set_cells(self, lids, f, k, w, nt):
        full = self.o.get_f()
        full[lids] = f
        self.o.set_f(full)
        fl = self.o.fields()
        kk, ww, nn = fl["k"].copy(), fl["omega"].copy(), fl["nut"].copy()
        kk[lids], ww[lids], nn[lids] = k, w, nt
        self.o.set_turb(kk, ww, nn)

    def set_wall_distance(self, d):
        self.o.set_wdist(d)

    def fields(self):
        return self.o.fields()

    def get_f(self):
        return self.o.get_f()

    def forces_edges(self):
        fr = self.o.forces(per_edge=True)
        return np.stack([fr["fx_edge"], fr["fy_edge"]], axis=1)


def _perturbed(case, seed):
    """The case with seeded per-cell perturbations of its initial fields, so that every cut
    face sees gradients from the first step on (a uniform start would hide a missing ring)."""
    import dataclasses
    rho, u, v, k, w = case.init_arrays()
    n = rho.shape[0]
    r = [mg.splitmix64_uniform(seed + j, n) for j in range(5)]
    du = 0.02 * case.uref
    return dataclasses.replace(case, rho=rho * (1 + 0.01 * r[0]), u=u + du * r[1], v=v + du * r[2],
                               k=k * (1 + 0.3 * r[3]), omega=w * (1 + 0.3 * r[4]))


def _cases():
    return {
        "naca_sst": _perturbed(mg.naca0012_cmesh(n_target=2500, re_c=1e4, alpha_deg=4.0), 11),
        "bfs_sst": _perturbed(mg.bfs_hybrid(n_target=1500), 12),
        "cavity": _perturbed(mg.cavity_delaunay(h_boundary=1 / 24, n_target=1200, re=400.0, z=5.0,
                                                seed=2), 13),
        "couette_periodic": _perturbed(mg.Case(mg.couette_channel(14, 10, kind="tri", jitter=0.2,
                                                                  seed=4), nu=0.01, cfl=0.5), 14),
    }


def _partition(case, nparts, depth=DEPTH):
    whole = Oracle(case)
    return MeshPartition(case, nparts, depth=depth, dt=whole.dt,
                         wdist=whole.geometry()["wdist"] if case.sst else None), whole


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_split_structure():
    case = _cases()["naca_sst"]
    pt, _ = _partition(case, 3)
    m = case.mesh.normalized()
    pairs, _ = face_neighbours(m)
    ptr, idx = adjacency(m.n_cells, pairs)
    owned = np.concatenate([P.cells[:P.n_owned] for P in pt.parts])
    assert np.array_equal(np.sort(owned), np.arange(m.n_cells))
    assert max(P.n_owned for P in pt.parts) - min(P.n_owned for P in pt.parts) <= 1
    for p, P in enumerate(pt.parts):
        ring = rings(ptr, idx, P.cells[:P.n_owned], DEPTH)
        want = np.nonzero(ring > 0)[0]
        assert np.array_equal(np.sort(P.cells[P.n_owned:]), want)
        assert np.all(np.diff(ring[P.cells[P.n_owned:]]) >= 0)        # ghosts ring by ring
        rc, _, why = fvlbm.check_case(P.case)
        assert rc == 0, why
        for q, lids in P.recv.items():
            Q = pt.parts[q]
            assert np.array_equal(P.cells[lids], Q.cells[Q.send[p]])
            assert np.all(Q.send[p] < Q.n_owned) and np.all(lids >= P.n_owned)
        assert sum(len(v) for v in P.recv.values()) == P.cells.shape[0] - P.n_owned


@pytest.mark.parametrize("name,nparts", [("naca_sst", 3), ("bfs_sst", 2), ("cavity", 3),
                                         ("couette_periodic", 2)])
def test_owned_cells_step_like_the_whole_mesh(name, nparts):
    case = _cases()[name]
    pt, whole = _partition(case, nparts)
    run = LocalPartitionedRun(pt, _OraclePart)
    run.step(6)
    whole.step(6)
    assert _rel(run.get_f(), whole.get_f()) < 1e-12
    fl, fw = run.fields(), whole.fields()
    for key in ("u", "v", "k", "omega", "nut"):
        assert _rel(fl[key] + 1.0, fw[key] + 1.0) < 1e-12, key
    fr, fo = run.forces(), whole.forces()
    for pair in (("fx", "fy"), ("cd", "cl")):  # each to the magnitude of its vector
        scale = max(abs(fo[pair[0]]), abs(fo[pair[1]]), 1e-300)
        for key in pair:
            assert abs(fr[key] - fo[key]) <= 1e-11 * scale, key


def test_laminar_depth_six_is_exact_and_five_is_not():
    """Without SST a step reaches 6 rings (2 per IMEX stage): 6 ghost rings keep the owned cells
    exact over several exchanged steps, 5 do not."""
    case = _cases()["cavity"]
    errs = {}
    for depth in (5, 6):
        pt, whole = _partition(case, 2, depth=depth)
        run = LocalPartitionedRun(pt, _OraclePart)
        run.step(3)
        whole.step(3)
        errs[depth] = _rel(run.get_f(), whole.get_f())
    assert errs[6] < 1e-13 and errs[5] > 1e-10, errs


def test_reach_of_one_step_ring_by_ring():
    """How far the cut faces reach in one step, per ring of part 0 (8 ghost rings, SST): after an
    exchanged step, one more step without the exchange.  The SST update reaches 2 rings: nu_t is
    exact up to ring 6 and wrong on rings 7 and 8.  The stages carry the error further, 2 rings
    per stage: f is wrong on ring 3 and exact on the owned cells (their 8 rings all held exact
    values at the start of the step)."""
    case = _cases()["naca_sst"]
    pt, whole = _partition(case, 2, depth=DEPTH)
    run = LocalPartitionedRun(pt, _OraclePart)
    run.step(1)
    whole.step(1)
    s, P = run.solvers[0], pt.parts[0]
    s.step(1)
    whole.step(1)
    m = case.mesh.normalized()
    pairs, _ = face_neighbours(m)
    ptr, idx = adjacency(m.n_cells, pairs)
    ring = rings(ptr, idx, P.cells[:P.n_owned], DEPTH)[P.cells]
    nut_err = np.abs(s.fields()["nut"] - whole.fields()["nut"][P.cells])
    f_err = np.abs(s.get_f() - whole.get_f()[P.cells]).max(axis=1)
    for r in range(DEPTH - 1):
        assert nut_err[ring == r].max() == 0.0, r
    assert nut_err[ring == DEPTH - 1].max() > 0.0 and nut_err[ring == DEPTH].max() > 0.0
    assert f_err[ring == 0].max() == 0.0
    assert f_err[ring == DEPTH - 5].max() > 1e-12


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        case = _cases()["naca_sst"]
        pt, whole = _partition(case, world)
        area = whole.geometry()["area"]
        r = PartitionedRank(pt, _OraclePart, dist, device="cpu", area=area)
        r.step(4)
        st = r.step(2, stats=True)
        out[rank] = {"stats": st, "f": r.gather_f(), "fields": r.gather_fields(("u", "v")),
                     "forces": r.forces()}
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_exchange_ghosts_and_combine(world):
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
        res = dict(out)
    whole = Oracle(_cases()["naca_sst"])
    whole.step(6)
    f, fo, fw = whole.get_f(), whole.forces(), whole.fields()
    for r in range(world):
        got = res[r]
        assert _rel(got["f"], f) < 1e-12
        assert _rel(got["fields"]["u"], fw["u"]) < 1e-12
        assert abs(got["forces"]["cl"] - fo["cl"]) <= 1e-11 * abs(fo["cl"])
        assert abs(got["stats"]["residual"] - whole.residual()) <= 1e-9 * whole.residual()
        assert abs(got["stats"]["mass"] - whole.mass()) <= 1e-13 * whole.mass()
        assert got["stats"] == res[0]["stats"]
