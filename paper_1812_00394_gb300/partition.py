"""One mesh split across ranks: owned cells, ghost rings and a ghost exchange once per step.

Sec. 4 of the paper states only that its code runs in parallel; this is the GB300 form of that
for one large mesh (the sweep of many meshes splits by instance instead, see shard.py).

Dependency depth of one time step (Sec. 3.2, Steps 1-7), in face rings around a cell:
  - the SST update reads the neighbours' limited k / omega gradients, which read theirs:
    2 rings of (u, v, k, omega) and 1 ring of nu_t;
  - each IMEX stage reads the upwind face values of the neighbours, which come from their
    least-squares gradients of f^(J): 2 rings per stage, 6 for the three stages.
So 8 rings of ghost cells around the cells a rank owns make one step of the owned cells exact
when every ghost holds the state (f, k, omega, nu_t) of t^n: the errors that the cut faces
introduce at the outermost ghosts travel inwards by at most 8 rings in one step.  After each
step every rank overwrites its ghosts with the values their owners computed (one exchange per
step, point to point between the ranks that share ghosts).

Each part is an ordinary solver instance over its owned cells (first) and its ghosts (after
them, ring by ring).  The faces that the split cuts become outlet edges of the part's mesh;
what they impose is wrong, but only the outer rings see it.  The time step and the wall
distance are the whole mesh's, passed in (a part sees only its own walls).

Combined results (FP64 on the host, then sums over ranks): fields of the owned cells; the
wall force of the wall edges owned cells carry (each wall edge has exactly one owner); mass;
the residual of the whole mesh from the sums of |u^{n+1} - u^n|^2 and |u^{n+1}|^2.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Sequence

import numpy as np

from . import meshgen as mg

DEPTH = 8  # face rings one time step reaches (2 for the SST update, 2 per IMEX stage)


# ------------------------------------------------------------------ mesh graph
def cell_edges(mesh: mg.Mesh):
    """Every cell edge as (cell, slot, node a, node b), the edge from node slot to slot + 1."""
    ptr = np.asarray(mesh.cell_ptr, np.int64)
    nodes = np.asarray(mesh.cell_nodes, np.int64)
    nv = np.diff(ptr)
    cell = np.repeat(np.arange(mesh.n_cells), nv)
    slot = np.arange(nodes.shape[0]) - np.repeat(ptr[:-1], nv)
    nxt = np.where(slot + 1 < np.repeat(nv, nv), np.arange(nodes.shape[0]) + 1,
                   np.repeat(ptr[:-1], nv))
    return cell, slot, nodes, nodes[nxt]


def _edge_keys(a, b, n_nodes):
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    return lo * np.int64(n_nodes) + hi


def face_neighbours(mesh: mg.Mesh):
    """(pairs [m, 2] of cells sharing an edge, including periodic partners; owner [n_bedges] =
    the cell each boundary edge belongs to)."""
    cell, _, a, b = cell_edges(mesh)
    key = _edge_keys(a, b, mesh.n_nodes)
    order = np.argsort(key, kind="stable")
    ks, cs = key[order], cell[order]
    same = np.nonzero(ks[1:] == ks[:-1])[0]
    pairs = np.stack([cs[same], cs[same + 1]], axis=1)
    bkey = _edge_keys(np.asarray(mesh.bedge_nodes)[:, 0].astype(np.int64),
                      np.asarray(mesh.bedge_nodes)[:, 1].astype(np.int64), mesh.n_nodes)
    pos = np.searchsorted(ks, bkey)
    if np.any(pos >= ks.shape[0]) or np.any(ks[np.minimum(pos, ks.shape[0] - 1)] != bkey):
        raise ValueError("a boundary edge is not an edge of the mesh")
    owner = cs[pos]
    pp = np.asarray(mesh.periodic_pairs, np.int64).reshape(-1, 2)
    if pp.shape[0]:
        pairs = np.concatenate([pairs, np.stack([owner[pp[:, 0]], owner[pp[:, 1]]], axis=1)])
    return pairs, owner


def adjacency(n_cells: int, pairs: np.ndarray):
    """CSR (ptr, idx) of the symmetric cell graph."""
    u = np.concatenate([pairs[:, 0], pairs[:, 1]])
    v = np.concatenate([pairs[:, 1], pairs[:, 0]])
    order = np.lexsort((v, u))
    u, v = u[order], v[order]
    ptr = np.zeros(n_cells + 1, np.int64)
    np.add.at(ptr, u + 1, 1)
    return np.cumsum(ptr), v


def rings(ptr, idx, seeds: np.ndarray, depth: int) -> np.ndarray:
    """Ring number of every cell within `depth` face rings of the seed cells (0 for the seeds;
    -1 beyond)."""
    ring = np.full(ptr.shape[0] - 1, -1, np.int64)
    ring[seeds] = 0
    front = np.asarray(seeds, np.int64)
    for r in range(1, depth + 1):
        if front.size == 0:
            break
        nb = np.concatenate([idx[ptr[c]:ptr[c + 1]] for c in front]) if front.size else front
        nb = np.unique(nb)
        nb = nb[ring[nb] < 0]
        ring[nb] = r
        front = nb
    return ring


def centroids(mesh: mg.Mesh) -> np.ndarray:
    """Mean of each cell's nodes (a point inside the cell, for the split only)."""
    ptr = np.asarray(mesh.cell_ptr, np.int64)
    nodes = np.asarray(mesh.cell_nodes, np.int64)
    nv = np.diff(ptr)
    xy = np.asarray(mesh.xy)[nodes]
    s = np.zeros((mesh.n_cells, 2))
    np.add.at(s, np.repeat(np.arange(mesh.n_cells), nv), xy)
    return s / nv[:, None]


def bisect(points: np.ndarray, nparts: int) -> np.ndarray:
    """Recursive coordinate bisection: part of each point, parts of equal size (+-1), each split
    across the longer side of its box at the matching order statistic (ties by index)."""
    part = np.zeros(points.shape[0], np.int64)

    def split(ids, p0, n):
        if n == 1:
            part[ids] = p0
            return
        nl = n // 2
        box = points[ids].max(axis=0) - points[ids].min(axis=0)
        ax = int(np.argmax(box))
        order = ids[np.lexsort((ids, points[ids, ax]))]
        cut = (ids.shape[0] * nl) // n
        split(order[:cut], p0, nl)
        split(order[cut:], p0 + nl, n - nl)

    split(np.arange(points.shape[0]), 0, nparts)
    return part


# ------------------------------------------------------------------ parts
@dataclasses.dataclass
class Part:
    cells: np.ndarray          # global ids: owned first, then the ghosts ring by ring
    n_owned: int
    case: mg.Case              # the part's mesh (cut faces as outlets) and initial fields
    wdist: np.ndarray          # wall distance of the whole mesh, per local cell
    bedge_global: np.ndarray   # global boundary-edge id of each local boundary edge (-1: cut)
    owned_walls: np.ndarray    # local boundary edges that are walls of owned cells
    recv: dict                 # owner rank -> local ids of the ghosts it sends (global-id order)
    send: dict                 # rank -> local ids of owned cells it needs (its recv order)


def submesh(mesh: mg.Mesh, cells: np.ndarray, owner_of_bedge: np.ndarray, rho0: float):
    """Mesh of the given cells (in that order): used nodes renumbered, node order per cell
    kept; global boundary edges of these cells kept (periodic pairs where both sides are in),
    every other edge that has a side outside becomes an outlet at rho0.  Returns (mesh, global
    boundary-edge id per local boundary edge, -1 for cut edges)."""
    cells = np.asarray(cells, np.int64)
    ptr = np.asarray(mesh.cell_ptr, np.int64)
    nodes = np.asarray(mesh.cell_nodes, np.int64)
    nv = ptr[cells + 1] - ptr[cells]
    gather = np.concatenate([np.arange(ptr[c], ptr[c + 1]) for c in cells])
    used, inv = np.unique(nodes[gather], return_inverse=True)
    sub_ptr = np.concatenate([[0], np.cumsum(nv)]).astype(np.int32)
    sub_nodes = inv.astype(np.int32)
    sub_xy = np.asarray(mesh.xy)[used]
    inside = np.zeros(mesh.n_cells, bool)
    inside[cells] = True
    # local edges and how many local cells share each
    lcell = np.repeat(np.arange(cells.shape[0]), nv)
    slot = np.arange(sub_nodes.shape[0]) - np.repeat(sub_ptr[:-1].astype(np.int64), nv)
    nxt = np.where(slot + 1 < np.repeat(nv, nv), np.arange(sub_nodes.shape[0]) + 1,
                   np.repeat(sub_ptr[:-1].astype(np.int64), nv))
    a, b = sub_nodes.astype(np.int64), sub_nodes[nxt].astype(np.int64)
    key = _edge_keys(used[a], used[b], mesh.n_nodes)        # keys in global node ids
    uk, cnt = np.unique(key, return_counts=True)
    open_keys = uk[cnt == 1]                                  # edges with one local side
    # global boundary edges of local cells (periodic ones only with both partners inside)
    bn = np.asarray(mesh.bedge_nodes, np.int64)
    bkey = _edge_keys(bn[:, 0], bn[:, 1], mesh.n_nodes)
    keep = inside[owner_of_bedge]
    btype = np.asarray(mesh.bedge_type).copy()
    pp = np.asarray(mesh.periodic_pairs, np.int64).reshape(-1, 2)
    ps = np.asarray(mesh.periodic_shift, np.float64).reshape(-1, 2)
    pair_in = keep[pp[:, 0]] & keep[pp[:, 1]] if pp.shape[0] else np.zeros(0, bool)
    for (ea, eb), ok in zip(pp, pair_in):
        if not ok:  # a periodic edge whose partner lies outside is a cut
            btype[ea] = btype[eb] = -1
    kept = np.nonzero(keep & (btype >= 0))[0]
    cut_keys = np.setdiff1d(open_keys, bkey[kept], assume_unique=False)
    # node pairs of the cut edges, in local ids, taken from the local cells' own edges
    first = {}
    for k_, ia, ib in zip(key.tolist(), a.tolist(), b.tolist()):
        first.setdefault(k_, (ia, ib))
    cut_nodes = np.array([first[k_] for k_ in cut_keys.tolist()], np.int64).reshape(-1, 2)
    g2l = np.full(mesh.n_nodes, -1, np.int64)
    g2l[used] = np.arange(used.shape[0])
    bedge_nodes = np.concatenate([g2l[bn[kept]], cut_nodes]).astype(np.int32)
    bedge_type = np.concatenate([np.asarray(mesh.bedge_type)[kept],
                                 np.full(cut_nodes.shape[0], mg.BC_OUTLET)]).astype(np.int32)
    cut_val = np.zeros((cut_nodes.shape[0], 5))
    cut_val[:, 0] = rho0
    cut_val[:, 4] = 1.0
    bedge_val = np.concatenate([np.asarray(mesh.bedge_val, np.float64).reshape(-1, 5)[kept], cut_val])
    bedge_global = np.concatenate([kept, np.full(cut_nodes.shape[0], -1)]).astype(np.int64)
    local_of_edge = np.full(bn.shape[0], -1, np.int64)
    local_of_edge[kept] = np.arange(kept.shape[0])
    sub_pp = np.array([[local_of_edge[ea], local_of_edge[eb]] for (ea, eb), ok in zip(pp, pair_in) if ok],
                      np.int32).reshape(-1, 2)
    sub_ps = ps[pair_in] if pp.shape[0] else np.zeros((0, 2))
    sub = mg.Mesh(xy=sub_xy, cell_ptr=sub_ptr, cell_nodes=sub_nodes, bedge_nodes=bedge_nodes,
                  bedge_type=bedge_type, bedge_val=bedge_val, periodic_pairs=sub_pp,
                  periodic_shift=sub_ps, name=(mesh.name + "/part"))
    return sub, bedge_global


class MeshPartition:
    """The split of one case into `nparts` parts with `depth` ghost rings.

    dt: the whole mesh's time step (required unless the case fixes dt or runs local time
    steps); wdist: the whole mesh's wall distance per cell (required for SST cases).  A caller
    with the library at hand takes both from ``fvlbm.case_geometry`` / ``fvlbm.check_case``.
    """

    def __init__(self, case: mg.Case, nparts: int, depth: int = DEPTH, dt: float | None = None,
                 wdist: np.ndarray | None = None, owner: np.ndarray | None = None):
        if nparts < 1:
            raise ValueError("nparts must be >= 1")
        mesh = case.mesh.normalized()
        nc = mesh.n_cells
        if case.sst and wdist is None:
            raise ValueError("an SST case needs the whole mesh's wall distance")
        if not case.local_dt and case.dt <= 0 and dt is None:
            raise ValueError("the whole mesh's time step is needed (case.dt or dt)")
        self.case, self.mesh, self.nparts, self.depth = case, mesh, nparts, depth
        self.dt = float(case.dt if case.dt > 0 else (dt if dt is not None else 0.0))
        self.wdist = None if wdist is None else np.asarray(wdist, np.float64)
        pairs, self.bedge_owner = face_neighbours(mesh)
        self.ptr, self.idx = adjacency(nc, pairs)
        self.owner = bisect(centroids(mesh), nparts) if owner is None else np.asarray(owner, np.int64)
        init = case.init_arrays()
        self.parts: list[Part] = []
        for p in range(nparts):
            own = np.nonzero(self.owner == p)[0]
            ring = rings(self.ptr, self.idx, own, depth)
            ghosts = np.nonzero(ring > 0)[0]
            ghosts = ghosts[np.lexsort((ghosts, ring[ghosts]))]
            cells = np.concatenate([own, ghosts])
            sub, bglob = submesh(mesh, cells, self.bedge_owner, case.rho0)
            rho, u, v, k, w = (a[cells] for a in init)
            sub_case = dataclasses.replace(case, mesh=sub, dt=self.dt if not case.local_dt else case.dt,
                                           rho=rho, u=u, v=v, k=k, omega=w,
                                           name=f"{case.name}/part{p}")
            local = np.full(nc, -1, np.int64)
            local[cells] = np.arange(cells.shape[0])
            walls = np.nonzero((bglob >= 0) & (np.asarray(sub.bedge_type) == mg.BC_WALL))[0]
            owned_walls = walls[self.owner[self.bedge_owner[bglob[walls]]] == p]
            recv = {}
            for q in np.unique(self.owner[ghosts]).tolist():
                g = np.sort(ghosts[self.owner[ghosts] == q])
                recv[int(q)] = local[g]
            wd = None if self.wdist is None else self.wdist[cells]
            self.parts.append(Part(cells=cells, n_owned=own.shape[0], case=sub_case, wdist=wd,
                                   bedge_global=bglob, owned_walls=owned_walls, recv=recv, send={}))
        # send lists: rank q sends to p the owned cells p's recv[q] holds, in the same order
        for p, P in enumerate(self.parts):
            for q, lids in P.recv.items():
                g = P.cells[lids]
                Q = self.parts[q]
                lq = np.full(nc, -1, np.int64)
                lq[Q.cells[:Q.n_owned]] = np.arange(Q.n_owned)
                Q.send[p] = lq[g]
        self.area = None

    def neighbours(self, p: int) -> list[int]:
        P = self.parts[p]
        return sorted(set(P.recv) | set(P.send))


# ------------------------------------------------------------------ runs
def _pack(solver, lids):
    f, k, w, nt = solver.get_cells(lids)
    return np.concatenate([f, k[:, None], w[:, None], nt[:, None]], axis=1)


def _unpack(solver, lids, data):
    solver.set_cells(lids, data[:, :9], data[:, 9], data[:, 10], data[:, 11])


class _Combine:
    """Owned-cell results of one part and their sums over parts."""

    def __init__(self, partition: MeshPartition, area: np.ndarray | None):
        self.pt = partition
        self.area = area

    def wall_force(self, p, solver):
        P = self.pt.parts[p]
        fxy = solver.forces_edges()
        return fxy[P.owned_walls].sum(axis=0)

    def coefficients(self, fx, fy):
        c = self.pt.case
        q = 0.5 * c.rho0 * c.uref * c.uref
        al = np.radians(c.alpha_deg)
        return {"fx": fx, "fy": fy,
                "cd": (fx * np.cos(al) + fy * np.sin(al)) / (q * c.lref),
                "cl": (-fx * np.sin(al) + fy * np.cos(al)) / (q * c.lref)}


XROW = 12  # doubles per cell in a ghost row: f (9), k, omega, nu_t


class LocalPartitionedRun:
    """Every part in this process (one handle each, e.g. on one GPU); the ghost exchange is a
    copy between the handles after each step: through host arrays, or with device_buffers=True
    through one device buffer per (owner, receiver) pair that the handles pack and unpack with
    their own kernels (the form a run on several GPUs moves with NCCL)."""

    def __init__(self, partition: MeshPartition, make_solver: Callable, device_buffers: bool = False):
        self.pt = partition
        self.solvers = [make_solver(P.case) for P in partition.parts]
        for P, s in zip(partition.parts, self.solvers):
            if P.wdist is not None:
                s.set_wall_distance(P.wdist)
        self.dev = None
        if device_buffers:
            import torch
            self.dev = {}
            for q, Q in enumerate(partition.parts):
                for p, lids in Q.send.items():
                    send_id = self.solvers[q].set_exchange_list(lids)
                    recv_id = self.solvers[p].set_exchange_list(partition.parts[p].recv[q])
                    buf = torch.empty((lids.shape[0], XROW), dtype=torch.float64, device="cuda")
                    self.dev[(q, p)] = (send_id, recv_id, buf)

    def exchange(self):
        if self.dev is not None:
            import torch
            for (q, p), (sid, _, buf) in self.dev.items():
                self.solvers[q].pack_cells_dev(sid, buf.data_ptr())
            torch.cuda.synchronize()  # the packs ran on the owners' streams
            for (q, p), (_, rid, buf) in self.dev.items():
                self.solvers[p].unpack_cells_dev(rid, buf.data_ptr())
            torch.cuda.synchronize()  # the buffers are reused by the next exchange
            return
        out = {}
        for q, Q in enumerate(self.pt.parts):
            for p, lids in Q.send.items():
                out[(q, p)] = _pack(self.solvers[q], lids)
        for (q, p), data in out.items():
            _unpack(self.solvers[p], self.pt.parts[p].recv[q], data)

    def step(self, n: int = 1):
        for _ in range(n):
            for s in self.solvers:
                s.step(1)
            self.exchange()

    def fields(self) -> dict:
        """Fields of every cell of the whole mesh (from their owners)."""
        nc = self.pt.mesh.n_cells
        out = {}
        for P, s in zip(self.pt.parts, self.solvers):
            fl = s.fields()
            for key, val in fl.items():
                out.setdefault(key, np.zeros(nc))[P.cells[:P.n_owned]] = np.asarray(val)[:P.n_owned]
        return out

    def get_f(self) -> np.ndarray:
        f = np.zeros((self.pt.mesh.n_cells, 9))
        for P, s in zip(self.pt.parts, self.solvers):
            f[P.cells[:P.n_owned]] = s.get_f()[:P.n_owned]
        return f

    def forces(self) -> dict:
        cb = _Combine(self.pt, None)
        fx = fy = 0.0
        for p, s in enumerate(self.solvers):
            a = cb.wall_force(p, s)
            fx += float(a[0])
            fy += float(a[1])
        return cb.coefficients(fx, fy)

    def close(self):
        for s in self.solvers:
            if hasattr(s, "close"):
                s.close()
        self.solvers = []


class PartitionedRank:
    """One rank's part under ``torch.distributed`` (NCCL between GPUs, gloo on CPU): the ghost
    exchange posts every receive, then every send, to the ranks it shares ghosts with, and
    waits for all of them."""

    def __init__(self, partition: MeshPartition, make_solver: Callable, dist, device: str = "cpu",
                 area: np.ndarray | None = None):
        self.pt, self.dist, self.device = partition, dist, device
        self.rank = dist.get_rank() if dist is not None else 0
        if dist is not None and dist.get_world_size() != partition.nparts:
            raise ValueError("one rank per part")
        self.part = partition.parts[self.rank]
        self.solver = make_solver(self.part.case)
        if self.part.wdist is not None:
            self.solver.set_wall_distance(self.part.wdist)
        self.area = area

    def _t(self, a):
        import torch
        return torch.as_tensor(np.ascontiguousarray(a, np.float64), device=self.device)

    def _device_lists(self):
        """On a GPU with a handle that packs on the device: the exchange lists registered once,
        one device buffer per peer; the rows then go from kernel to NCCL to kernel."""
        import torch
        P = self.part
        self._dsend = {p: (self.solver.set_exchange_list(l),
                           torch.empty((l.shape[0], XROW), dtype=torch.float64, device=self.device))
                       for p, l in sorted(P.send.items())}
        self._drecv = {q: (self.solver.set_exchange_list(l),
                           torch.empty((l.shape[0], XROW), dtype=torch.float64, device=self.device))
                       for q, l in sorted(P.recv.items())}

    def exchange(self):
        if self.dist is None:
            return
        import torch
        P = self.part
        on_device = str(self.device).startswith("cuda") and hasattr(self.solver, "pack_cells_dev")
        if on_device:
            if not hasattr(self, "_dsend"):
                self._device_lists()
            for p, (lid, buf) in self._dsend.items():
                self.solver.pack_cells_dev(lid, buf.data_ptr())
            torch.cuda.synchronize()  # the packs ran on the handle's stream
            reqs = [self.dist.irecv(buf, src=q) for q, (_, buf) in self._drecv.items()]
            reqs += [self.dist.isend(buf, dst=p) for p, (_, buf) in self._dsend.items()]
            for r in reqs:
                r.wait()
            torch.cuda.synchronize()  # the transfers ran on torch's stream
            for q, (lid, buf) in self._drecv.items():
                self.solver.unpack_cells_dev(lid, buf.data_ptr())
            return
        reqs, bufs = [], {}
        for q, lids in sorted(P.recv.items()):
            bufs[q] = torch.empty((lids.shape[0], XROW), dtype=torch.float64, device=self.device)
            reqs.append(self.dist.irecv(bufs[q], src=q))
        sends = []
        for p, lids in sorted(P.send.items()):
            sends.append(self._t(_pack(self.solver, lids)))
            reqs.append(self.dist.isend(sends[-1], dst=p))
        for r in reqs:
            r.wait()
        for q, lids in sorted(P.recv.items()):
            _unpack(self.solver, lids, bufs[q].cpu().numpy())

    def _allreduce(self, a):
        if self.dist is None:
            return np.asarray(a, np.float64)
        t = self._t(a).clone()
        self.dist.all_reduce(t)
        return t.cpu().numpy()

    def step(self, n: int = 1, stats: bool = False):
        """n steps of the whole mesh; with stats the combined FP64 residual of the last step and
        the mass (needs ``area``, the whole mesh's cell areas)."""
        P = self.part
        uo = None
        for k in range(n):
            if stats and k == n - 1:
                fl = self.solver.fields()
                uo = (np.asarray(fl["u"])[:P.n_owned], np.asarray(fl["v"])[:P.n_owned])
            self.solver.step(1)
            self.exchange()
        if not stats:
            return None
        fl = self.solver.fields()
        u, v = np.asarray(fl["u"])[:P.n_owned], np.asarray(fl["v"])[:P.n_owned]
        rho = np.asarray(fl["rho"])[:P.n_owned]
        num = float(np.sum((u - uo[0]) ** 2 + (v - uo[1]) ** 2)) if uo is not None else 0.0
        den = float(np.sum(u * u + v * v))
        mass = float(np.sum(rho * self.area[P.cells[:P.n_owned]])) if self.area is not None else 0.0
        bad = float(not np.all(np.isfinite(u) & np.isfinite(v) & np.isfinite(rho)))
        s = self._allreduce([num, den, mass, bad])
        res = float(np.sqrt(s[0]) / np.sqrt(s[1])) if s[1] > 0 else float(np.sqrt(s[0]))
        return {"residual": res, "mass": float(s[2]), "diverged": int(s[3] > 0)}

    def gather_fields(self, keys: Sequence[str] = ("rho", "u", "v")) -> dict:
        """Fields of every cell of the whole mesh on every rank (owned values, summed over
        ranks: each cell has one owner, the others add 0)."""
        P = self.part
        nc = self.pt.mesh.n_cells
        buf = np.zeros((len(keys), nc))
        fl = self.solver.fields()
        for j, key in enumerate(keys):
            buf[j, P.cells[:P.n_owned]] = np.asarray(fl[key])[:P.n_owned]
        buf = self._allreduce(buf)
        return {key: buf[j] for j, key in enumerate(keys)}

    def gather_f(self) -> np.ndarray:
        P = self.part
        f = np.zeros((self.pt.mesh.n_cells, 9))
        f[P.cells[:P.n_owned]] = self.solver.get_f()[:P.n_owned]
        return self._allreduce(f)

    def forces(self) -> dict:
        cb = _Combine(self.pt, None)
        a = self._allreduce(cb.wall_force(self.rank, self.solver))
        return cb.coefficients(float(a[0]), float(a[1]))

    def close(self):
        if hasattr(self.solver, "close"):
            self.solver.close()
