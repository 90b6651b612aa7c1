"""Sharding one batched sweep across ranks (one process per GPU).

The instances of a sweep are independent problems (separate meshes, no shared cells), so the
sweep splits across ranks without any exchange inside the time step: each rank advances one
batched handle that holds its share of the instances.  Only the step statistics and the
per-instance results are combined, as FP64 collectives over ``torch.distributed`` (NCCL
between GPUs, gloo for the CPU tests):

  - residual: the largest per-instance residual of any rank (a handle already reports the
    largest over its own instances);
  - mass: the sum over ranks of the per-rank sums of rho_i A_i;
  - diverged: set if any rank saw a non-finite value;
  - forces, fields: gathered per instance, in the sweep's instance order.

The assignment balances the cells per rank greedily (largest instance first, to the rank with
the fewest cells so far; ties to the lower rank), so that the slowest rank -- which sets the
step time -- carries as little as possible beyond the mean.
"""
from __future__ import annotations

from typing import Callable, Sequence

import numpy as np


def assign_instances(cells: Sequence[int], world: int) -> list[list[int]]:
    """Instance indices per rank: greedy longest-processing-time balance of the cell counts.
    Deterministic; each rank's list is in ascending instance order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(cells)), key=lambda i: (-int(cells[i]), i))
    load = [0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += int(cells[i])
    return [sorted(v) for v in out]


class ShardedSweep:
    """One rank's share of a sweep of ``cases``.

    ``make_solver(cases)`` builds the rank's batched solver (``fvlbm.Solver`` on a GPU); it must
    provide ``step(n, stats)``, ``fields(i)`` and ``forces(i)`` for its local instance i.
    ``dist`` is ``torch.distributed`` with an initialised process group, or None for one rank.
    Ranks with no instance (more ranks than instances) hold no solver and contribute nothing
    to the combined results.
    """

    def __init__(self, cases: Sequence, make_solver: Callable, dist=None, device: str = "cpu"):
        self.dist = dist
        self.world = dist.get_world_size() if dist is not None else 1
        self.rank = dist.get_rank() if dist is not None else 0
        self.device = device
        self.n_total = len(cases)
        self.cells = [int(c.mesh.n_cells) for c in cases]
        self.assignment = assign_instances(self.cells, self.world)
        self.mine = self.assignment[self.rank]
        self.local_of = {g: k for k, g in enumerate(self.mine)}
        self.solver = make_solver([cases[g] for g in self.mine]) if self.mine else None

    # ------------------------------------------------------------------ collectives
    def _tensor(self, a):
        import torch
        return torch.as_tensor(np.asarray(a, np.float64), device=self.device)

    def _allreduce(self, a, op: str):
        if self.dist is None:
            return np.asarray(a, np.float64)
        t = self._tensor(a).clone()
        ops = {"sum": self.dist.ReduceOp.SUM, "max": self.dist.ReduceOp.MAX}
        self.dist.all_reduce(t, op=ops[op])
        return t.cpu().numpy()

    # ------------------------------------------------------------------ stepping
    def local_cells(self) -> int:
        return sum(self.cells[g] for g in self.mine)

    def step(self, n: int = 1, stats: bool = False):
        """Advance every instance of the sweep by n steps (each rank its share); with stats the
        combined FP64 statistics of the whole sweep."""
        st = self.solver.step(n, stats) if self.solver is not None and n > 0 else None
        if not stats:
            return None
        if st is None:  # a rank without instances
            st = {"steps": 0, "residual": 0.0, "mass": 0.0, "diverged": 0}
        res = self._allreduce([st["residual"], float(st["diverged"]), float(st["steps"])], "max")
        mass = self._allreduce([st["mass"]], "sum")
        return {"steps": int(res[2]), "residual": float(res[0]), "mass": float(mass[0]),
                "diverged": int(res[1] > 0)}

    # ------------------------------------------------------------------ per-instance results
    def gather_forces(self) -> np.ndarray:
        """[n_instances, 4] (fx, fy, C_D, C_L) of every instance of the sweep, on every rank."""
        out = np.zeros((self.n_total, 4))
        for g in self.mine:
            f = self.solver.forces(self.local_of[g])
            out[g] = (f["fx"], f["fy"], f["cd"], f["cl"])
        return self._allreduce(out, "sum")

    def gather_fields(self, keys=("rho", "u", "v")) -> list[dict]:
        """Fields of every instance of the sweep, on every rank (host arrays)."""
        offs = np.concatenate([[0], np.cumsum(self.cells)])
        buf = np.zeros((len(keys), int(offs[-1])))
        for g in self.mine:
            fl = self.solver.fields(self.local_of[g])
            for k, key in enumerate(keys):
                buf[k, offs[g]:offs[g + 1]] = fl[key]
        buf = self._allreduce(buf, "sum")
        return [{key: buf[k, offs[g]:offs[g + 1]].copy() for k, key in enumerate(keys)}
                for g in range(self.n_total)]

    def close(self):
        if self.solver is not None and hasattr(self.solver, "close"):
            self.solver.close()
        self.solver = None
