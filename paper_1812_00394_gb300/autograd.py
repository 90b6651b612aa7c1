"""C_L and C_D of an airfoil case as a differentiable PyTorch function.

``forces(model, p)`` returns the tensor (C_L, C_D) after ``model.steps`` FP64 time steps
(Steps 1-7 of Sec. 3.2, through the C ABI) of the case with parameters

    p = [alpha (radians), inflow eddy-viscosity ratio nu_t/nu, d_1, ..., d_W]

where d_j is the displacement of wall node ``model.wall_nodes[j]`` along its outward normal.
alpha sets the far-field velocity (U cos alpha, U sin alpha) and the drag / lift directions;
the ratio sets the far-field omega_b = k_b / (nu ratio).  The differentiated map keeps the
initial state and the time step of the base case fixed (they are inputs of the time
integration, not functions of p).

Two backward passes compute the same derivatives of the discrete step:
  - "tangent" (any case): the library's forward mode (precision FVLBM_FP64_TANGENT); one batched
    tangent solve with one instance per parameter gives every column of the Jacobian
    J = d(C_L, C_D)/dp at once, and the gradient is grad_output @ J.  Its cost grows with the
    number of parameters.
  - "adjoint": the library's reverse mode at the parameter level (fvlbm_adjoint_params): one
    adjoint solve of J_w = grad_output . (C_L, C_D), and the library's own chain rule to the
    angle, the ratio and the wall displacements (including the explicit dependence of the drag
    and lift directions on alpha).  This module only packs arrays.  Its cost does not grow
    with the number of parameters.  It covers every reading variant.
The default ("auto") takes the adjoint.

``step_forces(model, f0, bval, xy)`` (with a ``StepForces`` model) is the full-input form:
(C_D, C_L) as a function of the initial distributions, every boundary value and every node
position, with a one-adjoint backward pass.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

from . import fvlbm
from .meshgen import BC_FARFIELD, BC_WALL


class AirfoilForces:
    """The parameter-to-(C_L, C_D) map of one airfoil case (see the module docstring)."""

    def __init__(self, base_case, wall_nodes, steps: int, device: int = 0, mode: str = "auto"):
        if mode not in ("auto", "tangent", "adjoint"):
            raise ValueError(f"unknown backward mode {mode!r}")
        self.mode = "adjoint" if mode == "auto" else mode
        self.base = dataclasses.replace(base_case, mesh=base_case.mesh.normalized())
        m = self.base.mesh
        self.steps = int(steps)
        self.device = device
        self.wall_nodes = np.asarray(wall_nodes, np.int64)
        self.ff = m.bedge_type == BC_FARFIELD
        bv = m.bedge_val[self.ff]
        self.U = float(np.hypot(bv[0, 1], bv[0, 2]))
        self.k_b = bv[:, 3].copy()
        self.normals = self._wall_normals()
        # the base case's time step from the host preprocessing (no device work)
        rc, self.dt, why = fvlbm.check_case(self.base, precision=fvlbm.FVLBM_FP64, kernel_path=1)
        if rc < 0:
            raise fvlbm.FvlbmError(rc, f"AirfoilForces: {why}")
        rho, u, v, k, w = self.base.init_arrays()
        self.init = dict(rho=rho, u=u, v=v, k=k, omega=w)

    def _wall_normals(self) -> np.ndarray:
        """Outward unit normal (away from the body) at each chosen wall node, from the chord of
        its two wall neighbours."""
        m = self.base.mesh
        wall = m.bedge_nodes[m.bedge_type == BC_WALL]
        centre = m.xy[np.unique(wall)].mean(0)
        out = np.zeros((len(self.wall_nodes), 2))
        for j, nd in enumerate(self.wall_nodes):
            nb = np.unique(wall[(wall == nd).any(1)])
            nb = nb[nb != nd]
            if nb.size != 2:
                raise ValueError(f"node {nd} is not an interior wall node")
            t = m.xy[nb[1]] - m.xy[nb[0]]
            n = np.array([-t[1], t[0]]) / np.linalg.norm(t)
            if np.dot(n, m.xy[nd] - centre) < 0:
                n = -n
            out[j] = n
        return out

    def n_params(self) -> int:
        return 2 + len(self.wall_nodes)

    def case_at(self, p: np.ndarray):
        """The case at parameters p (initial state and dt of the base case)."""
        alpha, ratio, disp = float(p[0]), float(p[1]), np.asarray(p[2:], np.float64)
        m = self.base.mesh
        bval = m.bedge_val.copy()
        bval[self.ff, 1] = self.U * math.cos(alpha)
        bval[self.ff, 2] = self.U * math.sin(alpha)
        bval[self.ff, 4] = self.k_b / (self.base.nu * ratio)
        xy = m.xy.copy()
        xy[self.wall_nodes] += disp[:, None] * self.normals
        mesh = dataclasses.replace(m, xy=xy, bedge_val=bval)
        return dataclasses.replace(self.base, mesh=mesh, dt=self.dt, alpha_deg=math.degrees(alpha),
                                   **self.init)

    def value(self, p: np.ndarray) -> np.ndarray:
        s = fvlbm.Solver(self.case_at(p), precision=fvlbm.FVLBM_FP64, device=self.device,
                         kernel_path=1)
        s.step(self.steps)
        f = s.forces()
        s.close()
        return np.array([f["cl"], f["cd"]])

    def _bval_directions(self, case, p: np.ndarray):
        """d(boundary values)/d alpha and d(boundary values)/d ratio at p."""
        m = case.mesh
        nb = m.n_bedges
        d_alpha = np.zeros((nb, 5))
        d_alpha[self.ff, 1] = -m.bedge_val[self.ff, 2]
        d_alpha[self.ff, 2] = m.bedge_val[self.ff, 1]
        d_ratio = np.zeros((nb, 5))
        d_ratio[self.ff, 4] = -m.bedge_val[self.ff, 4] / float(p[1])
        return d_alpha, d_ratio

    def vjp(self, p: np.ndarray, g: np.ndarray, out: np.ndarray) -> np.ndarray:
        """g @ d(C_L, C_D)/dp (g ordered like the outputs C_L, C_D) from the library's
        parameter-level adjoint, fvlbm_adjoint_params: one adjoint solve of
        J = g_CD C_D + g_CL C_L and its chain rule to (alpha, ratio, wall displacements), all
        behind the C ABI."""
        s = fvlbm.Solver(self.case_at(p), precision=fvlbm.FVLBM_FP64, device=self.device,
                         kernel_path=1)
        r = s.adjoint_params(self.steps, w_cd=float(g[1]), w_cl=float(g[0]),
                             wall_nodes=self.wall_nodes, wall_normals=self.normals)
        s.close()
        return np.concatenate([[r["dalpha"], r["dratio"]], r["dwall"]])

    def jacobian(self, p: np.ndarray) -> np.ndarray:
        """J[o, q] = d output_o / d p_q (outputs C_L, C_D) from one batched tangent solve."""
        case = self.case_at(p)
        m = case.mesh
        d_alpha, d_ratio = self._bval_directions(case, p)
        dirs = [{"dbedge_val": d_alpha, "dalpha": 1.0}, {"dbedge_val": d_ratio}]
        for j, nd in enumerate(self.wall_nodes):
            dxy = np.zeros_like(m.xy)
            dxy[nd] = self.normals[j]
            dirs.append({"dxy": dxy})
        _, grads = fvlbm.forces_gradient(case, dirs, self.steps, device=self.device)
        return np.array([[g["cl"] for g in grads], [g["cd"] for g in grads]])


class _ForcesFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, p, model):
        pn = p.detach().cpu().double().numpy()
        out = model.value(pn)
        ctx.model, ctx.pn, ctx.out = model, pn, out
        return torch.as_tensor(out, dtype=p.dtype, device=p.device)

    @staticmethod
    def backward(ctx, grad_out):
        gn = grad_out.detach().cpu().double().numpy()
        if ctx.model.mode == "adjoint":
            g = ctx.model.vjp(ctx.pn, gn, ctx.out)
        else:
            g = gn @ ctx.model.jacobian(ctx.pn)
        return torch.as_tensor(g, dtype=grad_out.dtype, device=grad_out.device), None


def forces(model: AirfoilForces, p: torch.Tensor) -> torch.Tensor:
    """(C_L, C_D) of ``model`` at parameters ``p`` (1-D tensor of length model.n_params()),
    differentiable with respect to p."""
    return _ForcesFunction.apply(p, model)


class StepForces:
    """(C_D, C_L) of one case after ``steps`` FP64 steps as a function of the full inputs: the
    initial distributions f0 [n_cells, 9] (cell-major, as ``Solver.get_f``), the boundary values
    [n_bedges, 5] and the node positions [n_nodes, 2].  The time step is the base case's, held
    fixed.  Its backward pass is one adjoint solve (``fvlbm_adjoint``) whatever the number of
    inputs: the vector-Jacobian product with respect to all three at once."""

    def __init__(self, base_case, steps: int, device: int = 0):
        self.base = dataclasses.replace(base_case, mesh=base_case.mesh.normalized())
        self.steps = int(steps)
        self.device = device
        probe = fvlbm.Solver(self.base, precision=fvlbm.FVLBM_FP64, device=device, kernel_path=1)
        self.dt = probe.dt()
        self.f0 = probe.get_f()
        probe.close()

    def inputs(self):
        """The base case's (f0, boundary values, node positions) as float64 tensors."""
        m = self.base.mesh
        return (torch.tensor(self.f0), torch.tensor(m.bedge_val.copy()), torch.tensor(m.xy.copy()))

    def solver(self, f0, bval, xy):
        mesh = dataclasses.replace(self.base.mesh, xy=np.ascontiguousarray(xy, np.float64),
                                   bedge_val=np.ascontiguousarray(bval, np.float64))
        case = dataclasses.replace(self.base, mesh=mesh, dt=self.dt)
        s = fvlbm.Solver(case, precision=fvlbm.FVLBM_FP64, device=self.device, kernel_path=1)
        s.set_f(np.ascontiguousarray(f0, np.float64))
        return s


class _StepForcesFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f0, bval, xy, model):
        arrs = [t.detach().cpu().double().numpy() for t in (f0, bval, xy)]
        s = model.solver(*arrs)
        s.step(model.steps)
        f = s.forces()
        s.close()
        ctx.model, ctx.arrs = model, arrs
        ctx.devs = [t.device for t in (f0, bval, xy)]
        return torch.tensor([f["cd"], f["cl"]], dtype=torch.float64, device=f0.device)

    @staticmethod
    def backward(ctx, g):
        gn = g.detach().cpu().double().numpy()
        s = ctx.model.solver(*ctx.arrs)
        _, df, db, dxy = s.adjoint(ctx.model.steps, w_cd=float(gn[0]), w_cl=float(gn[1]),
                                   shape=ctx.needs_input_grad[2])
        s.close()
        as_t = lambda a, d: None if a is None else torch.as_tensor(a, dtype=torch.float64, device=d)  # noqa: E731
        return (as_t(df, ctx.devs[0]) if ctx.needs_input_grad[0] else None,
                as_t(db, ctx.devs[1]) if ctx.needs_input_grad[1] else None,
                as_t(dxy, ctx.devs[2]) if ctx.needs_input_grad[2] else None, None)


def step_forces(model: StepForces, f0: torch.Tensor, bval: torch.Tensor, xy: torch.Tensor) -> torch.Tensor:
    """(C_D, C_L) of ``model`` from (f0, boundary values, node positions), differentiable with
    respect to each of them."""
    return _StepForcesFunction.apply(f0, bval, xy, model)
