"""Seeded synthetic inputs: unstructured 2-D meshes, boundary tables, initial fields.

Every workload of this library is generated here from a seed; there are no datasets.
This module builds node coordinates, cell-node connectivity and per-boundary-edge
tables only.  It holds none of the method's arithmetic (no equilibrium, no fluxes, no
geometry such as areas or normals): the CUDA library and the CPU oracle each derive
everything else from these arrays with their own code.

Mesh format (shared by every consumer):

* ``xy``            float64 [n_nodes, 2]   node coordinates
* ``cell_ptr``      int32   [n_cells + 1]  CSR offsets into ``cell_nodes``
* ``cell_nodes``    int32                  3 or 4 node ids per cell, counter-clockwise
* ``bedge_nodes``   int32   [n_bedges, 2]  the two nodes of each boundary edge
* ``bedge_type``    int32   [n_bedges]     BC_WALL / BC_INLET / BC_OUTLET / BC_FARFIELD /
  BC_PERIODIC
* ``bedge_val``     float64 [n_bedges, 5]  (rho_b, u_b, v_b, k_b, omega_b) of that edge
* ``periodic_pairs`` int32  [n_pairs, 2]   boundary-edge indices (a, b) glued together;
  edge b is edge a translated by ``periodic_shift``
* ``periodic_shift`` float64 [n_pairs, 2]

The paper's meshes were made with Salome (Sec. 4); these generators stand in for them
with meshes of the sizes and kinds the paper's test cases use: uniform quads and
jittered Delaunay triangles on the lid-driven cavity (Sec. 4.1), wall-clustered hybrid
quad/triangle meshes for the backward-facing step (Sec. 4.2) and an airfoil C-mesh
(Sec. 4.3).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

BC_WALL = 0
BC_INLET = 1
BC_OUTLET = 2
BC_FARFIELD = 3
BC_PERIODIC = 4

CS2 = 1.0 / 3.0  # lattice sound speed squared of D2Q9 (Eq. turbtau); used to state tau

__all__ = [
    "Mesh", "Case", "BC_WALL", "BC_INLET", "BC_OUTLET", "BC_FARFIELD", "BC_PERIODIC",
    "splitmix64_uniform", "quad_grid", "split_quads", "periodic_box", "couette_channel",
    "cavity_quad", "cavity_delaunay", "bfs_hybrid", "naca0012_cmesh", "batched_sweep",
]


# --------------------------------------------------------------------------- containers
@dataclass
class Mesh:
    xy: np.ndarray
    cell_ptr: np.ndarray
    cell_nodes: np.ndarray
    bedge_nodes: np.ndarray
    bedge_type: np.ndarray
    bedge_val: np.ndarray
    periodic_pairs: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.int32))
    periodic_shift: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.float64))
    name: str = ""

    @property
    def n_nodes(self) -> int:
        return int(self.xy.shape[0])

    @property
    def n_cells(self) -> int:
        return int(self.cell_ptr.shape[0] - 1)

    @property
    def n_bedges(self) -> int:
        return int(self.bedge_nodes.shape[0])

    def normalized(self) -> "Mesh":
        """Return a copy with every array contiguous and of the exact dtype the C code reads."""
        return Mesh(
            xy=np.ascontiguousarray(self.xy, np.float64),
            cell_ptr=np.ascontiguousarray(self.cell_ptr, np.int32),
            cell_nodes=np.ascontiguousarray(self.cell_nodes, np.int32),
            bedge_nodes=np.ascontiguousarray(self.bedge_nodes, np.int32).reshape(-1, 2),
            bedge_type=np.ascontiguousarray(self.bedge_type, np.int32),
            bedge_val=np.ascontiguousarray(self.bedge_val, np.float64).reshape(-1, 5),
            periodic_pairs=np.ascontiguousarray(self.periodic_pairs, np.int32).reshape(-1, 2),
            periodic_shift=np.ascontiguousarray(self.periodic_shift, np.float64).reshape(-1, 2),
            name=self.name,
        )


@dataclass
class Case:
    """A mesh plus physical parameters and initial fields (one solver instance).

    ``dt`` > 0 fixes the time step; otherwise ``cfl`` sets it from the convective
    limit of the mesh (computed by the solver).  ``rho``/``u``/``v``/``k``/``omega``
    are per-cell initial fields in the mesh's cell order.
    """
    mesh: Mesh
    nu: float
    rho0: float = 1.0
    dt: float = 0.0
    cfl: float = 0.0
    sst: bool = False
    uref: float = 0.1
    lref: float = 1.0
    alpha_deg: float = 0.0
    rho: np.ndarray | None = None
    u: np.ndarray | None = None
    v: np.ndarray | None = None
    k: np.ndarray | None = None
    omega: np.ndarray | None = None
    name: str = ""
    local_dt: bool = False   # local time stepping dt_i = cfl * limit_i (steady runs only)
    variant: int = 0         # reading variants (bit mask): 1 limiter on grad f, 2 SST
                             # non-orthogonal diffusion correction

    @property
    def tau(self) -> float:
        return self.nu / CS2

    def init_arrays(self):
        n = self.mesh.n_cells
        rho = np.full(n, self.rho0) if self.rho is None else np.asarray(self.rho, np.float64)
        u = np.zeros(n) if self.u is None else np.asarray(self.u, np.float64)
        v = np.zeros(n) if self.v is None else np.asarray(self.v, np.float64)
        k = np.zeros(n) if self.k is None else np.asarray(self.k, np.float64)
        w = np.ones(n) if self.omega is None else np.asarray(self.omega, np.float64)
        return [np.ascontiguousarray(a, np.float64) for a in (rho, u, v, k, w)]


# --------------------------------------------------------------------------- random numbers
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64_uniform(seed: int, n: int) -> np.ndarray:
    """``n`` doubles uniform on [-1, 1) from the SplitMix64 generator (Steele et al. 2014).

    State i is ``seed + (i+1) * 0x9E3779B97F4A7C15``; the output mix is the published one
    (shifts 30/27/31, multipliers 0xBF58476D1CE4E5B9 and 0x94D049BB133111EB); the top 53
    bits give a double in [0, 1) which is mapped to [-1, 1).
    """
    with np.errstate(over="ignore"):
        i = np.arange(1, n + 1, dtype=np.uint64)
        z = (np.uint64(seed) + i * np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        z = z ^ (z >> np.uint64(31))
    u01 = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u01 - 1.0


# --------------------------------------------------------------------------- structured grids
def quad_grid(xs: np.ndarray, ys: np.ndarray, jitter: float = 0.0, seed: int = 0):
    """Tensor-product quad grid on node lines ``xs`` x ``ys`` (counter-clockwise cells).

    ``jitter`` moves every interior node by up to ``jitter`` times the local spacing.
    Returns (xy, cells [nc,4], side edges dict: 'bottom','right','top','left' -> [n,2] node ids
    ordered along increasing x (bottom/top) or y (left/right)).
    """
    nx, ny = len(xs) - 1, len(ys) - 1
    X, Y = np.meshgrid(xs, ys, indexing="xy")  # [ny+1, nx+1]
    xy = np.stack([X.ravel(), Y.ravel()], 1).astype(np.float64)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        hx = np.minimum(np.diff(xs)[:-1], np.diff(xs)[1:])
        hy = np.minimum(np.diff(ys)[:-1], np.diff(ys)[1:])
        HX, HY = np.meshgrid(hx, hy, indexing="xy")
        idx = (np.arange(1, ny)[:, None] * (nx + 1) + np.arange(1, nx)[None, :]).ravel()
        d = rng.uniform(-jitter, jitter, (idx.size, 2))
        xy[idx, 0] += d[:, 0] * HX.ravel()
        xy[idx, 1] += d[:, 1] * HY.ravel()
    nid = lambda i, j: j * (nx + 1) + i  # noqa: E731
    I, J = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    I, J = I.ravel(), J.ravel()
    cells = np.stack([nid(I, J), nid(I + 1, J), nid(I + 1, J + 1), nid(I, J + 1)], 1)
    i = np.arange(nx)
    j = np.arange(ny)
    sides = {
        "bottom": np.stack([nid(i, 0), nid(i + 1, 0)], 1),
        "top": np.stack([nid(i, ny), nid(i + 1, ny)], 1),
        "left": np.stack([nid(0, j), nid(0, j + 1)], 1),
        "right": np.stack([nid(nx, j), nid(nx, j + 1)], 1),
    }
    return xy, cells.astype(np.int32), sides


def split_quads(cells4: np.ndarray, pattern: str = "alternate") -> np.ndarray:
    """Split each counter-clockwise quad (a,b,c,d) into two counter-clockwise triangles."""
    a, b, c, d = cells4.T
    n = cells4.shape[0]
    if pattern == "alternate":
        flip = (np.arange(n) % 2).astype(bool)
    else:
        flip = np.zeros(n, bool)
    t1 = np.where(flip[:, None], np.stack([a, b, d], 1), np.stack([a, b, c], 1))
    t2 = np.where(flip[:, None], np.stack([b, c, d], 1), np.stack([a, c, d], 1))
    tris = np.empty((2 * n, 3), np.int32)
    tris[0::2] = t1
    tris[1::2] = t2
    return tris


def _cells_to_csr(cells) -> tuple[np.ndarray, np.ndarray]:
    if isinstance(cells, np.ndarray):
        k = cells.shape[1]
        ptr = np.arange(cells.shape[0] + 1, dtype=np.int32) * k
        return ptr, cells.astype(np.int32).ravel()
    ptr = np.zeros(len(cells) + 1, np.int32)
    ptr[1:] = np.cumsum([len(c) for c in cells])
    return ptr, np.concatenate([np.asarray(c, np.int32) for c in cells])


def _bvals(n: int, rho=1.0, u=0.0, v=0.0, k=0.0, w=0.0) -> np.ndarray:
    out = np.empty((n, 5))
    out[:, 0], out[:, 1], out[:, 2], out[:, 3], out[:, 4] = rho, u, v, k, w
    return out


# --------------------------------------------------------------------------- test meshes
def periodic_box(n: int, kind: str = "quad", jitter: float = 0.0, seed: int = 0,
                 L: float = 1.0) -> Mesh:
    """Unit square (side ``L``) periodic in x and y; quads or split-quad triangles."""
    xs = np.linspace(0.0, L, n + 1)
    xy, cells, sides = quad_grid(xs, xs, jitter, seed)
    cells_out = split_quads(cells) if kind == "tri" else cells
    bn = np.concatenate([sides["bottom"], sides["top"], sides["left"], sides["right"]])
    nb = bn.shape[0]
    pairs = np.concatenate([
        np.stack([np.arange(n), n + np.arange(n)], 1),
        np.stack([2 * n + np.arange(n), 3 * n + np.arange(n)], 1),
    ]).astype(np.int32)
    shift = np.concatenate([np.tile([0.0, L], (n, 1)), np.tile([L, 0.0], (n, 1))])
    ptr, cn = _cells_to_csr(cells_out)
    return Mesh(xy, ptr, cn, bn, np.full(nb, BC_PERIODIC, np.int32), _bvals(nb),
                pairs, shift, name=f"periodic_{kind}_{n}").normalized()


def couette_channel(nx: int, ny: int, U: float = 0.1, H: float = 1.0, Lx: float = 1.0,
                    kind: str = "quad", jitter: float = 0.0, seed: int = 0,
                    stretch: float = 1.0) -> Mesh:
    """Channel periodic in x; bottom wall at rest, top wall moving at (U, 0).  ``stretch`` > 1
    grows the row heights geometrically from the bottom wall by that ratio per row."""
    xs = np.linspace(0.0, Lx, nx + 1)
    if stretch == 1.0:
        ys = np.linspace(0.0, H, ny + 1)
    else:
        hs = stretch ** np.arange(ny)
        ys = np.concatenate([[0.0], np.cumsum(hs)]) * (H / hs.sum())
        ys[-1] = H
    xy, cells, sides = quad_grid(xs, ys, jitter, seed)
    cells_out = split_quads(cells) if kind == "tri" else cells
    bn = np.concatenate([sides["bottom"], sides["top"], sides["left"], sides["right"]])
    bt = np.concatenate([np.full(nx, BC_WALL), np.full(nx, BC_WALL),
                         np.full(2 * ny, BC_PERIODIC)]).astype(np.int32)
    bv = _bvals(bn.shape[0])
    bv[nx:2 * nx, 1] = U
    pairs = np.stack([2 * nx + np.arange(ny), 2 * nx + ny + np.arange(ny)], 1).astype(np.int32)
    shift = np.tile([Lx, 0.0], (ny, 1))
    ptr, cn = _cells_to_csr(cells_out)
    return Mesh(xy, ptr, cn, bn, bt, bv, pairs, shift, name=f"couette_{kind}_{nx}x{ny}").normalized()


def _cavity_bc(bn: np.ndarray, xy: np.ndarray, lid_u: float):
    """Lid-driven cavity: the top side y = 1 moves at (lid_u, 0); the other sides are at rest."""
    mid_y = 0.5 * (xy[bn[:, 0], 1] + xy[bn[:, 1], 1])
    bt = np.full(bn.shape[0], BC_WALL, np.int32)
    bv = _bvals(bn.shape[0])
    bv[mid_y > 1.0 - 1e-12, 1] = lid_u
    return bt, bv


def cavity_quad(n: int = 64, re: float = 400.0, lid_u: float = 0.1, cfl: float = 0.5,
                noise: float = 1e-6, seed: int = 1, jitter: float = 0.0) -> Case:
    """Lid-driven cavity on an n x n uniform quad mesh stored as unstructured connectivity.

    Sec. 4.1 runs the lid-driven cavity; the small laminar case here is Re = 400, lid speed
    0.1, rho0 = 1, u = 0 plus seeded uniform noise of amplitude ``noise`` on rho.
    """
    xs = np.linspace(0.0, 1.0, n + 1)
    xy, cells, sides = quad_grid(xs, xs, jitter, seed)
    bn = np.concatenate([sides["bottom"], sides["right"], sides["top"], sides["left"]])
    bt, bv = _cavity_bc(bn, xy, lid_u)
    ptr, cn = _cells_to_csr(cells)
    m = Mesh(xy, ptr, cn, bn, bt, bv, name=f"cavity_quad_{n}").normalized()
    rho = 1.0 + noise * splitmix64_uniform(seed, m.n_cells)
    return Case(m, nu=lid_u * 1.0 / re, cfl=cfl, uref=lid_u, lref=1.0, rho=rho,
                name=f"cavity_quad{n}_re{re:g}")


def cavity_delaunay(h_boundary: float = 1.0 / 200.0, n_target: int = 40000, re: float = 1000.0,
                    lid_u: float = 0.1, z: float = 5.0, seed: int = 2,
                    noise: float = 1e-6, cfl: float = 0.0) -> Case:
    """Lid-driven cavity on a seeded Delaunay triangulation of the unit square.

    Boundary points sit at spacing ``h_boundary``; interior points form a hexagonal lattice
    sized for about ``n_target`` triangles, each point jittered by the seed.  The time step
    is ``z`` relaxation times (dt = z * tau, tau = nu / cs^2), or, when ``cfl`` > 0, ``cfl``
    times the convective limit of the mesh.
    """
    from scipy.spatial import Delaunay

    nb = int(round(1.0 / h_boundary))
    t = np.arange(nb) / nb
    zero, one = np.zeros(nb), np.ones(nb)
    bpts = np.concatenate([np.stack([t, zero], 1), np.stack([one, t], 1),
                           np.stack([1 - t, one], 1), np.stack([zero, 1 - t], 1)])
    n_int = max(4, (n_target - 4 * nb + 2) // 2)
    h = math.sqrt(2.0 / (math.sqrt(3.0) * n_int))
    rng = np.random.default_rng(seed)
    pts = []
    ys = np.arange(0.6 * h, 1.0 - 0.5 * h, h * math.sqrt(3.0) / 2.0)
    for r, y in enumerate(ys):
        xs = np.arange(0.6 * h + (r % 2) * 0.5 * h, 1.0 - 0.5 * h, h)
        pts.append(np.stack([xs, np.full_like(xs, y)], 1))
    ip = np.concatenate(pts)
    ip += rng.uniform(-0.15, 0.15, ip.shape) * h
    xy = np.concatenate([bpts, ip]).astype(np.float64)
    tri = Delaunay(xy).simplices.astype(np.int64)
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    cross = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    keep = np.abs(cross) > 1e-14
    tri = tri[keep]
    cross = cross[keep]
    flip = cross < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]
    ring = np.arange(4 * nb)
    bn = np.stack([ring, (ring + 1) % (4 * nb)], 1).astype(np.int32)
    bt, bv = _cavity_bc(bn, xy, lid_u)
    ptr, cn = _cells_to_csr(tri.astype(np.int32))
    m = Mesh(xy, ptr, cn, bn, bt, bv, name=f"cavity_delaunay_{tri.shape[0]}").normalized()
    nu = lid_u / re
    rho = 1.0 + noise * splitmix64_uniform(seed, m.n_cells)
    if cfl > 0.0:
        return Case(m, nu=nu, cfl=cfl, uref=lid_u, lref=1.0, rho=rho,
                    name=f"cavity_delaunay{m.n_cells}_re{re:.0f}_cfl{cfl:g}")
    return Case(m, nu=nu, dt=z * nu / CS2, uref=lid_u, lref=1.0, rho=rho,
                name=f"cavity_delaunay{m.n_cells}_re{re:.0f}_z{z:g}")


# --------------------------------------------------------------------------- turbulent meshes
def _stretched(n: int, L: float, first: float) -> np.ndarray:
    """Node coordinates 0..L with n intervals, geometric growth from a first spacing ``first``."""
    if first * n >= L:
        return np.linspace(0.0, L, n + 1)
    lo, hi = 1.0 + 1e-12, 2.0
    for _ in range(200):  # bisection on the growth ratio r: first * (r^n - 1)/(r - 1) = L
        r = 0.5 * (lo + hi)
        s = first * (r ** n - 1.0) / (r - 1.0)
        lo, hi = (r, hi) if s < L else (lo, r)
    r = 0.5 * (lo + hi)
    x = np.concatenate([[0.0], np.cumsum(first * r ** np.arange(n))])
    return x * (L / x[-1])


def _two_sided(n: int, L: float, first: float) -> np.ndarray:
    """0..L with n intervals (n even), clustered at both ends."""
    half = _stretched(n // 2, 0.5 * L, first)
    return np.concatenate([half, L - half[-2::-1]])


def _hybrid_cells(cells4: np.ndarray, tri_mask: np.ndarray):
    """Keep quads where ``tri_mask`` is false; split the others into two triangles.
    Returns CSR (ptr, nodes)."""
    quads = cells4[~tri_mask]
    tris = split_quads(cells4[tri_mask])
    nq, nt = quads.shape[0], tris.shape[0]
    ptr = np.concatenate([np.arange(nq + 1) * 4, 4 * nq + np.arange(1, nt + 1) * 3]).astype(np.int32)
    return ptr, np.concatenate([quads.ravel(), tris.ravel()]).astype(np.int32)


def bfs_hybrid(n_target: int = 80000, h: float = 1.0, expansion: float = 1.125,
               re_h: float = 3.6e4, uref: float = 0.1, yplus1: float = 1.0,
               intensity: float = 0.01, nut_ratio: float = 10.0, cfl: float = 0.5,
               seed: int = 3, _res: float = 1.0) -> Case:
    """Turbulent backward-facing step on a hybrid mesh (Sec. 4.2 geometry family).

    Step height h; channel height downstream ``expansion / (expansion - 1) * h``; inlet at
    -4h, outlet at +30h.  Quads are clustered at every wall (first cell height from y+ ~
    ``yplus1`` with a flat-plate skin-friction estimate) and cells away from walls are split
    into triangles.  Inlet: 1/7 power-law profile, turbulence intensity ``intensity`` and
    nu_t / nu = ``nut_ratio``.  The time step is ``cfl`` times the convective limit of the
    smallest (wall) cells.
    """
    H = expansion / (expansion - 1.0) * h          # downstream height
    Hin = H - h                                     # upstream channel height
    nu = uref * h / re_h
    cf = 0.026 / re_h ** (1.0 / 7.0)                # flat-plate estimate for the first cell
    utau = uref * math.sqrt(0.5 * cf)
    dy1 = yplus1 * nu / utau
    x_in, x_out = -4.0 * h, 30.0 * h
    # grid lines: x clustered at the step corner, y clustered at walls
    frac_up = 4.0 / 34.0
    # choose resolution from the target: cells ~ nx * ny (upstream only covers Hin)
    ny_lo = max(8, int(round(math.sqrt(n_target / 34.0 * 0.9) * 1.2 * _res)))
    ny_lo = ny_lo + (ny_lo % 2)
    ny_up = max(8, int(round(ny_lo * Hin / H * 1.6)))
    ny_up = ny_up + (ny_up % 2)
    ny_step = max(4, int(round(ny_lo * h / H * 3.0)))
    ny_step += ny_step % 2
    nx_total = max(20, int(n_target / (ny_up + ny_step) / 1.6 * _res))
    nx_up = max(6, int(round(nx_total * frac_up)))
    nx_dn = nx_total - nx_up
    xs_up = x_in + (-x_in) * (1.0 - _stretched(nx_up, 1.0, 0.5 / nx_up * 0.3)[::-1])
    xs_dn = _stretched(nx_dn, x_out, dy1 * 50.0)
    xs = np.concatenate([xs_up[:-1], xs_dn])
    ys_step = _two_sided(ny_step, h, dy1)
    ys_up = h + _two_sided(ny_up, Hin, dy1)
    ys = np.concatenate([ys_step[:-1], ys_up])
    nxu = len(xs_up) - 1
    nx = len(xs) - 1
    nyl = len(ys_step) - 1
    ny = len(ys) - 1
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    # keep nodes that belong to at least one cell of the domain (exclude the solid step block)
    nid = -np.ones((ny + 1, nx + 1), np.int64)
    valid_cell = np.ones((ny, nx), bool)
    valid_cell[:nyl, :nxu] = False
    used = np.zeros((ny + 1, nx + 1), bool)
    jj, ii = np.nonzero(valid_cell)
    for dj, di in ((0, 0), (0, 1), (1, 1), (1, 0)):
        used[jj + dj, ii + di] = True
    nid[used] = np.arange(used.sum())
    xy = np.stack([X[used], Y[used]], 1).astype(np.float64)
    cells4 = np.stack([nid[jj, ii], nid[jj, ii + 1], nid[jj + 1, ii + 1], nid[jj + 1, ii]], 1)
    # quads within a wall layer, triangles in the core
    yc = 0.5 * (ys[jj] + ys[jj + 1])
    xc = 0.5 * (xs[ii] + xs[ii + 1])
    dist = np.minimum(H - yc, np.where(xc < 0.0, yc - h, yc))
    dist = np.where((xc >= 0.0) & (yc < h), np.minimum(dist, np.abs(xc)), dist)
    tri_mask = dist > 0.25 * h
    ptr, cn = _hybrid_cells(cells4.astype(np.int32), tri_mask)
    # boundary edges
    bn, bt, bvl = [], [], []
    k_in = 1.5 * (intensity * uref) ** 2
    w_in = k_in / (nu * nut_ratio)

    def add(a, b, typ, val):
        bn.append((a, b)); bt.append(typ); bvl.append(val)
    # walls: bottom downstream, step face, upstream bottom, top
    for i in range(nxu, nx):
        add(nid[0, i], nid[0, i + 1], BC_WALL, (1.0, 0.0, 0.0, 0.0, 0.0))
    for j in range(nyl):
        add(nid[j, nxu], nid[j + 1, nxu], BC_WALL, (1.0, 0.0, 0.0, 0.0, 0.0))
    for i in range(nxu):
        add(nid[nyl, i], nid[nyl, i + 1], BC_WALL, (1.0, 0.0, 0.0, 0.0, 0.0))
    for i in range(nx):
        add(nid[ny, i], nid[ny, i + 1], BC_WALL, (1.0, 0.0, 0.0, 0.0, 0.0))
    # inlet (x = -4h) with a 1/7 power law in the wall distance of the upstream channel
    for j in range(nyl, ny):
        ym = 0.5 * (ys[j] + ys[j + 1])
        eta = min(ym - h, H - ym) / (0.5 * Hin)
        uin = uref * (8.0 / 7.0) * max(eta, 0.0) ** (1.0 / 7.0)
        add(nid[j, 0], nid[j + 1, 0], BC_INLET, (1.0, uin, 0.0, k_in, w_in))
    for j in range(ny):
        add(nid[j, nx], nid[j + 1, nx], BC_OUTLET, (1.0, 0.0, 0.0, k_in, w_in))
    m = Mesh(xy, ptr, cn, np.asarray(bn, np.int32), np.asarray(bt, np.int32),
             np.asarray(bvl, np.float64), name=f"bfs_hybrid_{len(ptr) - 1}").normalized()
    n = m.n_cells
    if _res == 1.0 and abs(n - n_target) > 0.05 * n_target:   # one resize to hit the target
        return bfs_hybrid(n_target, h, expansion, re_h, uref, yplus1, intensity, nut_ratio, cfl,
                          seed, _res=math.sqrt(n_target / n))
    return Case(m, nu=nu, cfl=cfl, sst=True, uref=uref, lref=h,
                rho=np.ones(n), u=np.zeros(n), v=np.zeros(n), k=np.full(n, k_in),
                omega=np.full(n, w_in), name=f"bfs{n}_reh{re_h:g}")


def _naca0012_y(x: np.ndarray) -> np.ndarray:
    """Half thickness of the NACA 0012 section (standard 4-digit formula, closed trailing edge)."""
    t = 0.12
    return 5.0 * t * (0.2969 * np.sqrt(np.maximum(x, 0.0)) - 0.1260 * x - 0.3516 * x ** 2
                      + 0.2843 * x ** 3 - 0.1036 * x ** 4)


def naca0012_cmesh(n_target: int = 200000, re_c: float = 6e6, uref: float = 0.1,
                   alpha_deg: float = 0.0, far: float = 20.0, yplus1: float = 1.0,
                   intensity: float = 0.01, nut_ratio: float = 1.0, cfl: float = 0.5,
                   quad_layer: float = 0.4, seed: int = 4) -> Case:
    """Turbulent NACA 0012 on an algebraic C-mesh (Sec. 4.3 case family).

    Chord 1, far-field boundary at ``far`` chords, first cell from y+ ~ ``yplus1`` at Re_c.
    Rows within ``quad_layer`` chords of the wall are quads; outer rows are split into
    triangles (hybrid).  Free stream at angle ``alpha_deg``.  The time step is ``cfl`` times the
    convective limit of the smallest cells (the collision is implicit, so dt >> tau).
    """
    nu = uref / re_c
    cf = 0.026 / re_c ** (1.0 / 7.0)
    utau = uref * math.sqrt(0.5 * cf)
    dy1 = yplus1 * nu / utau
    # points along the C: wake (lower), airfoil lower TE->LE, upper LE->TE, wake (upper)
    n_j = max(24, int(round(math.sqrt(n_target / 3.2))))
    eta = _stretched(n_j, 1.0, dy1 / far)
    n_quad_rows = int(np.sum(eta[1:] <= quad_layer / far))
    per_col = n_quad_rows + 2 * (n_j - n_quad_rows)
    n_i = max(48, int(round(n_target / per_col)))
    n_af = max(16, int(n_i * 0.55) // 2)          # points per airfoil side
    n_wk = max(8, (n_i - 2 * n_af) // 2)          # wake points per side
    beta = np.linspace(0.0, math.pi, n_af + 1)
    xa = 0.5 * (1.0 - np.cos(beta))               # LE clustered cosine spacing, 0..1
    xu = xa[::-1]                                  # TE -> LE (lower side traversed TE->LE)
    lower = np.stack([xu, -_naca0012_y(xu)], 1)
    upper = np.stack([xa[1:], _naca0012_y(xa[1:])], 1)
    wake_x = 1.0 + _stretched(n_wk, far, 0.5 / n_af * 2.0)[1:]
    wake_lo = np.stack([wake_x[::-1], np.zeros(n_wk)], 1)
    wake_up = np.stack([wake_x, np.zeros(n_wk)], 1)
    inner = np.concatenate([wake_lo, lower, upper, wake_up])       # [ni+1, 2]
    ni = inner.shape[0] - 1
    # outer C boundary: wake lines at y = -/+ far, semicircle around the leading region
    s = np.linspace(0.0, 1.0, ni + 1)
    ang = np.pi * 0.5 + np.pi * np.clip((s - 0.25) / 0.5, 0.0, 1.0)
    outer = np.empty_like(inner)
    for idx in range(ni + 1):
        xi = inner[idx, 0]
        if idx < n_wk or idx > ni - n_wk:
            outer[idx] = (xi, -far if idx < n_wk else far)
        else:
            th = math.pi * 1.5 - math.pi * (idx - n_wk) / (ni - 2 * n_wk)
            outer[idx] = (0.5 + far * math.cos(th), far * math.sin(th))
    del ang, s
    # wall-normal direction for the near-wall layer (orthogonal start, blend to the outer line
    # within a few hundredths of a chord; tapered to zero at the sharp trailing edge)
    tang = np.gradient(inner, axis=0)
    nrm = np.stack([-tang[:, 1], tang[:, 0]], 1)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True) + 1e-300
    on_af = (np.arange(ni + 1) >= n_wk) & (np.arange(ni + 1) <= ni - n_wk)
    taper = np.where(on_af, np.clip((1.0 - inner[:, 0]) / 0.05, 0.0, 1.0), 0.0)[:, None]
    X = np.empty((n_j + 1, ni + 1, 2))
    for j, e in enumerate(eta):
        lin = inner + e * (outer - inner)
        orth = inner + e * far * nrm
        wgt = taper * math.exp(-e * far / 0.01)
        X[j] = wgt * orth + (1.0 - wgt) * lin
    # node ids; the wake cut (j = 0, idx <= n_wk) and (j = 0, idx >= ni - n_wk) coincide,
    # trailing-edge node included
    nid = np.arange((n_j + 1) * (ni + 1)).reshape(n_j + 1, ni + 1)
    for i in range(n_wk + 1):
        nid[0, ni - i] = nid[0, i]
    used_ids = np.unique(nid)
    remap = -np.ones(nid.max() + 1, np.int64)
    remap[used_ids] = np.arange(used_ids.size)
    nid = remap[nid]
    xy = np.zeros((used_ids.size, 2))
    xy[nid.ravel()] = X.reshape(-1, 2)
    jj, ii = np.meshgrid(np.arange(n_j), np.arange(ni), indexing="ij")
    jj, ii = jj.ravel(), ii.ravel()
    cells4 = np.stack([nid[jj, ii], nid[jj, ii + 1], nid[jj + 1, ii + 1], nid[jj + 1, ii]], 1)
    # orient counter-clockwise
    P = xy[cells4]
    area2 = np.sum(P[:, :, 0] * np.roll(P[:, :, 1], -1, 1) - np.roll(P[:, :, 0], -1, 1) * P[:, :, 1], 1)
    cells4[area2 < 0] = cells4[area2 < 0][:, ::-1]
    tri_mask = eta[jj + 1] > quad_layer / far
    ptr, cn = _hybrid_cells(cells4.astype(np.int32), tri_mask)
    bn, bt, bvl = [], [], []
    a = math.radians(alpha_deg)
    uinf, vinf = uref * math.cos(a), uref * math.sin(a)
    k_inf = 1.5 * (intensity * uref) ** 2
    w_inf = k_inf / (nu * nut_ratio)
    for i in range(n_wk, ni - n_wk):
        bn.append((nid[0, i], nid[0, i + 1])); bt.append(BC_WALL); bvl.append((1.0, 0, 0, 0, 0))
    for i in range(ni):
        bn.append((nid[n_j, i], nid[n_j, i + 1])); bt.append(BC_FARFIELD)
        bvl.append((1.0, uinf, vinf, k_inf, w_inf))
    for j in (list(range(n_j))):
        bn.append((nid[j, 0], nid[j + 1, 0])); bt.append(BC_FARFIELD)
        bvl.append((1.0, uinf, vinf, k_inf, w_inf))
        bn.append((nid[j, ni], nid[j + 1, ni])); bt.append(BC_FARFIELD)
        bvl.append((1.0, uinf, vinf, k_inf, w_inf))
    m = Mesh(xy, ptr, cn, np.asarray(bn, np.int32), np.asarray(bt, np.int32),
             np.asarray(bvl, np.float64), name=f"naca0012_cmesh_{len(ptr) - 1}").normalized()
    n = m.n_cells
    return Case(m, nu=nu, cfl=cfl, sst=True, uref=uref, lref=1.0, alpha_deg=alpha_deg,
                rho=np.ones(n), u=np.full(n, uinf), v=np.full(n, vinf), k=np.full(n, k_inf),
                omega=np.full(n, w_inf), name=f"naca{n}_a{alpha_deg:g}")


def batched_sweep(seed: int = 5, n_cavity: int = 32, n_bfs: int = 4, n_naca: int = 12,
                  scale: float = 1.0) -> list[Case]:
    """The uneven multi-instance sweep: cavities 10k-40k triangles at Re 100-3200 (laminar),
    BFS 80k cells and NACA 0012 meshes of 50k-200k cells at angles 0-12 degrees (k-omega SST);
    every time step at CFL 0.5 of its own mesh.  ``scale`` multiplies every size (small test
    versions)."""
    rng = np.random.default_rng(seed)
    cases: list[Case] = []
    for i in range(n_cavity):
        n = int(round(math.exp(rng.uniform(math.log(10000), math.log(40000))) * scale))
        re = math.exp(rng.uniform(math.log(100.0), math.log(3200.0)))
        hb = 1.0 / max(8, int(round(math.sqrt(n) / 1.0)))
        cases.append(cavity_delaunay(h_boundary=hb, n_target=max(64, n), re=re, cfl=0.5,
                                     seed=1000 + i))
    for i in range(n_bfs):
        cases.append(bfs_hybrid(n_target=max(400, int(80000 * scale)), seed=2000 + i))
    for i in range(n_naca):
        n = int(rng.uniform(50000, 200000) * scale)
        al = float(rng.uniform(0.0, 12.0))
        cases.append(naca0012_cmesh(n_target=max(600, n), alpha_deg=al, seed=3000 + i))
    return cases
