"""Whole-step pin on tiny meshes.  One laminar time step of the oracle (Steps 1-7 of Sec. 3.2,
both schemes) is compared with an independent NumPy restatement of the same equations:
  - the D2Q9 equilibrium;
  - least squares by np.linalg.lstsq rather than normal equations;
  - the flux by faces, each added to its two cells with opposite signs, rather than per cell;
  - the boundary values (readings 6 and 7);
  - the IMEX stages of Eqs. (sumimeximplicitnew), (fnewstage) and (imextwo) with the tableau
    printed after Eq. (imextwo) (tests/golden/imex_tableau.json), or the explicit step.

The meshes:
  - a 2 x 2 jittered quad mesh with all four boundary kinds: a moving wall, an inlet, an outlet
    and a far field;
  - a doubly periodic 2 x 2 quad box, where each cell meets its x-neighbour through two faces,
    one of them periodic;
  - a jittered periodic 3 x 3 box of triangles.

Initial states are equilibria of random density and velocity plus a random non-equilibrium
part, so every term of the step is active.  The restatement shares no code with the oracle; a
dropped term, a wrong sign, index or shift in either one shows up far above the 1e-13 rounding
level of this comparison.
"""
import json
import os

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1812_00394_gb300 import meshgen as mg

GOLD = os.path.join(os.path.dirname(__file__), "golden")
E = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], float)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
CS2 = 1.0 / 3.0


def equilibrium(rho, u):
    """f^eq_alpha = w_alpha rho [1 + 3 e.u + 9/2 (e.u)^2 - 3/2 |u|^2] per row (reading 1)."""
    rho = np.atleast_1d(rho)
    u = np.atleast_2d(u)
    eu = u @ E.T
    return W * rho[:, None] * (1.0 + 3.0 * eu + 4.5 * eu ** 2 - 1.5 * (u * u).sum(1)[:, None])


def macros(f):
    rho = f.sum(1)
    return rho, (f @ E) / rho[:, None]


class Restated:
    """Face-based finite-volume data of a mesh and the laminar FVLBM step on it."""

    def __init__(self, m: mg.Mesh, nu: float, dt: float):
        m = m.normalized()
        self.nu, self.dt, self.tau = nu, dt, nu / CS2
        nc = m.n_cells
        polys = [m.cell_nodes[m.cell_ptr[i]:m.cell_ptr[i + 1]] for i in range(nc)]
        self.area = np.zeros(nc)
        self.c = np.zeros((nc, 2))
        for i, p in enumerate(polys):   # shoelace area and centroid
            x, y = m.xy[p, 0], m.xy[p, 1]
            x1, y1 = np.roll(x, -1), np.roll(y, -1)
            cr = x * y1 - x1 * y
            a = 0.5 * cr.sum()
            self.area[i] = a
            self.c[i] = [((x + x1) * cr).sum() / (6 * a), ((y + y1) * cr).sum() / (6 * a)]
        sides = {}
        for i, p in enumerate(polys):
            for k in range(len(p)):
                a, b = int(p[k]), int(p[(k + 1) % len(p)])
                sides.setdefault(frozenset((a, b)), []).append((i, a, b))
        # faces: owner, neighbour (-1: boundary), neighbour image offset, unit normal out of the
        # owner, length, midpoint (owner's frame), boundary kind and values
        self.faces = []
        bedge = {frozenset(map(int, m.bedge_nodes[e])): e for e in range(m.n_bedges)}
        glued = {}
        for q, (ea, eb) in enumerate(m.periodic_pairs):
            glued[int(ea)] = (int(eb), m.periodic_shift[q])
            glued[int(eb)] = None
        for key, owners in sides.items():
            i, a, b = owners[0]
            t = m.xy[b] - m.xy[a]
            length = float(np.hypot(*t))
            n = np.array([t[1], -t[0]]) / length
            mid = 0.5 * (m.xy[a] + m.xy[b])
            if len(owners) == 2:
                self.faces.append(dict(P=i, N=owners[1][0], s=np.zeros(2), n=n, l=length, x=mid))
                continue
            e = bedge[key]
            if e in glued:
                if glued[e] is None:
                    continue                      # the partner edge carries this face
                eb, shift = glued[e]
                j = sides[frozenset(map(int, m.bedge_nodes[eb]))][0][0]
                self.faces.append(dict(P=i, N=j, s=-shift, n=n, l=length, x=mid))
            else:
                self.faces.append(dict(P=i, N=-1, n=n, l=length, x=mid,
                                       kind=int(m.bedge_type[e]), val=m.bedge_val[e]))

    def boundary_value(self, F, f):
        """f_{alpha,bc} on a boundary face from its cell P (readings 6, 7)."""
        fP = f[F["P"]][None, :]
        rP, uP = macros(fP)
        neq = fP - equilibrium(rP, uP)
        v = F["val"]
        if F["kind"] in (mg.BC_WALL, mg.BC_INLET):
            return (equilibrium(rP, v[1:3][None, :]) + neq)[0]
        if F["kind"] == mg.BC_OUTLET:
            return (equilibrium(np.array([v[0]]), uP) + neq)[0]
        incoming = (E @ F["n"]) < 0.0
        return np.where(incoming, equilibrium(np.array([v[0]]), v[1:3][None, :])[0], fP[0])

    def gradients(self, f, fb):
        """Unweighted least-squares gradient of each f_alpha from the face neighbours' centroids
        (periodic images) and the boundary faces' midpoints and values (reading 5)."""
        nc = f.shape[0]
        rows = [[] for _ in range(nc)]
        for F, vb in zip(self.faces, fb):
            P, N = F["P"], F["N"]
            if N < 0:
                rows[P].append((F["x"] - self.c[P], vb - f[P]))
            else:
                d = self.c[N] + F["s"] - self.c[P]
                rows[P].append((d, f[N] - f[P]))
                rows[N].append((-d, f[P] - f[N]))
        g = np.zeros((nc, 9, 2))
        for i in range(nc):
            D = np.array([r[0] for r in rows[i]])
            R = np.array([r[1] for r in rows[i]])
            g[i] = np.linalg.lstsq(D, R, rcond=None)[0].T
        return g

    def convection(self, f):
        """Gamma^a = -(1/A) sum over faces of (e.n) f_face dl, upwind linear reconstruction
        (Eq. (advection), reading 5); each interior face adds to its two cells."""
        fb = [self.boundary_value(F, f) if F["N"] < 0 else None for F in self.faces]
        g = self.gradients(f, fb)
        ga = np.zeros_like(f)
        for F, vb in zip(self.faces, fb):
            P, N = F["P"], F["N"]
            en = E @ F["n"]
            if N < 0:
                ga[P] -= en * vb * F["l"] / self.area[P]
                continue
            fromP = f[P] + g[P] @ (F["x"] - self.c[P])
            fromN = f[N] + g[N] @ (F["x"] - (self.c[N] + F["s"]))
            flux = en * np.where(en >= 0.0, fromP, fromN) * F["l"]
            ga[P] -= flux / self.area[P]
            ga[N] += flux / self.area[N]
        return ga

    def imex_step(self, f, tab):
        mt, mi = np.array(tab["m_tilde"]), np.array(tab["m"])
        nt, ni = np.array(tab["n_tilde"]), np.array(tab["n"])
        dt, tau = self.dt, self.tau
        ga, gc = [], []
        for J in range(3):
            expl = f + dt * sum(mt[J, k] * ga[k] for k in range(J))
            eq = equilibrium(*macros(expl))     # collision invariants: moments of expl
            rhs = expl + dt * sum(mi[J, k] * gc[k] for k in range(J))
            z = dt * mi[J, J] / tau
            fJ = (rhs + z * eq) / (1.0 + z)
            gc.append((eq - fJ) / tau)
            ga.append(self.convection(fJ))
        return f + dt * sum(nt[J] * ga[J] + ni[J] * gc[J] for J in range(3))

    def euler_step(self, f):
        return f + self.dt * (self.convection(f) + (equilibrium(*macros(f)) - f) / self.tau)


def _four_boundary_mesh(seed):
    xs = np.array([0.0, 0.5, 1.0])
    xy, cells, sides = mg.quad_grid(xs, xs, 0.25, seed)
    bn = np.concatenate([sides["bottom"], sides["top"], sides["left"], sides["right"]])
    kind = np.array([mg.BC_WALL] * 2 + [mg.BC_FARFIELD] * 2 + [mg.BC_INLET] * 2 + [mg.BC_OUTLET] * 2,
                    np.int32)
    bv = np.zeros((8, 5))
    bv[0:2] = [1.0, 0.05, 0.0, 0.0, 1.0]      # wall sliding at u = 0.05
    bv[2:4] = [1.02, 0.08, 0.01, 0.0, 1.0]    # far field
    bv[4:6] = [1.0, 0.1, -0.02, 0.0, 1.0]     # inlet velocity
    bv[6:8] = [0.98, 0.0, 0.0, 0.0, 1.0]      # outlet density
    return mg.Mesh(xy, np.arange(5, dtype=np.int32) * 4, cells.ravel(), bn, kind, bv)


MESHES = {
    "four_boundary_kinds": lambda: _four_boundary_mesh(11),
    "periodic_quads_2x2": lambda: mg.periodic_box(2, kind="quad"),
    "periodic_triangles_3x3": lambda: mg.periodic_box(3, kind="tri", jitter=0.2, seed=5),
}


def _state(nc, seed):
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.05 * rng.standard_normal(nc)
    u = 0.05 * rng.standard_normal((nc, 2))
    return equilibrium(rho, u) + 2e-3 * rng.standard_normal((nc, 9))


@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("name", list(MESHES))
def test_one_step_matches_numpy_restatement(name, scheme):
    m = MESHES[name]().normalized()
    nu, dt = 0.01, 0.04             # z = dt / tau = 1.2: both schemes stable
    case = mg.Case(m, nu=nu, dt=dt)
    f0 = _state(m.n_cells, 3 + scheme)
    o = Oracle(case, scheme=scheme)
    o.set_f(f0)
    o.step(1)
    got = o.get_f()
    r = Restated(m, nu, dt)
    with open(os.path.join(GOLD, "imex_tableau.json")) as fh:
        tab = json.load(fh)
    want = r.imex_step(f0, tab) if scheme == 0 else r.euler_step(f0)
    change = np.abs(want - f0).max()
    assert change > 1e-4                       # the step does move the state
    assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max(), np.abs(got - want).max()


def test_restatement_sees_a_planted_term():
    """The comparison is sharp: dropping the collision's tableau weight m_33 from the
    restatement (one coefficient of the printed tableau) moves it far above tolerance."""
    m = MESHES["four_boundary_kinds"]().normalized()
    case = mg.Case(m, nu=0.01, dt=0.04)
    f0 = _state(m.n_cells, 3)
    o = Oracle(case)
    o.set_f(f0)
    o.step(1)
    with open(os.path.join(GOLD, "imex_tableau.json")) as fh:
        tab = json.load(fh)
    tab["m"][2][2] = 0.25
    want = Restated(m, 0.01, 0.04).imex_step(f0, tab)
    assert np.abs(o.get_f() - want).max() > 1e-6
