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
  - the same boundary kinds on a 3 x 3 grid with alternate cells split into triangles (mixed
    triangles and quads);
  - a doubly periodic 2 x 2 quad box, where each cell meets its x-neighbour through two faces,
    one of them periodic;
  - a jittered periodic 3 x 3 box of triangles.

A second comparison restates the SST update of Step 1 as well (Sec. 2 with readings 7-10, the
constants from tests/golden/sst_constants.json).  It takes two turbulent steps on a jittered
3 x 3 mesh with all four boundary kinds:
  - limited upwind convection and central diffusion of k and omega, by faces;
  - the blending functions, production, cross diffusion and point-implicit destruction;
  - the eddy viscosity and tau = (nu + nu_t) / cs^2, which then drives the IMEX stages.

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

    def __init__(self, m: mg.Mesh, nu: float, dt: float, variant: int = 0):
        m = m.normalized()
        self.nu, self.dt, self.tau = nu, dt, nu / CS2
        self.variant = variant
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
                self.faces.append(dict(P=i, N=-1, n=n, l=length, x=mid, e=e,
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
        g = np.zeros((nc, f.shape[1], 2), dtype=f.dtype)
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
        if self.variant & 1:
            g = g * self.venkatakrishnan(f, fb, g)[:, :, None]
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

    def venkatakrishnan(self, f, fb, g):
        """Variant 1: limiter of each f_alpha's reconstruction per cell.  D1 is the distance to
        the max (min) over the cell, its face neighbours and its boundary values, D2 the
        increment to a face, eps^2 = A^(3/2); phi = min over faces of
        [(D1^2 + eps^2) D2 + 2 D2^2 D1] / [D1^2 + 2 D2^2 + D1 D2 + eps^2] / D2."""
        psi = np.ones_like(f)
        for i, faces in enumerate(self._cell_faces()):
            vals = np.array([f[i]] + [f[N] if N >= 0 else fb[q] for _, N, q in faces])
            hi, lo = vals.max(0), vals.min(0)
            e2 = self.area[i] ** 1.5
            for r, _, _ in faces:
                d2 = g[i] @ r
                with np.errstate(divide="ignore", invalid="ignore"):
                    d1 = np.where(d2 > 0, hi - f[i], lo - f[i])
                    phi = ((d1 ** 2 + e2) * d2 + 2 * d2 ** 2 * d1) / (d1 ** 2 + 2 * d2 ** 2 + d1 * d2 + e2) / d2
                psi[i] = np.where(d2 != 0, np.minimum(psi[i], phi), psi[i])
        return psi

    def local_steps(self, cfl):
        """Local time stepping: dt_i = cfl / max_alpha sum over the cell's faces of
        max(e_alpha . n_out, 0) dl / A_i, the forward-Euler limit of first-order upwinding."""
        out = np.zeros((len(self.area), 9))
        for F in self.faces:
            out[F["P"]] += np.maximum(E @ F["n"], 0.0) * F["l"]
            if F["N"] >= 0:
                out[F["N"]] += np.maximum(-(E @ F["n"]), 0.0) * F["l"]
        return cfl / (out.max(1) / self.area)

    def imex_step(self, f, tab, stage_tau=None):
        mt, mi = np.array(tab["m_tilde"]), np.array(tab["m"])
        nt, ni = np.array(tab["n_tilde"]), np.array(tab["n"])
        dt = np.reshape(self.dt, (-1, 1)) if np.ndim(self.dt) else self.dt
        tau = np.reshape(self.tau, (-1, 1)) if np.ndim(self.tau) else self.tau
        ga, gc = [], []
        latest = f
        for J in range(3):
            if stage_tau is not None:           # variant 4: SST re-solved before each stage
                tau = np.reshape(stage_tau(J, latest), (-1, 1))
            expl = f + dt * sum(mt[J, k] * ga[k] for k in range(J))
            eq = equilibrium(*macros(expl))     # collision invariants: moments of expl
            rhs = expl + dt * sum(mi[J, k] * gc[k] for k in range(J))
            z = dt * mi[J, J] / tau
            fJ = (rhs + z * eq) / (1.0 + z)
            latest = fJ
            gc.append((eq - fJ) / tau)
            ga.append(self.convection(fJ))
        return f + dt * sum(nt[J] * ga[J] + ni[J] * gc[J] for J in range(3))

    # ---------------------------------------------------------------- SST (Step 1)
    def sst_setup(self, m: mg.Mesh, sst: dict, uref: float, lref: float):
        """Constants, omega floor and the wall distance (centroid to nearest wall edge)."""
        self.K = sst
        self.wmin = 1e-12 * uref / lref
        m = m.normalized()
        segs = [m.xy[m.bedge_nodes[e]] for e in range(m.n_bedges) if m.bedge_type[e] == mg.BC_WALL]
        self.wd = np.full(len(self.area), 1e30)
        for i, c in enumerate(self.c):
            for a, b in segs:
                t = np.clip(np.dot(c - a, b - a) / np.dot(b - a, b - a), 0.0, 1.0)
                self.wd[i] = min(self.wd[i], float(np.hypot(*(a + t * (b - a) - c))))

    def _cell_faces(self):
        """Per cell: (midpoint offset from the centroid, neighbour or -1, face index)."""
        out = [[] for _ in self.area]
        for q, F in enumerate(self.faces):
            out[F["P"]].append((F["x"] - self.c[F["P"]], F["N"], q))
            if F["N"] >= 0:
                out[F["N"]].append((F["x"] - F["s"] - self.c[F["N"]], F["P"], q))
        return out

    def _f1_f2(self, k, w, d, cd):
        K, nu = self.K, self.nu
        a = np.sqrt(k) / (K["beta_star"] * w * d)
        b = 500.0 * nu / (w * d * d)
        arg1 = np.minimum(np.maximum(a, b), 4.0 * K["sigma_w2"] * k / (cd * d * d))
        arg2 = np.maximum(2.0 * a, b)
        return np.tanh(arg1 ** 4), np.tanh(arg2 ** 2)

    def sst_update(self, f, k, w, nut):
        """One step of k, omega from the macros of f (t^n); returns k, omega, nu_t, tau."""
        K, nu, dt = self.K, self.nu, self.dt
        _, u = macros(f)
        phi = np.column_stack([u, k, w])                  # u, v, k, omega per cell
        pb = []
        for F in self.faces:                               # boundary values (reading 7)
            if F["N"] >= 0:
                pb.append(None)
                continue
            P, v = F["P"], F["val"]
            if F["kind"] == mg.BC_WALL:
                pb.append(np.array([v[1], v[2], 0.0, 60.0 * nu / (K["beta1"] * self.wd[P] ** 2)]))
            elif F["kind"] == mg.BC_OUTLET:
                pb.append(phi[P].copy())
            else:
                pb.append(np.array([v[1], v[2], v[3], v[4]]))
        g = self.gradients(phi, pb)                        # [nc, 4, 2]
        cf = self._cell_faces()
        lim = np.ones((len(k), 2))                         # Barth-Jespersen for k, omega
        for i, faces in enumerate(cf):
            for c in (2, 3):
                vals = [phi[i, c]] + [phi[N, c] if N >= 0 else pb[q][c] for _, N, q in faces]
                lo, hi = min(vals), max(vals)
                for r, _, _ in faces:
                    d = g[i, c] @ r
                    ratio = (hi - phi[i, c]) / d if d > 0 else ((lo - phi[i, c]) / d if d < 0 else 1.0)
                    lim[i, c - 2] = min(lim[i, c - 2], ratio)
        gl = g[:, 2:4, :] * lim[:, :, None]                # limited gradients of k, omega
        s11, s22 = g[:, 0, 0], g[:, 1, 1]
        s12 = 0.5 * (g[:, 0, 1] + g[:, 1, 0])
        SS = s11 ** 2 + s22 ** 2 + 2.0 * s12 ** 2
        div = s11 + s22
        gkgw = (g[:, 2, :] * g[:, 3, :]).sum(1)
        cd = np.maximum(2.0 * K["sigma_w2"] / w * gkgw, 1e-20)
        f1, _ = self._f1_f2(k, w, self.wd, cd)
        sk = f1 * K["sigma_k1"] + (1 - f1) * K["sigma_k2"]
        sw = f1 * K["sigma_w1"] + (1 - f1) * K["sigma_w2"]
        conv = np.zeros((len(k), 2))                       # sum of un phi_up dl, per cell
        diff = np.zeros((len(k), 2))                       # sum of Gamma dphi/dn dl, per cell
        for q, F in enumerate(self.faces):
            P, N = F["P"], F["N"]
            rP = F["x"] - self.c[P]
            fromP = phi[P, 2:4] + gl[P] @ rP
            if N < 0:
                b = pb[q]
                un = b[:2] @ F["n"]
                up = fromP if un >= 0 else b[2:4]
                dist = np.hypot(*rP)
                gam = nu + np.array([sk[P], sw[P]]) * nut[P]
                dn = (b[2:4] - phi[P, 2:4]) / dist
                if self.variant & 2:            # + grad phi . (n - r / |r|)
                    dn = dn + g[P, 2:4] @ (F["n"] - rP / dist)
                conv[P] += un * up * F["l"]
                diff[P] += gam * dn * F["l"]
                continue
            xN = self.c[N] + F["s"]
            un = 0.5 * (u[P] + u[N]) @ F["n"]
            fromN = phi[N, 2:4] + gl[N] @ (F["x"] - xN)
            up = fromP if un >= 0 else fromN
            dist = np.hypot(*(xN - self.c[P]))
            gam = nu + 0.5 * (np.array([sk[P], sw[P]]) * nut[P] + np.array([sk[N], sw[N]]) * nut[N])
            flux = un * up * F["l"]
            dn = (phi[N, 2:4] - phi[P, 2:4]) / dist
            if self.variant & 2:                # + mean grad phi . (n - d / |d|)
                dn = dn + 0.5 * (g[P, 2:4] + g[N, 2:4]) @ (F["n"] - (xN - self.c[P]) / dist)
            dflux = gam * dn * F["l"]
            conv[P] += flux
            conv[N] -= flux
            diff[P] += dflux
            diff[N] -= dflux
        kap2 = K["kappa"] ** 2 / np.sqrt(K["beta_star"])
        gamma = f1 * (K["beta1"] / K["beta_star"] - K["sigma_w1"] * kap2) + \
            (1 - f1) * (K["beta2"] / K["beta_star"] - K["sigma_w2"] * kap2)
        shear = 2.0 * SS - 2.0 / 3.0 * div ** 2
        pk = nut * shear - 2.0 / 3.0 * k * div
        if self.variant & 8:                    # P_k <= 10 beta* omega k
            pk = np.minimum(pk, 10.0 * K["beta_star"] * w * k)
        pw = gamma * shear - np.where(nut > 0, 2.0 / 3.0 * gamma * k * div / np.where(nut > 0, nut, 1.0), 0.0)
        cross = 2.0 * (1 - f1) * K["sigma_w2"] / w * gkgw
        rk = (-conv[:, 0] + diff[:, 0]) / self.area + pk
        rw = (-conv[:, 1] + diff[:, 1]) / self.area + pw + cross
        beta = f1 * K["beta1"] + (1 - f1) * K["beta2"]
        k1 = np.maximum((k + dt * rk) / (1 + dt * K["beta_star"] * w), 0.0)
        w1 = (w + dt * rw) / (1 + dt * beta * w)
        w1 = np.where(w1 > self.wmin, w1, self.wmin)
        _, f2 = self._f1_f2(k1, w1, self.wd, np.full(len(k), 1e-20))
        nut1 = K["a1"] * k1 / np.maximum(K["a1"] * w1, np.sqrt(2.0 * SS) * f2)
        return k1, w1, nut1, (nu + nut1) / CS2

    def euler_step(self, f):
        dt = np.reshape(self.dt, (-1, 1)) if np.ndim(self.dt) else self.dt
        tau = np.reshape(self.tau, (-1, 1)) if np.ndim(self.tau) else self.tau
        return f + dt * (self.convection(f) + (equilibrium(*macros(f)) - f) / tau)


def _four_boundary_mesh(seed, n=2):
    """n x n jittered quads on the unit square: a wall below sliding at u = 0.05, a far field
    above, an inlet on the left and an outlet on the right."""
    xs = np.linspace(0.0, 1.0, n + 1)
    xy, cells, sides = mg.quad_grid(xs, xs, 0.25, seed)
    bn = np.concatenate([sides["bottom"], sides["top"], sides["left"], sides["right"]])
    kind = np.repeat(np.array([mg.BC_WALL, mg.BC_FARFIELD, mg.BC_INLET, mg.BC_OUTLET], np.int32), n)
    bv = np.zeros((4 * n, 5))
    bv[0:n] = [1.0, 0.05, 0.0, 0.0, 1.0]          # wall velocity
    bv[n:2 * n] = [1.02, 0.08, 0.01, 0.0, 1.0]    # far field
    bv[2 * n:3 * n] = [1.0, 0.1, -0.02, 0.0, 1.0]  # inlet velocity
    bv[3 * n:] = [0.98, 0.0, 0.0, 0.0, 1.0]       # outlet density
    return mg.Mesh(xy, np.arange(n * n + 1, dtype=np.int32) * 4, cells.ravel(), bn, kind, bv)


def _hybrid_mesh(seed):
    """3 x 3 jittered grid on the unit square, alternate cells split into two triangles (a
    mixed triangle / quad mesh), with the four boundary kinds of _four_boundary_mesh."""
    m = _four_boundary_mesh(seed, n=3)
    cells4 = m.cell_nodes.reshape(-1, 4)
    ptr, nodes = mg._hybrid_cells(cells4, np.arange(9) % 2 == 0)
    return mg.Mesh(m.xy, ptr, nodes, m.bedge_nodes, m.bedge_type, m.bedge_val)


MESHES = {
    "four_boundary_kinds": lambda: _four_boundary_mesh(11),
    "hybrid_3x3": lambda: _hybrid_mesh(13),
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


@pytest.mark.parametrize("scheme", [0, 1])
def test_local_time_steps_match_numpy_restatement(scheme):
    """Local time stepping: each cell advances with its own dt_i = cfl / rate_i."""
    m = MESHES["periodic_triangles_3x3"]().normalized()
    case = mg.Case(m, nu=0.01, cfl=0.5, local_dt=True)
    o = Oracle(case, scheme=scheme)
    r = Restated(m, 0.01, 0.0)
    r.dt = r.local_steps(0.5)
    assert np.abs(o.dt_cells() - r.dt).max() <= 1e-14 * r.dt.max()
    assert r.dt.max() > 1.2 * r.dt.min()        # the jittered cells do differ
    f0 = _state(m.n_cells, 5 + scheme)
    o.set_f(f0)
    o.step(1)
    with open(os.path.join(GOLD, "imex_tableau.json")) as fh:
        tab = json.load(fh)
    want = r.imex_step(f0, tab) if scheme == 0 else r.euler_step(f0)
    assert np.abs(o.get_f() - want).max() <= 1e-13 * np.abs(want).max()


def restated_forces(r, f, rho0, U, L, alpha_deg):
    """Reading 12 on the restatement: the wall force, the momentum flux sum over wall faces of
    sum_alpha e_alpha (e_alpha . n) f_{alpha,bc} dl with n out of the fluid; C_D and C_L are
    its components along and across the free stream at alpha, over 1/2 rho0 U^2 L."""
    force = 0.0
    for F in r.faces:
        if F["N"] < 0 and F["kind"] == mg.BC_WALL:
            force = force + E.T @ ((E @ F["n"]) * r.boundary_value(F, f)) * F["l"]
    a = np.radians(alpha_deg)
    q = 0.5 * rho0 * U * U * L
    return {"fx": force[0], "fy": force[1], "cd": (force[0] * np.cos(a) + force[1] * np.sin(a)) / q,
            "cl": (-force[0] * np.sin(a) + force[1] * np.cos(a)) / q}


@pytest.mark.parametrize("seeded", ["f0", "boundary_values"])
def test_complex_step_tangent_matches_the_restatement(seeded):
    """The oracle's complex-step build (its own tangent) against the same method applied to the
    restatement: seed f0, or the boundary values of every edge, with imaginary parts
    h d (h = 1e-30), take two IMEX steps, and compare d(F_x, F_y, C_D, C_L) = Im / h."""
    m = MESHES["four_boundary_kinds"]().normalized()
    U, L, alpha, h = 0.1, 0.7, 10.0, 1e-30
    case = mg.Case(m, nu=0.01, dt=0.04, uref=U, lref=L, alpha_deg=alpha)
    f0 = _state(m.n_cells, 3)
    rng = np.random.default_rng(41)
    df = rng.standard_normal(f0.shape) * 1e-3 if seeded == "f0" else None
    dbv = None
    if seeded == "boundary_values":
        dbv = np.zeros((m.n_bedges, 5))
        dbv[:, :3] = rng.standard_normal((m.n_bedges, 3)) * 1e-2
    o = Oracle(case, complex_step=True)
    o.set_f(f0)
    o.cs_seed(dbedge_val=dbv, df=df, h=h)
    o.step(2)
    _, der = o.cs_forces(h)
    r = Restated(m, 0.01, 0.04)
    f = f0.astype(complex) + (1j * h * df if df is not None else 0.0)
    if dbv is not None:
        for F in r.faces:
            if F["N"] < 0:
                F["val"] = F["val"] + 1j * h * dbv[F["e"]]
    with open(os.path.join(GOLD, "imex_tableau.json")) as fh:
        tab = json.load(fh)
    for _ in range(2):
        f = r.imex_step(f, tab)
    want = {k: float(np.imag(v)) / h for k, v in restated_forces(r, f, case.rho0, U, L, alpha).items()}
    scale = max(abs(v) for v in want.values())
    assert scale > 0
    for key, v in want.items():
        assert abs(der[key] - v) <= 1e-10 * scale, (key, der[key], v)


def test_wall_force_matches_numpy_restatement():
    """Reading 12 (restated_forces) after one IMEX step, at alpha = 10 degrees."""
    m = MESHES["four_boundary_kinds"]().normalized()
    U, L, alpha = 0.1, 0.7, 10.0
    case = mg.Case(m, nu=0.01, dt=0.04, uref=U, lref=L, alpha_deg=alpha)
    f0 = _state(m.n_cells, 3)
    o = Oracle(case)
    o.set_f(f0)
    o.step(1)
    r = Restated(m, 0.01, 0.04)
    with open(os.path.join(GOLD, "imex_tableau.json")) as fh:
        f = r.imex_step(f0, json.load(fh))
    want = restated_forces(r, f, case.rho0, U, L, alpha)
    got = o.forces()
    for key, v in want.items():
        assert abs(got[key] - v) <= 1e-13 * max(abs(v), 1e-3), (key, got[key], v)


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


def _sst_run(sst_constants, variant=0, w_scale=1.0, scheme=0, mesh="quads"):
    """Two SST steps of the oracle and of the restatement (with the given constants and reading
    variant) from the same seeded state; returns both (f, k, omega, nu_t) per step, the initial
    k and omega, and the two wall distances."""
    m = (_four_boundary_mesh(11, n=3) if mesh == "quads" else _hybrid_mesh(13)).normalized()
    nc = m.n_cells
    rng = np.random.default_rng(29)
    k0 = 1e-3 * (1.0 + rng.uniform(0, 1, nc))
    w0 = w_scale * (0.5 + rng.uniform(0, 1, nc))
    m.bedge_val[:, 3] = np.where(m.bedge_type == mg.BC_WALL, 0.0, 1.2e-3)   # k_b
    m.bedge_val[:, 4] = np.where(m.bedge_type == mg.BC_WALL, 1.0, 0.8)      # omega_b
    nu, dt = 1e-3, 0.04
    o = Oracle(mg.Case(m, nu=nu, dt=dt, sst=True, k=k0, omega=w0, uref=0.1, lref=1.0,
                       variant=variant), scheme=scheme)
    f0 = _state(nc, 7)
    o.set_f(f0)
    with open(os.path.join(GOLD, "imex_tableau.json")) as fh:
        tab = json.load(fh)
    r = Restated(m, nu, dt, variant)
    r.sst_setup(m, sst_constants, 0.1, 1.0)
    f, k, w, nut = f0, k0, w0, k0 / w0           # Step 0: nu_t = k / omega
    steps = []
    for _ in range(2):
        if variant & 4:
            # each stage re-solves the update from k, omega, nu_t of t^n with the macros of the
            # latest stage value (f^n, f^(1), f^(2)); the last solve gives t^{n+1}
            start, solved = (k, w, nut), {}

            def stage_tau(J, latest, start=start, solved=solved):
                solved["out"] = r.sst_update(latest, *start)
                return solved["out"][3]
            f = r.imex_step(f, tab, stage_tau)
            k, w, nut, _ = solved["out"]
        else:
            k, w, nut, r.tau = r.sst_update(f, k, w, nut)
            f = r.imex_step(f, tab) if scheme == 0 else r.euler_step(f)
        o.step(1)
        got = o.fields()
        steps.append(((o.get_f(), got["k"], got["omega"], got["nut"]), (f, k, w, nut)))
    return steps, (k0, w0), (r.wd, o.geometry()["wdist"])


def _sst_constants():
    with open(os.path.join(GOLD, "sst_constants.json")) as fh:
        return json.load(fh)


@pytest.mark.parametrize("scheme,mesh", [(0, "quads"), (1, "quads"), (0, "hybrid")])
def test_two_sst_steps_match_numpy_restatement(scheme, mesh):
    steps, (k0, w0), (wd, wd_oracle) = _sst_run(_sst_constants(), scheme=scheme, mesh=mesh)
    assert np.allclose(wd, wd_oracle, rtol=1e-14, atol=0)
    for got, want in steps:
        assert np.abs(got[0] - want[0]).max() <= 1e-13 * np.abs(want[0]).max()
        for name, g, v in zip(("k", "omega", "nut"), got[1:], want[1:]):
            assert np.abs(g - v).max() <= 1e-12 * np.abs(v).max(), name
    k, _, nut = steps[-1][1][1:]                   # the restatement after two steps
    assert np.abs(k - k0).max() > 1e-2 * k0.max() and np.abs(nut - k0 / w0).max() > 1e-2 * nut.max()


@pytest.mark.parametrize("name,value", [("sigma_w2", 0.85), ("sigma_k1", 0.86), ("beta1", 0.0755),
                                        ("kappa", 0.405)])
def test_sst_restatement_sees_a_changed_constant(name, value):
    """The SST comparison is sharp: a constant of Sec. 2 moved by about 1 % in the restatement
    moves k, omega or nu_t far above the tolerance."""
    K = _sst_constants()
    K[name] = value
    steps, _, _ = _sst_run(K)
    got, want = steps[-1]
    worst = max(np.abs(g - v).max() / np.abs(v).max() for g, v in zip(got[1:], want[1:]))
    assert worst > 1e-8, (name, worst)


@pytest.mark.parametrize("variant", [1, 2, 4, 8, 1 | 2 | 8])
def test_reading_variants_match_numpy_restatement(variant):
    """The reading variants, restated term by term:
      - 1: Venkatakrishnan limiter on grad f;
      - 2: non-orthogonal diffusion correction of k and omega;
      - 4: SST re-solved before every stage;
      - 8: Menter's production limiter.
    omega starts near 0.1-0.15 so that nu_t = k / omega is large and the production limiter
    acts.  Each variant must change the result (so it is exercised), and the oracle and the
    restatement must agree to the rounding level."""
    K = _sst_constants()
    steps, _, _ = _sst_run(K, variant=variant, w_scale=0.1)
    base, _, _ = _sst_run(K, variant=0, w_scale=0.1)
    for got, want in steps:
        assert np.abs(got[0] - want[0]).max() <= 1e-13 * np.abs(want[0]).max()
        for name, g, v in zip(("k", "omega", "nut"), got[1:], want[1:]):
            assert np.abs(g - v).max() <= 1e-12 * np.abs(v).max(), name
    moved = max(np.abs(a - b).max() / np.abs(b).max() for a, b in zip(steps[-1][1], base[-1][1]))
    assert moved > 1e-6, moved
