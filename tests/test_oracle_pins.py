"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Every check here compares the oracle with something other than itself: a closed form, an
invariant of the lattice or of the scheme, a textbook flow, or a value printed in the paper
(golden fixtures under tests/golden/).  A plausible slip anywhere in the oracle -- a dropped
term, a wrong sign, a swapped tableau entry, a transposed gradient -- fails one of them.
"""
import dataclasses
import json
import math
import os

import numpy as np
import pytest

from oracle.oracle import Oracle, feq, sst_point
from paper_1812_00394_gb300 import meshgen as mg

GOLD = os.path.join(os.path.dirname(__file__), "golden")
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], float)
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], float)
CS2 = 1.0 / 3.0


def _gold(name):
    with open(os.path.join(GOLD, name)) as fh:
        return json.load(fh)


def _box_at_rest(n=12, kind="tri", jitter=0.25, seed=3):
    """Closed unit box, all walls at rest, jittered interior nodes."""
    xs = np.linspace(0, 1, n + 1)
    xy, cells, sides = mg.quad_grid(xs, xs, jitter, seed)
    cells = mg.split_quads(cells) if kind == "tri" else cells
    bn = np.concatenate([sides["bottom"], sides["right"], sides["top"], sides["left"]])
    ptr = np.arange(cells.shape[0] + 1, dtype=np.int32) * cells.shape[1]
    bv = np.zeros((bn.shape[0], 5))
    bv[:, 0] = 1.0
    return mg.Mesh(xy, ptr, cells.ravel(), bn, np.zeros(bn.shape[0], np.int32), bv).normalized()


# ----------------------------------------------------------------- equilibrium (D2Q9)
@pytest.mark.parametrize("rho,u,v", [(1.0, 0.0, 0.0), (1.3, 0.1, -0.05), (0.7, -0.08, 0.11)])
def test_feq_moments_closed_form(rho, u, v):
    """Sum f^eq = rho, sum e f^eq = rho u, sum e e f^eq = cs^2 rho I + rho u u (D2Q9 isotropy)."""
    f = feq(rho, u, v)
    assert abs(f.sum() - rho) < 1e-15
    assert abs((EX * f).sum() - rho * u) < 1e-15
    assert abs((EY * f).sum() - rho * v) < 1e-15
    assert abs((EX * EX * f).sum() - (CS2 * rho + rho * u * u)) < 1e-15
    assert abs((EY * EY * f).sum() - (CS2 * rho + rho * v * v)) < 1e-15
    assert abs((EX * EY * f).sum() - rho * u * v) < 1e-15


def test_feq_rest_weights():
    """At rest f^eq / rho are the D2Q9 weights 4/9, 1/9, 1/36 (Qian et al.)."""
    f = feq(2.0, 0.0, 0.0) / 2.0
    assert np.allclose(f, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, rtol=0, atol=1e-16)


# ----------------------------------------------------------------- IMEX tableau
def test_golden_tableau_order_conditions():
    """The printed tableau (Sec. 3.1) is second order: sum n = 1 and b.c = 1/2 for all four
    explicit/implicit pairings; the implicit part is stiffly accurate (last row of m = n)."""
    t = _gold("imex_tableau.json")
    mt, m = np.array(t["m_tilde"]), np.array(t["m"])
    nt, n = np.array(t["n_tilde"]), np.array(t["n"])
    ct, c = mt.sum(1), m.sum(1)
    assert abs(nt.sum() - 1) < 1e-15 and abs(n.sum() - 1) < 1e-15
    for b in (nt, n):
        for cc in (ct, c):
            assert abs(b @ cc - 0.5) < 1e-15
    assert np.allclose(m[2], n)


def _relaxation_factor_from_tableau(z):
    """Stability function of the implicit part: R(z) = 1 - z n^T (I + z m)^{-1} 1."""
    t = _gold("imex_tableau.json")
    m, n = np.array(t["m"]), np.array(t["n"])
    return 1.0 - z * n @ np.linalg.solve(np.eye(3) + z * m, np.ones(3))


@pytest.mark.parametrize("z", [0.5, 5.0, 50.0, 500.0])
def test_imex_relaxation_factor(z):
    """A uniform field in a closed box at rest has Gamma^a = 0, so one step multiplies the
    non-equilibrium part by the stability function of the printed implicit tableau.  This pins
    Eq. (fnewstage), the collision term and Eq. (imextwo) stage by stage."""
    m = _box_at_rest()
    dt = 0.01                                  # convective CFL ~ 0.25: round-off stays put
    nu = CS2 * dt / z
    case = mg.Case(m, nu=nu, dt=dt)
    o = Oracle(case)
    eq = feq(1.0, 0.0, 0.0)
    w = eq.copy()
    delta = 1e-3 * w * (EX ** 2 - EY ** 2)     # zero mass and momentum: pure non-equilibrium
    f0 = np.tile(eq + delta, (o.n_cells, 1))
    o.set_f(f0)
    o.step(1)
    f1 = o.get_f()
    R = _relaxation_factor_from_tableau(z)
    assert abs(R - (1 - 5 * z / 12) / ((1 + z / 4) * (1 + z / 3))) < 1e-14
    # Eq. (imextwo) adds dt/tau-weighted collision terms, so a rounding of f^(J) is scaled by ~z
    np.testing.assert_allclose(f1 - eq, np.tile(R * delta, (o.n_cells, 1)), rtol=0,
                               atol=1e-16 * (10 + z))


def test_moment_elimination():
    """After Eq. (fnewstage) every stage value carries the moments of Eq. (sumimeximplicitnew)."""
    case = mg.cavity_quad(16, re=100.0)
    o = Oracle(case)
    o.step(5)
    assert o.moment_defect() < 1e-15


# ----------------------------------------------------------------- gradient and flux
@pytest.mark.parametrize("kind", ["quad", "tri"])
def test_gradient_exact_on_linear_fields(kind):
    """The least-squares gradient reproduces a linear field exactly, interior and boundary."""
    m = _box_at_rest(10, kind, jitter=0.3, seed=11)
    o = Oracle(mg.Case(m, nu=1e-3, dt=1e-3))
    g = o.geometry()
    a, bx, by = 0.3, -1.7, 2.4
    phi = a + bx * g["cx"] + by * g["cy"]
    mid = 0.5 * (m.xy[m.bedge_nodes[:, 0]] + m.xy[m.bedge_nodes[:, 1]])
    phib = a + bx * mid[:, 0] + by * mid[:, 1]
    grad = o.gradient(phi, phib)
    np.testing.assert_allclose(grad[:, 0], bx, atol=1e-12)
    np.testing.assert_allclose(grad[:, 1], by, atol=1e-12)


def test_geometry_closed_forms():
    """Cell areas tile the unit square; on a uniform quad mesh the centroids are the cell
    centres and the wall distance is min(x, 1-x, y, 1-y)."""
    case = mg.cavity_quad(8)
    o = Oracle(case)
    g = o.geometry()
    assert abs(g["area"].sum() - 1.0) < 1e-14
    h = 1.0 / 8
    ii, jj = np.meshgrid(np.arange(8), np.arange(8), indexing="xy")
    np.testing.assert_allclose(g["cx"], (ii.ravel() + 0.5) * h, atol=1e-15)
    np.testing.assert_allclose(g["cy"], (jj.ravel() + 0.5) * h, atol=1e-15)
    d = np.minimum.reduce([g["cx"], 1 - g["cx"], g["cy"], 1 - g["cy"]])
    np.testing.assert_allclose(g["wdist"], d, atol=1e-15)
    tri = Oracle(mg.Case(_box_at_rest(9, "tri", 0.3, 5), nu=1e-3, dt=1e-3)).geometry()
    assert abs(tri["area"].sum() - 1.0) < 1e-14


@pytest.mark.parametrize("kind", ["quad", "tri"])
def test_free_stream_preserved(kind):
    """A uniform equilibrium f^eq(rho0, U) on a periodic jittered mesh is a fixed point: the
    face sums of Eq. (advection) over a closed cell vanish and the collision is zero."""
    m = mg.periodic_box(10, kind, jitter=0.3, seed=2)
    o = Oracle(mg.Case(m, nu=1e-3, cfl=0.5))
    f0 = np.tile(feq(1.0, 0.08, -0.05), (o.n_cells, 1))
    o.set_f(f0)
    assert np.abs(o.convection(f0)).max() < 1e-13
    o.step(10)
    assert np.abs(o.get_f() - f0).max() < 1e-14


def _advection_error(n, kind):
    m = mg.periodic_box(n, kind)
    o = Oracle(mg.Case(m, nu=1e30, cfl=0.5))   # tau -> infinity: collision off, pure transport
    g = o.geometry()
    w = feq(1.0, 0.0, 0.0)

    def exact(t):
        X = g["cx"][:, None] - EX[None, :] * t
        Y = g["cy"][:, None] - EY[None, :] * t
        return w[None, :] * (1 + 0.1 * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y))
    o.set_f(exact(0.0))
    nst = int(round(0.25 / o.dt))
    o.step(nst)
    return math.sqrt(np.mean((o.get_f() - exact(nst * o.dt)) ** 2))


@pytest.mark.parametrize("kind", ["quad", "tri"])
def test_pure_advection_second_order(kind):
    """Collision off, each f_alpha is transported at e_alpha; the explicit RK part of the
    tableau with the upwind linear reconstruction converges at second order."""
    e = [_advection_error(n, kind) for n in (16, 32, 64)]
    rates = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert min(rates) > 1.85, (e, rates)


# ----------------------------------------------------------------- conservation, Couette
def test_cavity_mass_conservation():
    """Closed cavity: interior fluxes telescope, wall faces carry no mass (u_w . n = 0) and the
    collision conserves mass, so sum rho A is constant up to the rounding of f itself."""
    case = mg.cavity_quad(32, re=400.0)
    o = Oracle(case)
    m0 = o.mass()
    o.step(400)
    assert abs(o.mass() - m0) / m0 < 400 * 1e-15


@pytest.mark.parametrize("kind,n,tol", [("quad", 16, 1e-11), ("tri", 16, 5e-5)])
def test_couette_profile_and_wall_shear(kind, n, tol):
    """Plane Couette flow (periodic in x, lid at U): the steady profile is u = U y / H, and the
    tangential force on the moving wall is -mu U / H per unit length with mu = rho nu and
    tau = nu / cs^2 (Eq. turbtau without eddy viscosity)."""
    U, H, nu = 0.1, 1.0, 0.05
    m = mg.couette_channel(4, n, U=U, H=H, Lx=1.0, kind=kind)
    o = Oracle(mg.Case(m, nu=nu, cfl=0.5, uref=U))
    o.step(int(3 * H * H / nu / o.dt))
    g, fl = o.geometry(), o.fields()
    err = math.sqrt(np.mean((fl["u"] - U * g["cy"] / H) ** 2)) / U
    assert err < tol
    fr = o.forces(per_edge=True)
    top = (m.bedge_type == mg.BC_WALL) & (m.bedge_val[:, 1] > 0)
    assert abs(fr["fx_edge"][top].sum() - (-nu * U / H * 1.0)) < 20 * tol * nu * U / H + 1e-13


def test_couette_second_order_on_triangles():
    U, H, nu = 0.1, 1.0, 0.05
    errs = []
    for n in (8, 16):
        m = mg.couette_channel(4, n, U=U, H=H, Lx=1.0, kind="tri")
        o = Oracle(mg.Case(m, nu=nu, cfl=0.5, uref=U))
        o.step(int(3 * H * H / nu / o.dt))
        g, fl = o.geometry(), o.fields()
        errs.append(math.sqrt(np.mean((fl["u"] - U * g["cy"] / H) ** 2)))
    assert math.log2(errs[0] / errs[1]) > 1.8, errs


def test_forces_fluid_at_rest():
    """Fluid at rest at uniform rho: the wall force is the pressure cs^2 rho times the wall
    length, along the outward normal of the fluid; the net force on a closed box is zero."""
    m = _box_at_rest(8, "tri", 0.2, 4)
    rho = 1.2
    case = mg.Case(m, nu=1e-3, dt=1e-3, rho=np.full(m.n_cells, rho))
    o = Oracle(case)
    fr = o.forces(per_edge=True)
    assert abs(fr["fx"]) < 1e-15 and abs(fr["fy"]) < 1e-15
    mid = 0.5 * (m.xy[m.bedge_nodes[:, 0]] + m.xy[m.bedge_nodes[:, 1]])
    left = mid[:, 0] < 1e-12
    assert abs(fr["fx_edge"][left].sum() - (-CS2 * rho * 1.0)) < 1e-14
    assert abs(fr["fy_edge"][left].sum()) < 1e-15


# ----------------------------------------------------------------- SST
def test_golden_sst_constants_derived():
    """C_w1, C_w2 from the printed constants (Sec. 2): the standard values 0.5532 and 0.4404."""
    c = _gold("sst_constants.json")
    cw1 = c["beta1"] / c["beta_star"] - c["sigma_w1"] * c["kappa"] ** 2 / math.sqrt(c["beta_star"])
    cw2 = c["beta2"] / c["beta_star"] - c["sigma_w2"] * c["kappa"] ** 2 / math.sqrt(c["beta_star"])
    assert abs(cw1 - 0.5532) < 1e-4 and abs(cw2 - 0.4404) < 1e-4


def test_sst_point_limits():
    """Limits of the blending functions: far from walls f1 = f2 = 0 and nu_t = k / omega; at
    a wall f1 = f2 = 1; with large strain nu_t = a1 k / S; CD_kw floors at 1e-20."""
    nu = 1e-5
    far = sst_point(1e-4, 10.0, 1e6, (0, 0), (0, 0), 0.0, nu)
    assert far["f1"] < 1e-30 and far["f2"] < 1e-15
    assert abs(far["nut"] - 1e-4 / 10.0) < 1e-18
    assert far["cdkw"] == 1e-20
    near = sst_point(1e-4, 10.0, 1e-6, (0, 0), (0, 0), 0.0, nu)
    assert near["f1"] == 1.0 and near["f2"] == 1.0
    strained = sst_point(1e-4, 10.0, 1e-6, (0, 0), (0, 0), 1e3, nu)
    assert abs(strained["nut"] - 0.31 * 1e-4 / 1e3) < 1e-18
    opp = sst_point(1e-4, 10.0, 1.0, (1.0, 0.0), (-1.0, 0.0), 0.0, nu)
    assert opp["cdkw"] == 1e-20
    pos = sst_point(1e-4, 10.0, 1.0, (1.0, 0.0), (2.0, 0.0), 0.0, nu)
    assert abs(pos["cdkw"] - 2 * 0.856 / 10.0 * 2.0) < 1e-15


def test_sst_point_values_with_each_branch_active():
    """Blending functions and eddy viscosity of Sec. 2 at points built so that each branch of
    arg1 = min(max(a, b), c) is the active one in turn, with round numbers:
      - a = sqrt(k) / (beta* omega d) = 0.9 / 1.8 = 0.5, the turbulent length-scale ratio;
      - b = 500 nu / (omega d^2) = 0.5, the viscous ratio;
      - c = 4 sigma_w2 k / (CD d^2) = 0.25 with CD = 2 sigma_w2 grad k . grad omega / omega.
    So f1 = tanh(arg1^4) and f2 = tanh(arg2^2), with arg2 = max(2a, b), are tanh of 1/16,
    1/256, 1/4 or 1.  nu_t = a1 k / max(a1 omega, S f2) is k / omega unless the strain term is
    larger.  A wrong constant (0.09, 500, 0.856, 0.31), power or factor 2 moves a value by far
    more than the rounding of these few operations."""
    nu, rel = 1e-5, 1e-13

    def close(x, y):
        return abs(x - y) <= rel * abs(y)

    # a active: k = 0.81, omega = 10, d = 2 -> a = 0.5, b = 1.25e-4, c = inf (CD at its floor)
    A = sst_point(0.81, 10.0, 2.0, (0, 0), (0, 0), 0.0, nu)
    assert close(A["f1"], math.tanh(0.5 ** 4)) and close(A["f2"], math.tanh(1.0))
    assert close(A["nut"], 0.081) and A["cdkw"] == 1e-20
    # b active: nu = 1e-4, omega = 10, d = 0.1 -> b = 0.5; k = 8.1e-5 -> a = 0.1, arg2 = 0.5
    B = sst_point(8.1e-5, 10.0, 0.1, (0, 0), (0, 0), 0.0, 1e-4)
    assert close(B["f1"], math.tanh(0.5 ** 4)) and close(B["f2"], math.tanh(0.25))
    # c active: the point of A with grad k = (1.8, 0), grad omega = (9, 0):
    # CD = 2 (0.856) (16.2) / 10 = 2.77344 and c = 4 (0.856) (0.81) / (2.77344 * 4) = 0.25
    C = sst_point(0.81, 10.0, 2.0, (1.8, 0.0), (9.0, 0.0), 0.0, nu)
    assert close(C["cdkw"], 2.77344)
    assert close(C["f1"], math.tanh(0.25 ** 4)) and close(C["f2"], math.tanh(1.0))
    # strain-limited eddy viscosity: S f2 = 10 tanh(1) > a1 omega = 3.1
    D = sst_point(0.81, 10.0, 2.0, (0, 0), (0, 0), 10.0, nu)
    assert close(D["nut"], 0.31 * 0.81 / (10.0 * math.tanh(1.0)))


def test_sst_homogeneous_decay():
    """Homogeneous, unstrained turbulence far from walls: d omega/dt = -beta2 omega^2 and
    dk/dt = -beta* omega k, with closed forms omega = w0/(1 + beta2 w0 t) and
    k = k0 (1 + beta2 w0 t)^(-beta*/beta2).  The point-implicit update reproduces omega
    exactly and converges to k at first order in dt."""
    m = mg.periodic_box(4, "quad")
    k0, w0, nu = 1e-3, 2.0, 1e-4
    T = 5.0
    errs = []
    for nst in (50, 100, 200):
        case = mg.Case(m, nu=nu, dt=T / nst, sst=True, k=np.full(16, k0), omega=np.full(16, w0))
        o = Oracle(case)
        o.step(nst)
        fl = o.fields()
        w_ex = w0 / (1 + 0.0828 * w0 * T)
        k_ex = k0 * (1 + 0.0828 * w0 * T) ** (-0.09 / 0.0828)
        np.testing.assert_allclose(fl["omega"], w_ex, rtol=1e-12)
        errs.append(abs(fl["k"][0] - k_ex) / k_ex)
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(0.9 < r < 1.1 for r in rates), (errs, rates)


def test_sst_with_zero_k_is_laminar():
    """k = 0 everywhere and on every boundary: nu_t = 0, tau = nu / cs^2, and the coupled step
    equals the laminar step bit for bit."""
    case = mg.cavity_quad(12, re=200.0)
    a = Oracle(case)
    lam = mg.Case(case.mesh, nu=case.nu, cfl=case.cfl, rho=case.rho, sst=True,
                  k=np.zeros(case.mesh.n_cells), omega=np.full(case.mesh.n_cells, 5.0))
    b = Oracle(lam)
    a.step(20)
    b.step(20)
    assert np.array_equal(a.get_f(), b.get_f())
    assert np.all(b.fields()["nut"] == 0.0)


# ----------------------------------------------------------------- explicit Euler (Part I)
@pytest.mark.parametrize("z", [0.5, 1.5, 2.5])
def test_euler_relaxation_factor(z):
    """The explicit scheme of Part I multiplies f^neq of a uniform field by 1 - z per step: it is
    stable only for dt < 2 tau (Sec. 3.1), which the IMEX tableau removes (R(z) -> 0)."""
    m = _box_at_rest()
    dt = 0.01
    o = Oracle(mg.Case(m, nu=CS2 * dt / z, dt=dt), scheme=1)
    eq = feq(1.0, 0.0, 0.0)
    delta = 1e-3 * eq * (EX ** 2 - EY ** 2)
    o.set_f(np.tile(eq + delta, (o.n_cells, 1)))
    o.step(1)
    np.testing.assert_allclose(o.get_f() - eq, np.tile((1 - z) * delta, (o.n_cells, 1)),
                               rtol=0, atol=1e-16 * (10 + z))


def test_euler_couette_matches_imex_steady_state():
    """Both integrators have the same steady state (the spatial operator is shared): Couette
    flow (CFL 0.5, dt = 0.28 tau) converges to u = U y / H with the explicit scheme too."""
    U, H, nu = 0.1, 1.0, 0.05
    m = mg.couette_channel(4, 8, U=U, H=H, Lx=1.0)
    o = Oracle(mg.Case(m, nu=nu, cfl=0.5, uref=U), scheme=1)
    o.step(int(3 * H * H / nu / o.dt))
    g, fl = o.geometry(), o.fields()
    assert np.abs(fl["u"] - U * g["cy"] / H).max() < 1e-9


# ----------------------------------------------------------------- local time stepping
def test_local_dt_closed_form_on_rectangles():
    """Local time stepping (steady-state acceleration, not in the paper): dt_i = CFL * limit_i
    with limit_i = 1 / max_alpha sum_m max(e_alpha . n_m, 0) dl_m / A_i.  On an hx x hy
    rectangle the maximum is the diagonal velocity, 1/hx + 1/hy, so dt_i = CFL hx hy/(hx + hy);
    the global dt is the smallest dt_i."""
    m = mg.couette_channel(5, 9, stretch=1.4)
    cfl = 0.7
    o = Oracle(mg.Case(m, nu=0.01, cfl=cfl, local_dt=True))
    P = m.xy[m.cell_nodes.reshape(-1, 4)]
    hx = P[:, :, 0].max(1) - P[:, :, 0].min(1)
    hy = P[:, :, 1].max(1) - P[:, :, 1].min(1)
    want = cfl * hx * hy / (hx + hy)
    np.testing.assert_allclose(o.dt_cells(), want, rtol=1e-13, atol=0)
    assert o.dt == o.dt_cells().min()
    assert want.max() / want.min() > 5        # the stretching really spreads the steps
    g = Oracle(mg.Case(m, nu=0.01, cfl=cfl))
    assert g.dt == o.dt and np.all(g.dt_cells() == g.dt)


def _separate_boxes(sides):
    """Disconnected closed square cells of the given side lengths, all edges walls at rest."""
    xy, cells, bn = [], [], []
    x0 = 0.0
    for k, h in enumerate(sides):
        xy += [(x0, 0.0), (x0 + h, 0.0), (x0 + h, h), (x0, h)]
        c = [4 * k, 4 * k + 1, 4 * k + 2, 4 * k + 3]
        cells.append(c)
        bn += [(c[0], c[1]), (c[1], c[2]), (c[2], c[3]), (c[3], c[0])]
        x0 += h + 0.5
    nb = len(bn)
    bv = np.zeros((nb, 5))
    bv[:, 0] = 1.0
    return mg.Mesh(np.array(xy), np.arange(len(sides) + 1, dtype=np.int32) * 4,
                   np.array(cells, np.int32).ravel(), np.array(bn, np.int32),
                   np.zeros(nb, np.int32), bv).normalized()


def test_local_dt_relaxation_factor_per_cell():
    """Isolated closed cells of different sizes holding a uniform non-equilibrium field
    (Gamma^a = 0 in each): with local time steps every cell multiplies its non-equilibrium
    part by R(z_i), z_i = dt_i / tau, the stability function of the printed tableau at its
    own step, and dt_i = CFL h_i / 2 for a square of side h_i."""
    sides = [0.05, 0.1, 0.3, 1.0]
    m = _separate_boxes(sides)
    nu, cfl = 2e-4, 2.0
    o = Oracle(mg.Case(m, nu=nu, cfl=cfl, local_dt=True))
    dti = o.dt_cells()
    np.testing.assert_allclose(dti, cfl * np.array(sides) / 2, rtol=1e-14)
    eq = feq(1.0, 0.0, 0.0)
    delta = 1e-3 * eq * (EX ** 2 - EY ** 2)
    o.set_f(np.tile(eq + delta, (o.n_cells, 1)))
    o.step(1)
    f1 = o.get_f()
    for i in range(o.n_cells):
        z = dti[i] / (nu / CS2)
        R = _relaxation_factor_from_tableau(z)
        np.testing.assert_allclose(f1[i] - eq, R * delta, rtol=0, atol=1e-16 * (10 + z))


def test_local_dt_on_uniform_mesh_matches_global():
    """On a uniform quad mesh every cell has the same limit, so local stepping is the global
    step (up to the last bit of each cell's own limit)."""
    case = mg.cavity_quad(12, re=400.0)
    a = Oracle(case)
    b = Oracle(dataclasses.replace(case, local_dt=True))
    assert np.abs(b.dt_cells() / a.dt - 1).max() < 1e-14
    a.step(10)
    b.step(10)
    assert np.abs(a.get_f() - b.get_f()).max() < 1e-13


def test_local_dt_needs_cfl():
    m = _box_at_rest(4)
    with pytest.raises(ValueError):
        Oracle(mg.Case(m, nu=1e-3, dt=1e-3, local_dt=True))


def test_local_dt_accelerates_steady_couette():
    """Stretched Couette channel (row heights x1.25 per row, 16 rows): the global step is set
    by the thinnest row; local steps let every row move at its own limit.  Both reach a steady
    state; local stepping needs several times fewer steps, and its steady profile differs from
    the global one only at the level of the scheme's own dependence on the step (the IMEX
    fixed point moves with dt; 2.1e-5 U here)."""
    U, H, nu = 0.1, 1.0, 0.02
    m = mg.couette_channel(4, 16, U=U, H=H, stretch=1.25)
    out = {}
    for local in (False, True):
        o = Oracle(mg.Case(m, nu=nu, cfl=0.5, uref=U, local_dt=local))
        n = 0
        while o.residual() > 1e-12 or n == 0:
            o.step(500)
            n += 500
            assert n <= 40000
        out[local] = (n, o.fields()["u"], o.geometry()["cy"])
    (ng, ug, cy), (nl, ul, _) = out[False], out[True]
    assert np.abs(ug - U * cy / H).max() < 1e-8 * U       # global: the exact linear profile
    assert nl * 5 < ng
    assert np.abs(ul - ug).max() < 5e-5 * U


# ----------------------------------------------------------------- reading variants
def test_limiter_variant_closed_forms():
    """Variant 1 (Venkatakrishnan limiter on the reconstruction of f, a reading that Sec. 3.2
    leaves open).  For a linear field on uniform quads an interior face sees an increment D2
    half of the neighbour difference D1 (ratio 2), where the limiter function is exactly 1 for
    any smoothing e2; a cell on the x boundary sees its face value as the extremum (ratio 1),
    where it is (3 D2^2 + e2) / (4 D2^2 + e2) with D2 = b h / 2 and e2 = h^3."""
    n, b = 10, 0.7
    m = _box_at_rest(n, "quad", 0.0, 0)
    o = Oracle(mg.Case(m, nu=1e-3, dt=1e-3))
    g = o.geometry()
    phi = 0.3 + b * g["cx"]
    mid = 0.5 * (m.xy[m.bedge_nodes[:, 0]] + m.xy[m.bedge_nodes[:, 1]])
    phib = 0.3 + b * mid[:, 0]
    psi = o.limiter(phi, phib)
    h = 1.0 / n
    xb = (g["cx"] < h) | (g["cx"] > 1 - h)
    np.testing.assert_allclose(psi[~xb], 1.0, rtol=0, atol=1e-14)
    d2, e2 = b * h / 2, h ** 3
    np.testing.assert_allclose(psi[xb], (3 * d2 ** 2 + e2) / (4 * d2 ** 2 + e2), rtol=1e-12)


def test_limiter_variant_changes_only_when_on():
    """Variant 1 off is the default path bit for bit; on, a smooth cavity flow changes little
    (the limiter acts near extrema only)."""
    case = mg.cavity_quad(16, re=400.0)
    a, b = Oracle(case), Oracle(dataclasses.replace(case, variant=1))
    c = Oracle(dataclasses.replace(case, variant=0))
    for x in (a, b, c):
        x.step(30)
    assert np.array_equal(a.get_f(), c.get_f())
    ua, ub = a.fields()["u"], b.fields()["u"]
    assert 0 < np.abs(ua - ub).max() < 0.05 * np.abs(ua).max()


def test_nonorthogonal_variant_linear_k_has_no_net_diffusion():
    """Variant 2 (non-orthogonal correction of the SST diffusion): the face-normal gradient
    (k_j - k_i)/|d| + mean grad k . (n - d/|d|) is exact for a linear k, so with u = 0 the
    diffusive fluxes of a linear k cancel around every interior cell (up to the variation of
    the coefficient through nu_t = k / omega ~ 1e-4 nu) and k only decays; without the
    correction the skewed triangles leave a net flux of the order of nu |grad k| / h."""
    n = 14
    xs = np.linspace(0, 1, n + 1)
    xy, cells, sides = mg.quad_grid(xs, xs, 0.3, 5)
    cells = mg.split_quads(cells)
    bn = np.concatenate([sides["bottom"], sides["right"], sides["top"], sides["left"]])
    bv = np.zeros((bn.shape[0], 5))
    bv[:, 0] = 1.0
    m = mg.Mesh(xy, np.arange(cells.shape[0] + 1, dtype=np.int32) * 3, cells.ravel(), bn,
                np.zeros(bn.shape[0], np.int32), bv).normalized()
    g = Oracle(mg.Case(m, nu=1e-2, dt=1e-3)).geometry()
    k = 1e-3 * (1 + g["cx"] + 0.5 * g["cy"])
    w = np.full(m.n_cells, 1e3)
    inner = (np.minimum(g["cx"], 1 - g["cx"]) > 2.5 / n) & (np.minimum(g["cy"], 1 - g["cy"]) > 2.5 / n)
    scale = 1e-2 * 1e-3 * math.hypot(1, 0.5) * n
    out = {}
    for var in (0, 2):
        o = Oracle(mg.Case(m, nu=1e-2, dt=1e-3, sst=True, k=k, omega=w, variant=var))
        o.step(1)
        rk = (o.fields()["k"] * (1 + 1e-3 * 0.09 * 1e3) - k) / 1e-3   # point-implicit decay removed
        out[var] = np.abs(rk[inner]).max() / scale
    assert out[2] < 1e-3 and out[0] > 1.0, out


def test_per_stage_sst_variant_orders():
    """Variant 4 (the other reading of Step 5: SST solved again before every stage from
    (k, omega, nu_t) of t^n with the latest stage's macros, each stage with its own tau).
    Over one step from a developed state the macros change by O(dt), so nu_t (a point function
    of the strain rate) moves by O(dt), while k and u, which only feel it through a dt-weighted
    update, move by O(dt^2): halving dt halves the first and quarters the others."""
    base = mg.bfs_hybrid(n_target=1500)
    o = Oracle(base)
    o.step(200)
    f0, fl = o.get_f(), o.fields()
    diffs = []
    for frac in (1.0, 0.5):
        res = {}
        for v in (0, 4):
            c = dataclasses.replace(base, variant=v, k=fl["k"], omega=fl["omega"],
                                    dt=o.dt * frac, cfl=0.0)
            x = Oracle(c)
            x.set_f(f0)
            x.step(1)
            res[v] = x.fields()
        diffs.append({key: np.abs(res[4][key] - res[0][key]).max() for key in ("k", "nut", "u")})
    ratio = {key: diffs[0][key] / diffs[1][key] for key in diffs[0]}
    assert 1.8 < ratio["nut"] < 2.2, ratio
    assert 3.5 < ratio["k"] < 4.5, ratio
    assert 3.5 < ratio["u"] < 4.5, ratio
    # in a closed cavity with k = 0 (walls keep it 0) there is no eddy viscosity, and the
    # variant is the default bit for bit
    c0 = dataclasses.replace(mg.cavity_quad(16, re=400.0), sst=True)
    a, b = Oracle(c0), Oracle(dataclasses.replace(c0, variant=4))
    a.step(5)
    b.step(5)
    assert np.array_equal(a.get_f(), b.get_f())


def test_production_limiter_variant_homogeneous_shear():
    """Variant 8 (Menter's production limiter P_k <= 10 beta* omega k; the paper lists none)
    and the default production term, in closed form: in plane shear u = S y with uniform k and
    omega, the interior cells see no convection, diffusion or cross diffusion of k, and
    P_k = nu_t 2 S_ij S_ij = (k / omega) S^2 (nu_t of t^n = k / omega), so one point-implicit
    step gives k' = (k + dt P) / (1 + dt beta* omega) with P = k S^2 / omega (default) or
    min(k S^2 / omega, 10 beta* omega k) (variant)."""
    S, k0, w0, dt, n = 0.03, 1e-4, 0.01, 0.02, 16
    m = mg.couette_channel(6, n, U=S, H=1.0)
    g = Oracle(mg.Case(m, nu=1e-3, dt=dt)).geometry()
    inner = (g["cy"] > 2.5 / n) & (g["cy"] < 1 - 2.5 / n)
    for var, P in ((0, k0 * S * S / w0), (8, min(k0 * S * S / w0, 10 * 0.09 * w0 * k0))):
        case = mg.Case(m, nu=1e-3, dt=dt, sst=True, uref=S, u=S * g["cy"],
                       k=np.full(m.n_cells, k0), omega=np.full(m.n_cells, w0), variant=var)
        o = Oracle(case)
        o.step(1)
        kn = o.fields()["k"][inner]
        np.testing.assert_allclose(kn, (k0 + dt * P) / (1 + dt * 0.09 * w0), rtol=1e-12)


# ------------------------------------------------------------------ the oracle's own tangent
@pytest.mark.parametrize("sst", [False, True])
def test_complex_step_build_real_parts_equal_the_oracle(sst):
    """The complex-step build (the same source in complex arithmetic) carries in its real parts
    exactly the double oracle's values, seeded or not (the seed is O(h^2) = 1e-60 in the real
    parts)."""
    case = mg.naca0012_cmesh(n_target=600, alpha_deg=3.0) if sst else \
        mg.cavity_quad(10, re=400.0, jitter=0.2, seed=7)
    m = case.mesh.normalized()
    ref = Oracle(case)
    ref.step(6)
    cs = Oracle(case, complex_step=True)
    rng = np.random.default_rng(1)
    cs.cs_seed(rng.standard_normal((m.n_bedges, 5)), rng.standard_normal((m.n_cells, 9)))
    cs.step(6)
    np.testing.assert_array_equal(cs.get_f(), ref.get_f())
    val, _ = cs.cs_forces()
    assert val == {k: ref.forces()[k] for k in ("fx", "fy", "cd", "cl")}


def test_complex_step_tangent_against_central_differences():
    """Laminar cavity, random seed of f^0 and of the boundary values: the complex-step
    derivative of the wall force after 10 steps against central differences of the double
    oracle (the laminar step has no branch that the perturbation crosses)."""
    case = mg.cavity_quad(12, re=400.0, jitter=0.2, seed=7)
    m = case.mesh.normalized()
    rng = np.random.default_rng(3)
    f0 = Oracle(case).get_f()
    g = 1e-3 * rng.standard_normal(f0.shape)
    d = np.zeros((m.n_bedges, 5))
    d[:, :3] = 1e-2 * rng.standard_normal((m.n_bedges, 3))
    cs = Oracle(case, complex_step=True)
    cs.cs_seed(d, g)
    cs.step(10)
    _, der = cs.cs_forces()
    h, out = 1e-6, []
    for sgn in (1.0, -1.0):
        c = dataclasses.replace(case, mesh=dataclasses.replace(m, bedge_val=m.bedge_val + sgn * h * d))
        o = Oracle(c)
        o.set_f(f0 + sgn * h * g)
        o.step(10)
        out.append(o.forces())
    for key in ("fx", "fy"):
        fd = (out[0][key] - out[1][key]) / (2 * h)
        assert abs(der[key] - fd) <= 1e-6 * abs(fd), (key, der[key], fd)


@pytest.mark.parametrize("which", ["bfs", "naca"])
def test_complex_step_tangent_on_sst_states(which):
    """SST cases, from a state 30 steps into the run (k and omega no longer uniform, so no
    limiter sits at a tie): the complex-step derivative of the wall force along a random seed of
    f against central differences of the double oracle, to 1e-7 (measured 2e-9 at h = 1e-4)."""
    case = mg.bfs_hybrid(n_target=800) if which == "bfs" else mg.naca0012_cmesh(n_target=800, alpha_deg=3.0)
    warm, n, h = 30, 10, 1e-4
    base = Oracle(case)
    base.step(warm)
    fw = base.get_f()
    g = 1e-3 * np.random.default_rng(9).standard_normal(fw.shape)
    cs = Oracle(case, complex_step=True)
    cs.step(warm)
    cs.cs_seed(None, g)
    cs.step(n)
    _, der = cs.cs_forces()
    out = []
    for sgn in (1.0, -1.0):
        o = Oracle(case)
        o.step(warm)
        o.set_f(fw + sgn * h * g)
        o.step(n)
        out.append(o.forces())
    for key in ("fx", "fy"):
        fd = (out[0][key] - out[1][key]) / (2 * h)
        assert abs(der[key] - fd) <= 1e-7 * abs(fd), (key, der[key], fd)
