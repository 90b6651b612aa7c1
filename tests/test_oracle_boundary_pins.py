"""Physics pins of the oracle's SST limiter and open-boundary readings.

These parts of the oracle are readings of points the paper leaves to Part I or to Menter's
model (the Barth-Jespersen limiter of the k / omega reconstruction, the inlet / outlet / far
field face values of f, the SST boundary values).  Each is pinned here by a property that the
reading must have whatever its arithmetic, checked with numbers formed outside the oracle
(NumPy geometry, hand values), so that a plausible slip -- a swapped min / max, a dropped
boundary value, an inflow / outflow sign turned round, the wrong density or velocity taken from
the boundary record -- fails:

  - Barth-Jespersen limiter (Sec. 3.2's second-order upwind scheme on unstructured cells,
    reading 7 of the design): every limited face value lies within [min, max] of the cell, its
    face neighbours and its boundary values; the limiter is the largest such factor (some face
    touches a bound unless it is 1); it is 1 for a linear field on the interior of a uniform
    quad mesh.
  - Far field (Part I reading): a uniform f^eq(rho_inf, U_inf) inside far-field edges is a
    fixed point; the convection term of a cell bounded by far-field edges only equals the
    closed form in which incoming directions (e . n < 0) take the far-field equilibrium and
    outgoing ones the cell's own value.
  - Inlet / outlet: a uniform channel flow f^eq(rho0, u_in) between an inlet at u_in and an
    outlet at rho_out = rho0 stays uniform to round-off, although the inlet record carries a
    density and the outlet record a velocity that these readings must not use.
  - SST boundary values (Menter 1994, Sec. 3.2): wall k = 0 and omega = 60 nu / (beta1 d^2)
    against a value computed by hand; inlet and far field pass k_b, omega_b through; the
    outlet takes the cell's values (zero gradient).
"""
import numpy as np
import pytest

from oracle.oracle import Oracle, feq
from paper_1812_00394_gb300 import meshgen as mg

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], float)
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], float)


def _box(n, kind="quad", jitter=0.0, seed=0, btype=mg.BC_WALL, bval=(1.0, 0.0, 0.0, 0.0, 1.0)):
    """Unit box with every edge of one boundary type and one boundary record."""
    xs = np.linspace(0.0, 1.0, n + 1)
    xy, cells, sides = mg.quad_grid(xs, xs, jitter, seed)
    cells = mg.split_quads(cells) if kind == "tri" else cells
    bn = np.concatenate([sides["bottom"], sides["right"], sides["top"], sides["left"]])
    ptr = np.arange(cells.shape[0] + 1, dtype=np.int32) * cells.shape[1]
    bv = np.tile(np.asarray(bval, float), (bn.shape[0], 1))
    return mg.Mesh(xy, ptr, cells.ravel(), bn, np.full(bn.shape[0], btype, np.int32), bv).normalized()


def _faces(mesh):
    """Per cell: list of (edge midpoint, outward normal * length) from the node positions."""
    out = []
    for i in range(mesh.n_cells):
        q = mesh.xy[mesh.cell_nodes[mesh.cell_ptr[i]:mesh.cell_ptr[i + 1]]]
        r = np.roll(q, -1, axis=0)
        mid = 0.5 * (q + r)
        t = r - q
        out.append((mid, np.stack([t[:, 1], -t[:, 0]], 1)))
    return out


def _neighbour_data(mesh, phi, phib):
    """Per cell the values of its face neighbours and boundary edges (by shared edges)."""
    edge_cells = {}
    for i in range(mesh.n_cells):
        nd = mesh.cell_nodes[mesh.cell_ptr[i]:mesh.cell_ptr[i + 1]]
        for a, b in zip(nd, np.roll(nd, -1)):
            edge_cells.setdefault((min(a, b), max(a, b)), []).append(i)
    bedge = {(min(a, b), max(a, b)): k for k, (a, b) in enumerate(mesh.bedge_nodes)}
    data = [[] for _ in range(mesh.n_cells)]
    for e, cs in edge_cells.items():
        if len(cs) == 2:
            data[cs[0]].append(phi[cs[1]])
            data[cs[1]].append(phi[cs[0]])
        else:
            data[cs[0]].append(phib[bedge[e]])
    return data


# ----------------------------------------------------------------- Barth-Jespersen limiter
@pytest.mark.parametrize("kind,seed", [("tri", 1), ("quad", 2), ("tri", 3)])
def test_bj_limited_face_values_stay_within_neighbour_bounds(kind, seed):
    m = _box(10, kind=kind, jitter=0.3, seed=seed, btype=mg.BC_FARFIELD)
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.0, 1.0, m.n_cells)
    phib = rng.uniform(-0.5, 1.5, m.n_bedges)      # boundary values can set the bounds
    o = Oracle(mg.Case(m, nu=1e-3, cfl=0.5))
    psi = o.bj_limiter(phi, phib)
    g = o.gradient(phi, phib)
    geo = o.geometry()
    data = _neighbour_data(m, phi, phib)
    faces = _faces(m)
    n_active = 0
    for i in range(m.n_cells):
        lo = min(phi[i], min(data[i]))
        hi = max(phi[i], max(data[i]))
        mid, _ = faces[i]
        r = mid - np.array([geo["cx"][i], geo["cy"][i]])
        inc = r @ g[i]
        vals = phi[i] + psi[i] * inc
        span = hi - lo
        assert 0.0 <= psi[i] <= 1.0 + 1e-15, (i, psi[i])
        assert np.all(vals <= hi + 1e-12 * span) and np.all(vals >= lo - 1e-12 * span), i
        if psi[i] < 1.0:
            # the largest factor: some face value sits on a bound
            touch = np.minimum(np.abs(vals - hi), np.abs(vals - lo)).min()
            assert touch <= 1e-12 * span, (i, psi[i], touch)
            n_active += 1
    assert n_active > m.n_cells // 4        # random data: the limiter is active in many cells


def test_bj_limiter_is_one_for_a_linear_field_on_a_uniform_quad_mesh():
    """On a uniform quad mesh the least-squares gradient of a linear field is exact and every
    face-midpoint value lies halfway between the cell and the neighbour across the face, so no
    interior cell is limited."""
    n = 12
    m = _box(n, kind="quad", btype=mg.BC_FARFIELD)
    o = Oracle(mg.Case(m, nu=1e-3, cfl=0.5))
    geo = o.geometry()
    a, b, c = 0.3, 1.7, -0.9
    phi = a + b * geo["cx"] + c * geo["cy"]
    mid = 0.5 * (m.xy[m.bedge_nodes[:, 0]] + m.xy[m.bedge_nodes[:, 1]])
    phib = a + b * mid[:, 0] + c * mid[:, 1]        # boundary values on the same linear field
    psi = o.bj_limiter(phi, phib)
    interior = ((geo["cx"] > 1.0 / n) & (geo["cx"] < 1 - 1.0 / n) &
                (geo["cy"] > 1.0 / n) & (geo["cy"] < 1 - 1.0 / n))
    assert interior.sum() == (n - 2) ** 2
    np.testing.assert_allclose(psi[interior], 1.0, rtol=0, atol=1e-12)
    # a quadratic perturbation that makes a cell a local maximum limits it to 0
    phi2 = phi.copy()
    k = int(np.argmin((geo["cx"] - 0.5) ** 2 + (geo["cy"] - 0.5) ** 2))
    phi2[k] += 10.0
    assert o.bj_limiter(phi2, phib)[k] == 0.0


# ----------------------------------------------------------------- far field
def test_far_field_uniform_equilibrium_is_a_fixed_point():
    rho_inf, ux, uy = 1.02, 0.06, -0.025
    m = _box(10, kind="tri", jitter=0.25, seed=5, btype=mg.BC_FARFIELD, bval=(rho_inf, ux, uy, 0.0, 1.0))
    n = m.n_cells
    case = mg.Case(m, nu=2e-3, cfl=0.5, rho=np.full(n, rho_inf), u=np.full(n, ux), v=np.full(n, uy))
    o = Oracle(case)
    f0 = o.get_f()
    np.testing.assert_allclose(f0, np.tile(feq(rho_inf, ux, uy), (n, 1)), rtol=0, atol=1e-16)
    o.step(50)
    assert np.abs(o.get_f() - f0).max() <= 1e-14


@pytest.mark.parametrize("nodes", [[(0.0, 0.0), (1.0, 0.1), (0.8, 0.9), (-0.1, 0.7)],
                                   [(0.0, 0.0), (0.9, -0.2), (0.3, 0.8)]], ids=["quad", "tri"])
def test_far_field_convection_takes_the_free_stream_on_incoming_directions(nodes):
    """One cell whose every edge is far field (so no interior face and no reconstruction enters):
    with the cell at f1 = f^eq(rho1, u1) and the far field at (rho_inf, U_inf),
    Gamma^a_alpha = -(1/A) sum_m (e_alpha . n_m) dl_m f_m,alpha, where f_m is the far-field
    equilibrium on incoming directions (e . n < 0) and the cell's own f1 on outgoing ones."""
    xy = np.array(nodes, float)
    nv = len(nodes)
    bn = np.stack([np.arange(nv), np.roll(np.arange(nv), -1)], 1)
    rho_inf, ux, uy = 1.0, 0.08, 0.03
    bv = np.tile([rho_inf, ux, uy, 0.0, 1.0], (nv, 1))
    m = mg.Mesh(xy, np.array([0, nv], np.int32), np.arange(nv, dtype=np.int32), bn,
                np.full(nv, mg.BC_FARFIELD, np.int32), bv).normalized()
    o = Oracle(mg.Case(m, nu=2e-3, dt=1e-3))
    f1 = feq(1.01, -0.02, 0.05)
    finf = feq(rho_inf, ux, uy)
    ga = o.convection(f1[None, :])[0]
    mid, nl = _faces(m)[0]
    area = 0.5 * np.sum(xy[:, 0] * np.roll(xy[:, 1], -1) - np.roll(xy[:, 0], -1) * xy[:, 1])
    want = np.zeros(9)
    for k in range(nv):
        en = EX * nl[k, 0] + EY * nl[k, 1]          # (e . n) dl
        want -= en * np.where(en < 0.0, finf, f1) / area
    assert np.abs(want).max() > 1e-3
    np.testing.assert_allclose(ga, want, rtol=0, atol=1e-14 * np.abs(want).max())
    # the same with incoming and outgoing exchanged differs by O(1): the pin can tell them apart
    swapped = np.zeros(9)
    for k in range(nv):
        en = EX * nl[k, 0] + EY * nl[k, 1]
        swapped -= en * np.where(en < 0.0, f1, finf) / area
    assert np.abs(swapped - want).max() > 1e-2 * np.abs(want).max()


# ----------------------------------------------------------------- inlet / outlet
def _channel(nx=12, ny=6, u_in=0.05, rho0=1.0, jitter=0.2, seed=4):
    """Channel of length 2 and height 1 periodic in y, inlet on the left, outlet on the right.
    The inlet record carries a density of 1.05 and the outlet record a velocity of (-0.07, 0.02):
    the readings use the cell density at the inlet and the cell velocity at the outlet, so
    neither may enter."""
    xs = np.linspace(0.0, 2.0, nx + 1)
    ys = np.linspace(0.0, 1.0, ny + 1)
    xy, cells, sides = mg.quad_grid(xs, ys, jitter, seed)
    cells = mg.split_quads(cells)
    bn = np.concatenate([sides["bottom"], sides["top"], sides["left"], sides["right"]])
    bt = np.concatenate([np.full(nx, mg.BC_PERIODIC), np.full(nx, mg.BC_PERIODIC),
                         np.full(ny, mg.BC_INLET), np.full(ny, mg.BC_OUTLET)]).astype(np.int32)
    bv = np.zeros((bn.shape[0], 5))
    bv[:, 0] = rho0
    bv[2 * nx:2 * nx + ny] = (1.05, u_in, 0.0, 0.0, 1.0)
    bv[2 * nx + ny:] = (rho0, -0.07, 0.02, 0.0, 1.0)
    pairs = np.stack([np.arange(nx), nx + np.arange(nx)], 1).astype(np.int32)
    shift = np.tile([0.0, 1.0], (nx, 1))
    ptr = np.arange(cells.shape[0] + 1, dtype=np.int32) * 3
    return mg.Mesh(xy, ptr, cells.ravel(), bn, bt, bv, pairs, shift).normalized()


def test_uniform_channel_flow_between_inlet_and_outlet_stays_uniform():
    u_in, rho0 = 0.05, 1.0
    m = _channel(u_in=u_in, rho0=rho0)
    n = m.n_cells
    case = mg.Case(m, nu=5e-3, cfl=0.5, rho=np.full(n, rho0), u=np.full(n, u_in), v=np.zeros(n))
    o = Oracle(case)
    f0 = o.get_f()
    o.step(50)
    assert np.abs(o.get_f() - f0).max() <= 1e-14
    fl = o.fields()
    assert np.abs(fl["u"] - u_in).max() <= 1e-14 and np.abs(fl["rho"] - rho0).max() <= 1e-14


def test_channel_outlet_density_sets_the_level():
    """Started 2 % above the outlet density, the channel relaxes towards rho_out: the outlet
    reads its density from the record (a reading that took the cell's density would leave the
    mass unchanged)."""
    u_in, rho0 = 0.05, 1.0
    m = _channel(u_in=u_in, rho0=rho0)
    n = m.n_cells
    case = mg.Case(m, nu=5e-3, cfl=0.5, rho=np.full(n, 1.02 * rho0), u=np.full(n, u_in), v=np.zeros(n))
    o = Oracle(case)
    m0 = o.mass()
    o.step(200)
    assert o.mass() < m0 - 1e-3 * m0


# ----------------------------------------------------------------- SST boundary values
def test_sst_wall_omega_hand_value_and_pass_through_values():
    """Uniform 16 x 16 quads on the unit square, walls at the bottom, inlet on the left, far
    field on top, outlet on the right.  The bottom wall cells' centroids sit at d = 1/32, the
    nearest wall, so omega_b = 60 nu / (beta1 d^2) = 60 * 1e-3 * 1024 / 0.075 = 819.2."""
    n = 16
    xs = np.linspace(0.0, 1.0, n + 1)
    xy, cells, sides = mg.quad_grid(xs, xs)
    bn = np.concatenate([sides["bottom"], sides["right"], sides["top"], sides["left"]])
    bt = np.concatenate([np.full(n, mg.BC_WALL), np.full(n, mg.BC_OUTLET), np.full(n, mg.BC_FARFIELD),
                         np.full(n, mg.BC_INLET)]).astype(np.int32)
    bv = np.zeros((4 * n, 5))
    bv[:, 0] = 1.0
    bv[2 * n:3 * n] = (1.0, 0.1, 0.0, 3e-6, 40.0)      # far field k_b, omega_b
    bv[3 * n:] = (1.0, 0.1, 0.0, 5e-6, 70.0)           # inlet k_b, omega_b
    ptr = np.arange(cells.shape[0] + 1, dtype=np.int32) * 4
    m = mg.Mesh(xy, ptr, cells.ravel(), bn, bt, bv).normalized()
    rng = np.random.default_rng(0)
    k0 = rng.uniform(1e-6, 2e-6, m.n_cells)
    w0 = rng.uniform(10.0, 20.0, m.n_cells)
    u0 = rng.uniform(0.0, 0.1, m.n_cells)
    case = mg.Case(m, nu=1e-3, cfl=0.5, sst=True, k=k0, omega=w0, u=u0)
    o = Oracle(case)
    ub = o.sst_bvals()
    wall = slice(0, n)
    assert np.all(ub[wall, 2] == 0.0)                          # k = 0 on the wall
    np.testing.assert_allclose(ub[wall, 3], 819.2, rtol=1e-13)  # Menter's wall omega
    assert np.all(ub[wall, 0] == 0.0) and np.all(ub[wall, 1] == 0.0)
    np.testing.assert_array_equal(ub[2 * n:3 * n, 2:], np.tile([3e-6, 40.0], (n, 1)))
    np.testing.assert_array_equal(ub[3 * n:, 2:], np.tile([5e-6, 70.0], (n, 1)))
    # outlet: the owner cell's own values (right column of cells: x in (15/16, 1))
    geo = o.geometry()
    right = np.flatnonzero(geo["cx"] > 1 - 1.0 / n)
    right = right[np.argsort(geo["cy"][right])]
    fl = o.fields()
    np.testing.assert_array_equal(ub[n:2 * n, 2], fl["k"][right])
    np.testing.assert_array_equal(ub[n:2 * n, 3], fl["omega"][right])
    np.testing.assert_array_equal(ub[n:2 * n, 0], fl["u"][right])
