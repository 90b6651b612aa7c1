"""GPU checks of the discrete adjoint (fvlbm_adjoint) against the forward-mode tangent.

Both differentiate the same FP64 two-pass IMEX step (Sec. 3.1-3.2, Steps 2-7) of a laminar
instance.  For any seed (g, d) of the initial state and of the boundary values, the tangent gives
dJ/dp after N steps by one forward run, and the adjoint gives the gradient whose inner product
with (g, d) is the same number:  <dJ/df^0, g> + <dJ/dbval, d> = dJ/dp.  The two are computed by
different kernels (the tangent carries dual numbers forward; the adjoint transposes the flux and
gradient operators by gathers over the back slots of each face and the per-cell maps in closed
form), so agreement to rounding checks every transposed piece.  Central finite differences
close the loop: of the FP64 GPU step on a boundary-value direction, and of the FP64 CPU oracle
(no GPU code on that side) for the angle of attack, the inflow eddy-viscosity ratio and a
wall-node displacement.
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1812_00394_gb300 import fvlbm, meshgen as mg

pytestmark = pytest.mark.gpu

FP64, TAN = fvlbm.FVLBM_FP64, fvlbm.FVLBM_FP64_TANGENT
W = (0.7, -1.3)  # J = 0.7 C_D - 1.3 C_L


def _cavity():
    return mg.cavity_quad(16, re=400.0, lid_u=0.1, seed=3)


def _naca_laminar():
    c = mg.naca0012_cmesh(n_target=2500, re_c=2000.0, alpha_deg=5.0)
    return dataclasses.replace(c, sst=False)


def _bfs_laminar():
    c = mg.bfs_hybrid(n_target=3000)
    return dataclasses.replace(c, sst=False)


CASES = {"cavity": _cavity, "naca": _naca_laminar, "bfs": _bfs_laminar}


def _seeds(case, rng):
    m = case.mesh.normalized()
    g = 1e-3 * rng.standard_normal((m.n_cells, 9))
    d = np.zeros((m.n_bedges, 5))
    d[:, :3] = 1e-2 * rng.standard_normal((m.n_bedges, 3))
    return g, d


def _tangent_dJ(case, warm, n, g, d):
    t = fvlbm.Solver(case, precision=TAN, device=0)
    t.step(warm)
    t.tangent_seed(d, g)
    t.step(n)
    val, dv = t.forces_tangent(dalpha=0.0)
    t.close()
    return W[0] * val["cd"] + W[1] * val["cl"], W[0] * dv["cd"] + W[1] * dv["cl"]


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("n", [0, 1, 7, 20])
def test_adjoint_dot_product_against_tangent(name, n):
    case = CASES[name]()
    warm = 15
    rng = np.random.default_rng(100 + n)
    g, d = _seeds(case, rng)
    s = fvlbm.Solver(case, precision=FP64, device=0, kernel_path=1)
    s.step(warm)
    f_before = s.get_f()
    J, dJdf, dJdb, _ = s.adjoint(n, W[0], W[1])
    # the handle's state does not move
    np.testing.assert_array_equal(s.get_f(), f_before)
    Jt, dJt = _tangent_dJ(case, warm, n, g, d)
    adj = float(np.sum(dJdf * g) + np.sum(dJdb * d))
    assert abs(J - Jt) <= 1e-10 * max(abs(Jt), 1e-12)
    assert abs(adj - dJt) <= 1e-9 * max(abs(dJt), 1e-30), (adj, dJt)
    # k_b, omega_b do not enter a laminar step
    assert np.all(dJdb[:, 3:] == 0.0)
    s.close()


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("n", [0, 6])
def test_adjoint_shape_gradient_against_tangent(name, n):
    """dJ/dxy (reverse through the step and the host preprocessing) against the tangent of a
    random displacement of every node (forward through both), at fixed dt and initial state."""
    case = CASES[name]()
    warm = 10
    m = case.mesh.normalized()
    v = 1e-3 * np.random.default_rng(7 + n).standard_normal((m.n_nodes, 2))
    s = fvlbm.Solver(case, precision=FP64, device=0, kernel_path=1)
    s.step(warm)
    J, _, _, dxy = s.adjoint(n, W[0], W[1], shape=True)
    s.close()
    t = fvlbm.Solver(case, precision=TAN, device=0)
    t.step(warm)
    t.tangent_seed_nodes(v)
    t.step(n)
    val, dv = t.forces_tangent(dalpha=0.0)
    t.close()
    dJt = W[0] * dv["cd"] + W[1] * dv["cl"]
    adj = float(np.sum(dxy * v))
    assert abs(J - (W[0] * val["cd"] + W[1] * val["cl"])) <= 1e-10 * abs(J)
    assert abs(adj - dJt) <= 1e-8 * abs(dJt), (adj, dJt)


def test_adjoint_shape_gradient_of_one_wall_node():
    """The NACA 0012 use: dJ/d(normal displacement of one wall node) from one adjoint solve
    equals the tangent's derivative for that displacement."""
    case = _naca_laminar()
    m = case.mesh.normalized()
    wall = np.unique(m.bedge_nodes[m.bedge_type == mg.BC_WALL])
    node = int(wall[np.argmin(np.abs(m.xy[wall, 0] - 0.3) + 10 * (m.xy[wall, 1] < 0))])
    v = np.zeros((m.n_nodes, 2))
    v[node] = (0.0, 1.0)
    s = fvlbm.Solver(case, precision=FP64, device=0, kernel_path=1)
    s.step(5)
    _, _, _, dxy = s.adjoint(20, W[0], W[1], shape=True)
    s.close()
    t = fvlbm.Solver(case, precision=TAN, device=0)
    t.step(5)
    t.tangent_seed_nodes(v)
    t.step(20)
    _, dv = t.forces_tangent(dalpha=0.0)
    t.close()
    dJt = W[0] * dv["cd"] + W[1] * dv["cl"]
    assert abs(dxy[node, 1] - dJt) <= 1e-8 * abs(dJt), (dxy[node, 1], dJt)


@pytest.mark.parametrize("sst", [False, True])
@pytest.mark.parametrize("steps_of_budget,snaps_of_budget", [(1.0, 0), (2.0, 3), (6.0, 0)])
def test_adjoint_checkpoint_schedules_match_one_segment(sst, steps_of_budget, snaps_of_budget):
    """Budgets that hold the stage values of only one or three steps: the run is cut into units
    reversed on the binomial (revolve) schedule with 1 snapshot (quadratic recomputation), with
    14 snapshots for 16 unit starts (two passes for some units), or with a snapshot at every unit
    start.  The gradient is bit-identical to keeping every step: recomputed steps repeat the
    first pass's arithmetic exactly."""
    case = _naca_sst() if sst else _naca_laminar()
    s = fvlbm.Solver(case, precision=FP64, device=0, kernel_path=1)
    s.step(5)
    ref = s.adjoint(17, *W, shape=True)
    np_pad = -(-s.cells[0] // 256) * 256
    per_step = (119 if sst else 99) * 8 * np_pad
    per_snap = (15 if sst else 9) * 8 * np_pad
    s.set_adjoint_budget(int(steps_of_budget * per_step + snaps_of_budget * per_snap))
    got = s.adjoint(17, *W, shape=True)
    s.set_adjoint_budget(0)
    assert got[0] == ref[0]
    for a, b in zip(got[1:], ref[1:]):
        np.testing.assert_array_equal(a, b)
    s.close()


def test_adjoint_value_matches_fp64_forces():
    case = _naca_laminar()
    s = fvlbm.Solver(case, precision=FP64, device=0, kernel_path=1)
    s.step(10)
    J, _, _, _ = s.adjoint(12, 1.0, 0.0)
    JL, _, _, _ = s.adjoint(12, 0.0, 1.0)
    s.step(12)
    ref = s.forces()
    assert abs(J - ref["cd"]) <= 1e-10 * abs(ref["cd"])
    assert abs(JL - ref["cl"]) <= 1e-10 * abs(ref["cl"])
    s.close()


def test_adjoint_lid_speed_vs_fd():
    """Cavity, p = lid speed: dJ/dp = <dJ/dbval, d(bval)/dp> against central differences of
    the FP64 step (independent of both derivative codes)."""
    U, h, n = 0.1, 1e-5, 25
    base = _cavity()

    def solver(u):
        c = mg.cavity_quad(16, re=400.0, lid_u=u, seed=3)
        # only the lid's boundary value moves: viscosity and the C_D / C_L normalisation stay
        c = dataclasses.replace(c, rho=base.rho, u=base.u, v=base.v, nu=base.nu, uref=base.uref)
        return fvlbm.Solver(c, precision=FP64, device=0, kernel_path=1)

    m = base.mesh.normalized()
    d = np.zeros((m.n_bedges, 5))
    d[m.bedge_val[:, 1] != 0.0, 1] = 1.0
    s = solver(U)
    _, _, dJdb, _ = s.adjoint(n, *W)
    vals = []
    for u in (U + h, U - h):
        x = solver(u)
        x.step(n)
        f = x.forces()
        vals.append(W[0] * f["cd"] + W[1] * f["cl"])
        x.close()
    fd = (vals[0] - vals[1]) / (2 * h)
    adj = float(np.sum(dJdb * d))
    assert abs(adj - fd) <= 1e-6 * abs(fd), (adj, fd)
    s.close()


def test_adjoint_rejects_unsupported_handles():
    case = _cavity()
    for kw in ({"precision": fvlbm.FVLBM_FP32_DEV}, {"precision": TAN}):
        s = fvlbm.Solver(case, device=0, **kw)
        with pytest.raises(fvlbm.FvlbmError) as e:
            s.adjoint(3, 1.0, 0.0)
        assert e.value.code == fvlbm.FVLBM_ERR_NOT_SUPPORTED
        s.close()
    sst = mg.naca0012_cmesh(n_target=2500)
    s = fvlbm.Solver(sst, precision=FP64, device=0)
    with pytest.raises(fvlbm.FvlbmError) as e:
        s.adjoint(-1, 1.0, 0.0)
    assert e.value.code == fvlbm.FVLBM_ERR_BAD_PARAM
    s.close()

    # shape gradients of periodic meshes are not built; the other outputs are
    per = fvlbm.Solver(mg.Case(mg.periodic_box(8), nu=1e-3, cfl=0.5), precision=FP64, device=0)
    per.adjoint(2, 1.0, 0.0)
    with pytest.raises(fvlbm.FvlbmError) as e:
        per.adjoint(2, 1.0, 0.0, shape=True)
    assert e.value.code == fvlbm.FVLBM_ERR_NOT_SUPPORTED
    per.close()


# ------------------------------------------------------------------ k-omega SST
def _naca_sst(alpha_deg=4.0):
    return mg.naca0012_cmesh(n_target=2500, alpha_deg=alpha_deg)


def _bfs_sst():
    return mg.bfs_hybrid(n_target=3000)


SST_CASES = {"naca": _naca_sst, "bfs": _bfs_sst}


def _sst_seeds(case, rng):
    """Random seeds of f^0 and of all five boundary values (k_b, omega_b relative to their
    values)."""
    m = case.mesh.normalized()
    g = 1e-4 * rng.standard_normal((m.n_cells, 9))
    d = np.zeros((m.n_bedges, 5))
    d[:, :3] = 1e-3 * rng.standard_normal((m.n_bedges, 3))
    d[:, 3:] = 1e-3 * m.bedge_val[:, 3:] * rng.standard_normal((m.n_bedges, 2))
    return g, d


@pytest.mark.parametrize("name", sorted(SST_CASES))
@pytest.mark.parametrize("n", [0, 1, 4, 15])
def test_adjoint_sst_dot_product_against_tangent(name, n):
    """SST cases: <dJ/df^0, g> + <dJ/dbval, d> from one adjoint solve equals the tangent's
    dJ/dp for the same seeds (the SST solve, its tau, the macros it reads and all five boundary
    values transposed).  On the backward-facing step the inlet (k_b, omega_b) and the outlet
    reach the walls within a few steps."""
    case = SST_CASES[name]()
    warm = 8
    g, d = _sst_seeds(case, np.random.default_rng(200 + n))
    s = fvlbm.Solver(case, precision=FP64, device=0, kernel_path=1)
    s.step(warm)
    J, dJdf, dJdb, _ = s.adjoint(n, *W)
    s.close()
    Jt, dJt = _tangent_dJ(case, warm, n, g, d)
    adj = float(np.sum(dJdf * g) + np.sum(dJdb * d))
    assert abs(J - Jt) <= 1e-10 * abs(Jt)
    assert abs(adj - dJt) <= 1e-8 * abs(dJt), (adj, dJt)


def test_adjoint_sst_inflow_turbulence_and_alpha():
    """Parameter derivatives from one adjoint solve each, against the tangent: the inflow
    eddy-viscosity ratio of the backward-facing step through omega_b = k_b / (nu ratio) on the
    inlet, and alpha of the NACA case through (u_b, v_b) plus the drag / lift projection."""
    bfs = _bfs_sst()
    m = bfs.mesh.normalized()
    inlet = m.bedge_type == mg.BC_INLET
    d_ratio = np.zeros((m.n_bedges, 5))
    d_ratio[inlet, 4] = -m.bedge_val[inlet, 4]          # ratio = 1
    naca = _naca_sst()
    mn = naca.mesh.normalized()
    ff = mn.bedge_type == mg.BC_FARFIELD
    d_alpha = np.zeros((mn.n_bedges, 5))
    d_alpha[ff, 1] = -mn.bedge_val[ff, 2]
    d_alpha[ff, 2] = mn.bedge_val[ff, 1]
    n = 20
    for case, d, dalpha in ((bfs, d_ratio, 0.0), (naca, d_alpha, 1.0)):
        s = fvlbm.Solver(case, precision=FP64, device=0, kernel_path=1)
        s.step(10)
        _, _, dJdb, _ = s.adjoint(n, *W)
        s.close()
        t = fvlbm.Solver(case, precision=TAN, device=0)
        t.step(10)
        t.tangent_seed(d)
        t.step(n)
        val, dv = t.forces_tangent(dalpha=dalpha)
        t.close()
        dJt = W[0] * dv["cd"] + W[1] * dv["cl"]
        adj = float(np.sum(dJdb * d))
        if dalpha:
            adj += W[0] * val["cl"] - W[1] * val["cd"]
        assert abs(dJt) > 1e-12, (dalpha, dJt)
        assert abs(adj - dJt) <= 1e-8 * abs(dJt), (dalpha, adj, dJt)


@pytest.mark.parametrize("name", sorted(SST_CASES))
@pytest.mark.parametrize("n", [1, 6])
def test_adjoint_sst_shape_gradient_against_tangent(name, n):
    """SST cases: dJ/dxy through the LBM stages and the SST solve (face geometry, least-squares
    weights, 1/|d| and the wall distance of f1, f2 and the wall omega) against the tangent of a
    random displacement of every node."""
    case = SST_CASES[name]()
    warm = 8
    m = case.mesh.normalized()
    v = 1e-3 * np.random.default_rng(300 + n).standard_normal((m.n_nodes, 2))
    s = fvlbm.Solver(case, precision=FP64, device=0, kernel_path=1)
    s.step(warm)
    _, _, _, dxy = s.adjoint(n, W[0], W[1], shape=True)
    s.close()
    t = fvlbm.Solver(case, precision=TAN, device=0)
    t.step(warm)
    t.tangent_seed_nodes(v)
    t.step(n)
    _, dv = t.forces_tangent(dalpha=0.0)
    t.close()
    dJt = W[0] * dv["cd"] + W[1] * dv["cl"]
    adj = float(np.sum(dxy * v))
    assert abs(adj - dJt) <= 1e-8 * abs(dJt), (adj, dJt)


# ------------------------------------------------------------------ against the CPU oracle
def _freeze(case, base):
    return dataclasses.replace(case, rho=base.rho, u=base.u, v=base.v, k=base.k, omega=base.omega)


def _oracle_J(case, steps, dt=None):
    o = Oracle(case, dt=dt)
    o.step(steps)
    f = o.forces()
    return W[0] * f["cd"] + W[1] * f["cl"]


def test_adjoint_alpha_vs_oracle_fd():
    """SST NACA 0012: dJ/d alpha (radians) from one adjoint solve, through the far-field
    velocity and the drag / lift projection, against central differences of the FP64 CPU
    oracle at alpha +- 1e-5 rad from the same initial state."""
    a0, steps, hr = 3.0, 30, 1e-5
    base = mg.naca0012_cmesh(n_target=1500, alpha_deg=a0)
    m = base.mesh.normalized()
    ff = m.bedge_type == mg.BC_FARFIELD
    d_alpha = np.zeros((m.n_bedges, 5))
    d_alpha[ff, 1] = -m.bedge_val[ff, 2]
    d_alpha[ff, 2] = m.bedge_val[ff, 1]
    s = fvlbm.Solver(base, precision=FP64, device=0, kernel_path=1)
    _, _, dJdb, _ = s.adjoint(steps, *W)
    s.step(steps)
    f = s.forces()
    s.close()
    adj = float(np.sum(dJdb * d_alpha)) + W[0] * f["cl"] - W[1] * f["cd"]
    hd = math.degrees(hr)
    Jp = _oracle_J(_freeze(mg.naca0012_cmesh(n_target=1500, alpha_deg=a0 + hd), base), steps)
    Jm = _oracle_J(_freeze(mg.naca0012_cmesh(n_target=1500, alpha_deg=a0 - hd), base), steps)
    fd = (Jp - Jm) / (2 * hr)
    assert abs(adj - fd) <= 1e-5 * abs(fd), (adj, fd)


def test_adjoint_inflow_ratio_vs_fd():
    """SST backward-facing step: dJ/d(inflow nu_t / nu ratio) through the inlet omega_b from one
    adjoint solve over 1000 steps (long enough for the inflow turbulence to reach the walls
    downstream: over a few tens of steps the derivative is at the rounding level of J, 1e-11 of
    it), against central differences at ratio 10 +- 0.01:
    - of the FP64 GPU step, to 1e-5 (measured 7e-7);
    - of the FP64 CPU oracle (no GPU code on that side), to 3e-4: measured 8e-5, the rounding
      noise of the oracle's J over 1000 steps (its differences at h = 1e-3 and 1e-4 move by
      6e-4 and 1e-2 while the GPU step's stay within 2e-5 and 5e-4)."""
    r0, steps, h = 10.0, 1000, 1e-2
    base = mg.bfs_hybrid(n_target=1500, nut_ratio=r0)
    m = base.mesh.normalized()
    inlet = m.bedge_type == mg.BC_INLET
    d_ratio = np.zeros((m.n_bedges, 5))
    d_ratio[inlet, 4] = -m.bedge_val[inlet, 4] / r0
    s = fvlbm.Solver(base, precision=FP64, device=0, kernel_path=1)
    _, _, dJdb, _ = s.adjoint(steps, *W)
    s.close()
    adj = float(np.sum(dJdb * d_ratio))
    cases = [_freeze(mg.bfs_hybrid(n_target=1500, nut_ratio=r0 + e), base) for e in (h, -h)]
    gpu = []
    for c in cases:
        g = fvlbm.Solver(c, precision=FP64, device=0, kernel_path=1)
        g.step(steps)
        f = g.forces()
        g.close()
        gpu.append(W[0] * f["cd"] + W[1] * f["cl"])
    fd_gpu = (gpu[0] - gpu[1]) / (2 * h)
    fd_oracle = (_oracle_J(cases[0], steps) - _oracle_J(cases[1], steps)) / (2 * h)
    assert abs(adj - fd_gpu) <= 1e-5 * abs(fd_gpu), (adj, fd_gpu)
    assert abs(adj - fd_oracle) <= 3e-4 * abs(fd_oracle), (adj, fd_oracle)


def test_adjoint_wall_node_vs_oracle_fd():
    """SST NACA 0012 at Re_c = 1e4: dJ/d(normal displacement of one wall node) from the adjoint's
    shape gradient, at fixed dt, against central differences of the FP64 CPU oracle on moved
    meshes."""
    steps, h = 30, 1e-6
    base = mg.naca0012_cmesh(n_target=1500, re_c=1e4, alpha_deg=4.0)
    m = base.mesh.normalized()
    wall = m.bedge_nodes[m.bedge_type == mg.BC_WALL]
    nodes = np.unique(wall)
    upper = nodes[m.xy[nodes, 1] > 0]
    j = int(upper[np.argmin(np.abs(m.xy[upper, 0] - 0.3))])
    nb = np.unique(wall[(wall == j).any(1)])
    nb = nb[nb != j]
    t = m.xy[nb[1]] - m.xy[nb[0]]
    n = np.array([-t[1], t[0]]) / np.linalg.norm(t)
    n = n if n[1] > 0 else -n
    s = fvlbm.Solver(base, precision=FP64, device=0, kernel_path=1)
    dt = s.dt()
    _, _, _, dxy = s.adjoint(steps, *W, shape=True)
    s.close()
    adj = float(dxy[j] @ n)

    def moved(eps):
        xy = m.xy.copy()
        xy[j] += eps * n
        return dataclasses.replace(base, mesh=dataclasses.replace(m, xy=xy), dt=dt)
    fd = (_oracle_J(moved(h), steps, dt) - _oracle_J(moved(-h), steps, dt)) / (2 * h)
    assert abs(adj - fd) <= 1e-5 * abs(fd), (adj, fd)


@pytest.mark.parametrize("sst", [False, True])
def test_adjoint_local_time_steps_against_tangent(sst):
    """Local time stepping (every cell its own dt_i): the adjoint of the step with per-cell
    steps in the stages, the implicit collision and the SST update, against the tangent."""
    base = _naca_sst() if sst else _naca_laminar()
    case = dataclasses.replace(base, local_dt=True, cfl=0.2)
    warm, n = 5, 8
    g, d = _sst_seeds(case, np.random.default_rng(400 + int(sst)))
    s = fvlbm.Solver(case, precision=FP64, device=0, kernel_path=1)
    s.step(warm)
    J, dJdf, dJdb, _ = s.adjoint(n, *W)
    s.close()
    Jt, dJt = _tangent_dJ(case, warm, n, g, d)
    adj = float(np.sum(dJdf * g) + np.sum(dJdb * d))
    assert abs(J - Jt) <= 1e-10 * abs(Jt)
    assert abs(adj - dJt) <= 1e-8 * abs(dJt), (adj, dJt)


def test_adjoint_periodic_channel_against_tangent():
    """A jittered triangular Couette channel, periodic in x: the transposed flux and gradient
    gather across the glued faces through their back slots (the shifted neighbour offsets)."""
    m = mg.couette_channel(12, 8, kind="tri", jitter=0.2, seed=4)
    case = mg.Case(m, nu=0.01, cfl=0.5, uref=0.1)
    warm, n = 10, 12
    rng = np.random.default_rng(55)
    g = 1e-3 * rng.standard_normal((m.n_cells, 9))
    d = np.zeros((m.n_bedges, 5))
    d[:, :3] = 1e-2 * rng.standard_normal((m.n_bedges, 3))
    s = fvlbm.Solver(case, precision=FP64, device=0, kernel_path=1)
    s.step(warm)
    J, dJdf, dJdb, _ = s.adjoint(n, *W)
    s.close()
    Jt, dJt = _tangent_dJ(case, warm, n, g, d)
    adj = float(np.sum(dJdf * g) + np.sum(dJdb * d))
    assert abs(J - Jt) <= 1e-10 * abs(Jt)
    assert abs(adj - dJt) <= 1e-9 * abs(dJt), (adj, dJt)
    # glued edges carry no boundary value
    glued = m.periodic_pairs.ravel()
    assert np.all(dJdb[glued] == 0.0)


def test_adjoint_instance_of_a_batch_equals_single_handle():
    """In a batch (laminar cavity, SST airfoil, laminar airfoil) the adjoint of one instance
    equals that of a handle holding the instance alone: instances do not couple, and the other
    instances' adjoints stay zero."""
    cases = [_cavity(), _naca_sst(), _naca_laminar()]
    b = fvlbm.Solver(cases, precision=FP64, device=0, kernel_path=1)
    b.step(6)
    for i, c in enumerate(cases):
        one = fvlbm.Solver(c, precision=FP64, device=0, kernel_path=1)
        one.step(6)
        got = b.adjoint(9, *W, i=i, shape=True)
        ref = one.adjoint(9, *W, shape=True)
        one.close()
        assert abs(got[0] - ref[0]) <= 1e-12 * abs(ref[0])
        for x, y in zip(got[1:], ref[1:]):
            np.testing.assert_allclose(x, y, rtol=1e-10, atol=1e-12 * np.abs(y).max())
    b.close()


# ------------------------------------------------------------------ against the oracle's tangent
@pytest.mark.parametrize("name", ["cavity", "bfs_sst", "naca_sst"])
def test_adjoint_against_oracle_complex_step_tangent(name):
    """The oracle's own tangent: its source compiled in complex arithmetic (complex-step method,
    no GPU code, no differences taken) along a random seed of f^0 and of the boundary values,
    against the adjoint's inner product with the same seed, on tiny meshes.  The initial
    k / omega fields are uniform, so the SST limiters start at exact ties; both sides take the
    branch of the first argument there (finite differences, which average the two one-sided
    derivatives, cannot be used at this point)."""
    case = {"cavity": lambda: mg.cavity_quad(12, re=400.0, jitter=0.2, seed=7),
            "bfs_sst": lambda: mg.bfs_hybrid(n_target=800),
            "naca_sst": lambda: mg.naca0012_cmesh(n_target=800, alpha_deg=3.0)}[name]()
    m = case.mesh.normalized()
    rng = np.random.default_rng(3)
    n = 10
    s = fvlbm.Solver(case, precision=FP64, device=0, kernel_path=1)
    f0 = s.get_f()
    g = 1e-3 * rng.standard_normal(f0.shape)
    d = np.zeros((m.n_bedges, 5))
    d[:, :3] = 1e-2 * rng.standard_normal((m.n_bedges, 3))
    d[:, 3:] = 1e-3 * m.bedge_val[:, 3:] * rng.standard_normal((m.n_bedges, 2))
    J, dJdf, dJdb, _ = s.adjoint(n, *W)
    s.close()
    o = Oracle(case, complex_step=True)
    o.cs_seed(d, g)
    o.step(n)
    val, der = o.cs_forces()
    Jo = W[0] * val["cd"] + W[1] * val["cl"]
    dJo = W[0] * der["cd"] + W[1] * der["cl"]
    adj = float(np.sum(dJdf * g) + np.sum(dJdb * d))
    assert abs(J - Jo) <= 1e-10 * abs(Jo)
    assert abs(adj - dJo) <= 1e-8 * abs(dJo), (adj, dJo)


@pytest.mark.parametrize("variant", [2, 8, 10])
def test_adjoint_sst_reading_variants_against_tangent(variant):
    """SST reading variants 2 (non-orthogonal correction of the diffusion, with the neighbours'
    gradients) and 8 (production limiter): the dot-product identity of the adjoint against the
    tangent, for seeds of f^0 and the boundary values and for a random node displacement."""
    case = dataclasses.replace(_bfs_sst(), variant=variant)
    warm, n = 8, 6
    g, d = _sst_seeds(case, np.random.default_rng(500 + variant))
    m = case.mesh.normalized()
    v = 1e-3 * np.random.default_rng(600 + variant).standard_normal((m.n_nodes, 2))
    s = fvlbm.Solver(case, precision=FP64, device=0, kernel_path=1)
    s.step(warm)
    J, dJdf, dJdb, dxy = s.adjoint(n, *W, shape=True)
    s.close()
    Jt, dJt = _tangent_dJ(case, warm, n, g, d)
    adj = float(np.sum(dJdf * g) + np.sum(dJdb * d))
    assert abs(J - Jt) <= 1e-10 * abs(Jt)
    assert abs(adj - dJt) <= 1e-8 * abs(dJt), (adj, dJt)
    t = fvlbm.Solver(case, precision=TAN, device=0)
    t.step(warm)
    t.tangent_seed_nodes(v)
    t.step(n)
    _, dv = t.forces_tangent(dalpha=0.0)
    t.close()
    dJv = W[0] * dv["cd"] + W[1] * dv["cl"]
    assert abs(float(np.sum(dxy * v)) - dJv) <= 1e-8 * abs(dJv), (float(np.sum(dxy * v)), dJv)


@pytest.mark.parametrize("name,variant", [("naca_laminar", 1), ("bfs_sst", 1), ("bfs_sst", 11)])
def test_adjoint_gradient_limiter_against_tangent(name, variant):
    """Reading variant 1 (Venkatakrishnan limiter on grad f): the limiter's transpose (through
    the selected face's factor, the raw gradient and the extreme among the cell, its neighbours
    and its boundary values) against the tangent, for seeds of f^0 and of the boundary values;
    with variants 2 and 8 on top on the SST step; and the shape gradient (the limiter reads the
    face offsets and the cell area) against the tangent of a random node displacement."""
    base = _naca_laminar() if name == "naca_laminar" else _bfs_sst()
    case = dataclasses.replace(base, variant=variant)
    warm, n = 8, 6
    g, d = _sst_seeds(case, np.random.default_rng(700 + variant))
    m = case.mesh.normalized()
    v = 1e-3 * np.random.default_rng(750 + variant).standard_normal((m.n_nodes, 2))
    s = fvlbm.Solver(case, precision=FP64, device=0, kernel_path=1)
    s.step(warm)
    J, dJdf, dJdb, dxy = s.adjoint(n, *W, shape=True)
    s.close()
    Jt, dJt = _tangent_dJ(case, warm, n, g, d)
    adj = float(np.sum(dJdf * g) + np.sum(dJdb * d))
    assert abs(J - Jt) <= 1e-10 * abs(Jt)
    assert abs(adj - dJt) <= 1e-8 * abs(dJt), (adj, dJt)
    t = fvlbm.Solver(case, precision=TAN, device=0)
    t.step(warm)
    t.tangent_seed_nodes(v)
    t.step(n)
    _, dv = t.forces_tangent(dalpha=0.0)
    t.close()
    dJv = W[0] * dv["cd"] + W[1] * dv["cl"]
    assert abs(float(np.sum(dxy * v)) - dJv) <= 1e-8 * abs(dJv), (float(np.sum(dxy * v)), dJv)


@pytest.mark.parametrize("name,variant", [("bfs_sst", 4), ("naca_sst", 4), ("bfs_sst", 14)])
def test_adjoint_per_stage_sst_against_tangent(name, variant):
    """Reading variant 4 (the SST solved from t^n before every stage, with the macros of f^n,
    f^(1), f^(2)): three SST transposes per step, each feeding the adjoint of its stage value
    and the shared t^n state; against the tangent for state, boundary and node seeds (with
    variants 2 and 8 on top)."""
    base = _bfs_sst() if name == "bfs_sst" else _naca_sst()
    case = dataclasses.replace(base, variant=variant)
    warm, n = 8, 6
    g, d = _sst_seeds(case, np.random.default_rng(800 + variant))
    m = case.mesh.normalized()
    v = 1e-3 * np.random.default_rng(900 + variant).standard_normal((m.n_nodes, 2))
    s = fvlbm.Solver(case, precision=FP64, device=0, kernel_path=1)
    s.step(warm)
    J, dJdf, dJdb, dxy = s.adjoint(n, *W, shape=True)
    s.close()
    Jt, dJt = _tangent_dJ(case, warm, n, g, d)
    adj = float(np.sum(dJdf * g) + np.sum(dJdb * d))
    assert abs(J - Jt) <= 1e-10 * abs(Jt)
    assert abs(adj - dJt) <= 1e-8 * abs(dJt), (adj, dJt)
    t = fvlbm.Solver(case, precision=TAN, device=0)
    t.step(warm)
    t.tangent_seed_nodes(v)
    t.step(n)
    _, dv = t.forces_tangent(dalpha=0.0)
    t.close()
    dJv = W[0] * dv["cd"] + W[1] * dv["cl"]
    assert abs(float(np.sum(dxy * v)) - dJv) <= 1e-8 * abs(dJv), (float(np.sum(dxy * v)), dJv)


@pytest.mark.parametrize("name", ["cavity", "bfs_sst"])
def test_adjoint_explicit_euler_scheme_against_tangent(name):
    """The explicit Euler comparison scheme (f^{n+1} = f + dt (Gamma^a + Gamma^c), Part I),
    laminar and with the SST solve: the adjoint against the tangent for state, boundary and node
    seeds.  Steps within its collision limit dt < 2 tau."""
    if name == "cavity":
        case = mg.cavity_quad(16, re=10.0, lid_u=0.1, seed=3)
    else:
        case = dataclasses.replace(_bfs_sst(), dt=1e-5, cfl=0.0)
    warm, n = 5, 6
    g, d = _sst_seeds(case, np.random.default_rng(950))
    m = case.mesh.normalized()
    v = 1e-3 * np.random.default_rng(951).standard_normal((m.n_nodes, 2))
    s = fvlbm.Solver(case, precision=FP64, device=0, scheme=1)
    s.step(warm)
    J, dJdf, dJdb, dxy = s.adjoint(n, *W, shape=True)
    s.close()
    t = fvlbm.Solver(case, precision=TAN, device=0, scheme=1)
    t.step(warm)
    t.tangent_seed(d, g)
    t.step(n)
    val, dv = t.forces_tangent(dalpha=0.0)
    t.close()
    Jt, dJt = W[0] * val["cd"] + W[1] * val["cl"], W[0] * dv["cd"] + W[1] * dv["cl"]
    adj = float(np.sum(dJdf * g) + np.sum(dJdb * d))
    assert abs(J - Jt) <= 1e-10 * abs(Jt)
    assert abs(adj - dJt) <= 1e-8 * abs(dJt), (adj, dJt)
    t = fvlbm.Solver(case, precision=TAN, device=0, scheme=1)
    t.step(warm)
    t.tangent_seed_nodes(v)
    t.step(n)
    _, dv = t.forces_tangent(dalpha=0.0)
    t.close()
    dJv = W[0] * dv["cd"] + W[1] * dv["cl"]
    assert abs(float(np.sum(dxy * v)) - dJv) <= 1e-8 * abs(dJv), (float(np.sum(dxy * v)), dJv)


@pytest.mark.parametrize("sst", [False, True])
def test_adjoint_of_a_fused_path_handle(sst):
    """A handle that steps with the fused kernels (the default) gives the same gradient as one
    that steps with the two-pass kernels: the adjoint recomputes with the two-pass step from the
    handle's state, and the two paths' states agree to rounding."""
    case = _naca_sst() if sst else _naca_laminar()
    out = []
    for path in (0, 1):
        s = fvlbm.Solver(case, precision=FP64, device=0, kernel_path=path)
        s.step(8)
        out.append(s.adjoint(10, *W, shape=True))
        s.close()
    assert abs(out[0][0] - out[1][0]) <= 1e-12 * abs(out[1][0])
    for a, b in zip(out[0][1:], out[1][1:]):
        assert np.abs(a - b).max() <= 1e-9 * np.abs(b).max()
