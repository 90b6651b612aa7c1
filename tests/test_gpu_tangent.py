"""GPU checks of the forward-mode tangent (FVLBM_FP64_TANGENT) against central finite
differences: of the GPU FP64 step, and of the FP64 CPU oracle (independent of the CUDA path).

The tangent differentiates the discrete step (Steps 1-7 of Sec. 3.2) with respect to one scalar
parameter p that enters through boundary values.  The finite differences perturb only those
boundary values and start from the same initial state, which is what the tangent seeds
(d f^0 / dp = 0, d k^0 / dp = d omega^0 / dp = 0).
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1812_00394_gb300 import fvlbm, meshgen as mg

pytestmark = pytest.mark.gpu

FP64, TAN = fvlbm.FVLBM_FP64, fvlbm.FVLBM_FP64_TANGENT


def _freeze_init(case, base):
    """``case`` with the initial fields of ``base`` (only the boundary values differ)."""
    return dataclasses.replace(case, rho=base.rho, u=base.u, v=base.v, k=base.k,
                               omega=base.omega)


def _naca(alpha_deg=4.0, nut_ratio=1.0, n=2500):
    return mg.naca0012_cmesh(n_target=n, alpha_deg=alpha_deg, nut_ratio=nut_ratio)


def _dbval_alpha(case):
    """d(rho_b, u_b, v_b, k_b, omega_b)/d(alpha in radians): far field (U cos a, U sin a)."""
    m = case.mesh.normalized()
    d = np.zeros((m.n_bedges, 5))
    ff = m.bedge_type == mg.BC_FARFIELD
    d[ff, 1] = -m.bedge_val[ff, 2]
    d[ff, 2] = m.bedge_val[ff, 1]
    return d


def _dbval_nut_ratio(case, ratio):
    """omega_b = k_b / (nu * ratio) on the far field: d omega_b / d ratio = -omega_b / ratio."""
    m = case.mesh.normalized()
    d = np.zeros((m.n_bedges, 5))
    ff = m.bedge_type == mg.BC_FARFIELD
    d[ff, 4] = -m.bedge_val[ff, 4] / ratio
    return d


def _gpu_forces(case, steps):
    s = fvlbm.Solver(case, precision=FP64, device=0, kernel_path=1)
    s.step(steps)
    out = s.forces()
    s.close()
    return out


def test_tangent_values_match_fp64():
    case = _naca()
    t = fvlbm.Solver(case, precision=TAN, device=0)
    s = fvlbm.Solver(case, precision=FP64, device=0, kernel_path=1)
    t.tangent_seed(_dbval_alpha(case))
    t.step(30)
    s.step(30)
    ft, fs = t.get_f(), s.get_f()
    assert np.abs(ft - fs).max() <= 1e-12 * np.abs(fs).max()
    val, _ = t.forces_tangent(dalpha=1.0)
    ref = s.forces()
    for key in ("fx", "fy", "cd", "cl"):
        assert abs(val[key] - ref[key]) <= 1e-10 * max(abs(ref[key]), 1e-12), key
    # plain forces on a tangent handle equal the value part
    plain = t.forces()
    assert plain["cl"] == val["cl"]


def test_tangent_zero_seed_gives_zero_derivative():
    case = _naca()
    t = fvlbm.Solver(case, precision=TAN, device=0)
    t.step(10)
    assert np.abs(t.get_f_tangent()).max() == 0.0
    _, d = t.forces_tangent()
    assert all(v == 0.0 for v in d.values())


def test_tangent_entry_points_reject_plain_handles():
    s = fvlbm.Solver(mg.cavity_quad(16), precision=FP64, device=0)
    with pytest.raises(fvlbm.FvlbmError) as e:
        s.get_f_tangent()
    assert e.value.code == fvlbm.FVLBM_ERR_NOT_SUPPORTED


@pytest.mark.parametrize("steps", [1, 40])
def test_tangent_lid_speed_vs_fd_laminar(steps):
    """Laminar cavity, p = lid speed: df/dp after `steps` steps against central differences.
    The laminar step has no branches that depend on the state, so the match is tight."""
    U, h = 0.1, 1e-5
    base = mg.cavity_quad(24, re=400.0, lid_u=U, seed=3)

    def with_lid(u):
        c = mg.cavity_quad(24, re=400.0, lid_u=u, seed=3)
        return dataclasses.replace(_freeze_init(c, base), nu=base.nu)

    m = base.mesh.normalized()
    d = np.zeros((m.n_bedges, 5))
    d[m.bedge_val[:, 1] != 0.0, 1] = 1.0
    t = fvlbm.Solver(base, precision=TAN, device=0)
    t.tangent_seed(d)
    t.step(steps)
    df = t.get_f_tangent()
    fp = fvlbm.Solver(with_lid(U + h), precision=FP64, device=0, kernel_path=1)
    fm = fvlbm.Solver(with_lid(U - h), precision=FP64, device=0, kernel_path=1)
    fp.step(steps)
    fm.step(steps)
    fd = (fp.get_f() - fm.get_f()) / (2 * h)
    assert np.linalg.norm(df - fd) <= 1e-7 * np.linalg.norm(fd)


def test_tangent_initial_state_seed_vs_fd():
    """p scales a perturbation of f^0 (df^0/dp = g): the tangent of the state after 20 steps
    against central differences of the FP64 step."""
    base = mg.cavity_quad(20, re=400.0, seed=5)
    s = fvlbm.Solver(base, precision=FP64, device=0, kernel_path=1)
    f0 = s.get_f()
    rng = np.random.default_rng(11)
    g = 1e-3 * rng.standard_normal(f0.shape)
    h = 1e-4
    fp = fvlbm.Solver(base, precision=FP64, device=0, kernel_path=1)
    fm = fvlbm.Solver(base, precision=FP64, device=0, kernel_path=1)
    fp.set_f(f0 + h * g)
    fm.set_f(f0 - h * g)
    fp.step(20)
    fm.step(20)
    fd = (fp.get_f() - fm.get_f()) / (2 * h)
    t = fvlbm.Solver(base, precision=TAN, device=0)
    t.tangent_seed(df=g)
    np.testing.assert_array_equal(t.get_f_tangent(), g)
    t.step(20)
    df = t.get_f_tangent()
    assert np.linalg.norm(df - fd) <= 1e-6 * np.linalg.norm(fd)


def test_tangent_alpha_vs_gpu_fd_sst():
    """SST NACA 0012: d(C_D, C_L)/d alpha (per radian) after 60 steps against central
    differences of two FP64 runs at alpha +- 1e-5 rad (same initial state)."""
    a0, steps = 4.0, 60
    base = _naca(a0)
    hr = 1e-5
    hd = math.degrees(hr)
    cp = _freeze_init(_naca(a0 + hd), base)
    cm = _freeze_init(_naca(a0 - hd), base)
    t = fvlbm.Solver(base, precision=TAN, device=0)
    t.tangent_seed(_dbval_alpha(base))
    t.step(steps)
    _, d = t.forces_tangent(dalpha=1.0)
    fp, fm = _gpu_forces(cp, steps), _gpu_forces(cm, steps)
    for key in ("cd", "cl", "fx", "fy"):
        fd = (fp[key] - fm[key]) / (2 * hr)
        scale = max(abs(fd), abs(d["cl"]) * 1e-3)
        assert abs(d[key] - fd) <= 1e-5 * scale, (key, d[key], fd)


def test_tangent_nut_ratio_vs_gpu_fd_sst():
    """SST NACA 0012: d(C_D, C_L)/d(far-field eddy-viscosity ratio) through omega_b."""
    r0, steps, h = 1.0, 60, 1e-5
    base = _naca(6.0, r0)
    cp = _freeze_init(_naca(6.0, r0 + h), base)
    cm = _freeze_init(_naca(6.0, r0 - h), base)
    t = fvlbm.Solver(base, precision=TAN, device=0)
    t.tangent_seed(_dbval_nut_ratio(base, r0))
    t.step(steps)
    _, d = t.forces_tangent()
    fp, fm = _gpu_forces(cp, steps), _gpu_forces(cm, steps)
    for key in ("cd", "cl"):
        fd = (fp[key] - fm[key]) / (2 * h)
        scale = max(abs(fd), 1e-12)
        assert abs(d[key] - fd) <= 1e-4 * scale + 1e-10, (key, d[key], fd)


def test_tangent_alpha_vs_oracle_fd():
    """The same derivative against central differences of the FP64 CPU oracle (no GPU code on
    that side)."""
    a0, steps, hr = 3.0, 30, 1e-5
    base = _naca(a0, n=1500)
    hd = math.degrees(hr)
    op = Oracle(_freeze_init(_naca(a0 + hd, n=1500), base))
    om = Oracle(_freeze_init(_naca(a0 - hd, n=1500), base))
    op.step(steps)
    om.step(steps)
    fp, fm = op.forces(), om.forces()
    t = fvlbm.Solver(base, precision=TAN, device=0)
    t.tangent_seed(_dbval_alpha(base))
    t.step(steps)
    _, d = t.forces_tangent(dalpha=1.0)
    for key in ("cd", "cl"):
        fd = (fp[key] - fm[key]) / (2 * hr)
        assert abs(d[key] - fd) <= 1e-5 * max(abs(fd), abs(d["cl"]) * 1e-3), (key, d[key], fd)


def _wall_node_normal(case, which=0.3):
    """A wall node on the upper surface near x = `which` chords and its outward unit normal
    (from the neighbouring wall nodes), as a [n_nodes, 2] displacement field."""
    m = case.mesh.normalized()
    wall = m.bedge_nodes[m.bedge_type == mg.BC_WALL]
    nodes = np.unique(wall)
    upper = nodes[m.xy[nodes, 1] > 0]
    j = int(upper[np.argmin(np.abs(m.xy[upper, 0] - which))])
    nb = np.unique(wall[(wall == j).any(1)])
    nb = nb[nb != j]
    t = m.xy[nb[1]] - m.xy[nb[0]]
    n = np.array([-t[1], t[0]]) / np.linalg.norm(t)
    if n[1] < 0:
        n = -n
    d = np.zeros_like(m.xy)
    d[j] = n
    return d


def _moved(case, dxy, eps, dt):
    m = case.mesh.normalized()
    mesh = dataclasses.replace(m, xy=m.xy + eps * dxy)
    return dataclasses.replace(case, mesh=mesh, dt=dt)


@pytest.mark.parametrize("node_x", [0.05, 0.5])
def test_tangent_wall_node_displacement_vs_gpu_fd(node_x):
    """d(C_D, C_L)/d(normal displacement of one wall node) on an SST NACA 0012 at Re_c = 1e4
    (first cell ~2e-3 chord), at fixed dt, after 40 steps: tangent against central differences
    of the FP64 step on moved meshes."""
    base = mg.naca0012_cmesh(n_target=2500, re_c=1e4, alpha_deg=4.0)
    dxy = _wall_node_normal(base, node_x)
    t = fvlbm.Solver(base, precision=TAN, device=0)
    dt = t.dt()
    t.tangent_seed_nodes(dxy)
    t.step(40)
    _, d = t.forces_tangent()
    h = 1e-6
    fp = _gpu_forces(_moved(base, dxy, h, dt), 40)
    fm = _gpu_forces(_moved(base, dxy, -h, dt), 40)
    for key in ("cd", "cl"):
        fd = (fp[key] - fm[key]) / (2 * h)
        assert abs(d[key] - fd) <= 1e-4 * abs(fd) + 1e-9, (key, d[key], fd)


def test_tangent_interior_node_displacement_vs_fd_laminar():
    """Laminar cavity, one interior node two cells below the moving lid displaced: df/dp after
    40 steps against central differences (geometry enters the face fluxes and gradient weights
    of the four cells around the node; the flow there is developed, so the derivative is well
    above the rounding level of the differences)."""
    base = mg.cavity_quad(16, re=400.0, jitter=0.2, seed=7)
    m = base.mesh.normalized()
    j = int(np.argmin(np.linalg.norm(m.xy - np.array([0.5, 0.875]), axis=1)))
    dxy = np.zeros_like(m.xy)
    dxy[j] = (0.6, 0.8)
    t = fvlbm.Solver(base, precision=TAN, device=0)
    dt = t.dt()
    t.tangent_seed_nodes(dxy)
    t.step(40)
    df = t.get_f_tangent()
    h = 1e-6
    sp = fvlbm.Solver(_moved(base, dxy, h, dt), precision=FP64, device=0, kernel_path=1)
    sm = fvlbm.Solver(_moved(base, dxy, -h, dt), precision=FP64, device=0, kernel_path=1)
    sp.step(40)
    sm.step(40)
    fd = (sp.get_f() - sm.get_f()) / (2 * h)
    assert np.linalg.norm(df - fd) <= 1e-5 * np.linalg.norm(fd)
    # with every seed cleared (geometry and state; laminar, so no k / omega) the derivative is 0
    t.tangent_seed_nodes(np.zeros_like(dxy))
    t.tangent_seed(df=np.zeros_like(df))
    t.step(3)
    assert np.abs(t.get_f_tangent()).max() == 0.0


def test_tangent_batch_directions_match_single():
    """Several directions as one batch (one instance per direction, one launch per kernel)
    give the same derivatives as separate single-instance handles."""
    base = _naca(4.0, n=1500)
    dirs = [_dbval_alpha(base), _dbval_nut_ratio(base, 1.0)]
    b = fvlbm.Solver([base, base], precision=TAN, device=0)
    for i, dv in enumerate(dirs):
        b.tangent_seed(dv, i=i)
    b.step(20)
    for i, dv in enumerate(dirs):
        s = fvlbm.Solver(base, precision=TAN, device=0)
        s.tangent_seed(dv)
        s.step(20)
        np.testing.assert_allclose(b.get_f_tangent(i), s.get_f_tangent(), rtol=0, atol=1e-12 *
                                   max(np.abs(s.get_f_tangent()).max(), 1e-300))


def test_forces_gradient_many_directions_in_one_batch():
    """d(C_D, C_L) along alpha, the inflow eddy-viscosity ratio and the normal displacements of
    eight wall nodes, as one batched tangent solve: every direction equals its own
    single-instance tangent, and the alpha and one wall-node direction match central
    differences of the FP64 step."""
    base = mg.naca0012_cmesh(n_target=2500, re_c=1e4, alpha_deg=4.0)
    steps = 30
    dirs = [{"dbedge_val": _dbval_alpha(base), "dalpha": 1.0},
            {"dbedge_val": _dbval_nut_ratio(base, 1.0)}]
    for x in np.linspace(0.05, 0.9, 8):
        dirs.append({"dxy": _wall_node_normal(base, float(x))})
    val, grads = fvlbm.forces_gradient(base, dirs, steps, device=0)
    assert len(grads) == len(dirs)
    for k in (0, 1, 5):
        s = fvlbm.Solver(base, precision=TAN, device=0)
        if "dxy" in dirs[k]:
            s.tangent_seed_nodes(dirs[k]["dxy"])
        else:
            s.tangent_seed(dirs[k]["dbedge_val"])
        s.step(steps)
        _, g1 = s.forces_tangent(dalpha=dirs[k].get("dalpha", 0.0))
        for key in ("cd", "cl"):
            assert abs(grads[k][key] - g1[key]) <= 1e-12 * max(abs(g1[key]), 1e-30), (k, key)
    # alpha against central differences at fixed dt and initial state
    t = fvlbm.Solver(base, precision=TAN, device=0)
    dt = t.dt()
    hr = 1e-5
    cp = dataclasses.replace(_freeze_init(mg.naca0012_cmesh(n_target=2500, re_c=1e4,
                                                           alpha_deg=4.0 + math.degrees(hr)), base), dt=dt)
    cm = dataclasses.replace(_freeze_init(mg.naca0012_cmesh(n_target=2500, re_c=1e4,
                                                           alpha_deg=4.0 - math.degrees(hr)), base), dt=dt)
    fp, fm = _gpu_forces(cp, steps), _gpu_forces(cm, steps)
    fd = (fp["cl"] - fm["cl"]) / (2 * hr)
    assert abs(grads[0]["cl"] - fd) <= 1e-5 * abs(fd)
    # a wall node against central differences on moved meshes
    h = 1e-6
    fp = _gpu_forces(_moved(base, dirs[5]["dxy"], h, dt), steps)
    fm = _gpu_forces(_moved(base, dirs[5]["dxy"], -h, dt), steps)
    fd = (fp["cl"] - fm["cl"]) / (2 * h)
    assert abs(grads[5]["cl"] - fd) <= 1e-4 * abs(fd) + 1e-9


@pytest.mark.parametrize("name", ["cavity", "bfs_sst", "naca_sst"])
def test_tangent_against_oracle_complex_step(name):
    """The tangent (dual numbers on the GPU) against the oracle's own tangent (its source in
    complex arithmetic on the CPU) along one random seed of f^0 and of the boundary values, on
    tiny meshes: d(C_D, C_L)/dp after 10 steps to 1e-8 and the values to 1e-10, both relative to
    the larger of the two coefficients."""
    case = {"cavity": lambda: mg.cavity_quad(12, re=400.0, jitter=0.2, seed=7),
            "bfs_sst": lambda: mg.bfs_hybrid(n_target=800),
            "naca_sst": lambda: mg.naca0012_cmesh(n_target=800, alpha_deg=3.0)}[name]()
    m = case.mesh.normalized()
    rng = np.random.default_rng(5)
    t = fvlbm.Solver(case, precision=TAN, device=0)
    f0 = t.get_f()
    g = 1e-3 * rng.standard_normal(f0.shape)
    d = np.zeros((m.n_bedges, 5))
    d[:, :3] = 1e-2 * rng.standard_normal((m.n_bedges, 3))
    d[:, 3:] = 1e-3 * m.bedge_val[:, 3:] * rng.standard_normal((m.n_bedges, 2))
    t.tangent_seed(d, g)
    t.step(10)
    val, dv = t.forces_tangent(dalpha=0.0)
    t.close()
    o = Oracle(case, complex_step=True)
    o.cs_seed(d, g)
    o.step(10)
    ov, od = o.cs_forces()
    # relative to the larger coefficient: the cavity's C_L is a 1e-7 remainder of cancelling
    # wall forces, so its own size is no scale for rounding
    sv = max(abs(ov["cd"]), abs(ov["cl"]))
    sd = max(abs(od["cd"]), abs(od["cl"]))
    for key in ("cd", "cl"):
        assert abs(val[key] - ov[key]) <= 1e-10 * sv, key
        assert abs(dv[key] - od[key]) <= 1e-8 * sd, (key, dv[key], od[key])
