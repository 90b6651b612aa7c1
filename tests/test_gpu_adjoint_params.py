"""fvlbm_adjoint_params: the parameter-level gradient of w . (C_D, C_L) behind the C ABI.

One adjoint solve on the GPU (FP64) and the library's own chain rule to the free-stream angle,
the inflow eddy-viscosity ratio and wall-node normal displacements (the Sec. 4.3 airfoil
parameters), checked against central differences of the FP64 CPU oracle run on the same
parameter map (autograd.AirfoilForces.case_at forms the perturbed cases), to 1e-5 relative.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1812_00394_gb300 import autograd as fa, fvlbm, meshgen as mg

pytestmark = pytest.mark.gpu

STEPS = 20


def _model(sst):
    import dataclasses
    if sst:
        base = mg.naca0012_cmesh(n_target=2500, re_c=1e4, alpha_deg=4.0)
    else:
        base = dataclasses.replace(mg.naca0012_cmesh(n_target=2500, re_c=2000.0, alpha_deg=3.0),
                                   sst=False)
    m = base.mesh.normalized()
    wall = np.unique(m.bedge_nodes[m.bedge_type == mg.BC_WALL])
    upper = wall[m.xy[wall, 1] > 0]
    lower = wall[m.xy[wall, 1] < 0]
    picks = [int(upper[np.argmin(np.abs(m.xy[upper, 0] - 0.3))]),
             int(lower[np.argmin(np.abs(m.xy[lower, 0] - 0.6))])]
    return fa.AirfoilForces(base, picks, steps=STEPS, device=0, mode="adjoint")


def _oracle_J(model, p, w):
    o = Oracle(model.case_at(p))
    o.step(STEPS)
    f = o.forces()
    return w[0] * f["cd"] + w[1] * f["cl"], f


@pytest.mark.parametrize("sst", [False, True], ids=["laminar", "sst"])
def test_adjoint_params_match_oracle_central_differences(sst):
    model = _model(sst)
    alpha = math.radians(4.0 if sst else 3.0)
    p0 = np.array([alpha, 1.3, 0.0, 0.0])
    w = (0.7, -0.4)                                   # J = 0.7 C_D - 0.4 C_L
    s = fvlbm.Solver(model.case_at(p0), precision=fvlbm.FVLBM_FP64, device=0, kernel_path=1)
    r = s.adjoint_params(STEPS, w_cd=w[0], w_cl=w[1], wall_nodes=model.wall_nodes,
                         wall_normals=model.normals)
    s.close()
    J0, f0 = _oracle_J(model, p0, w)
    assert abs(r["J"] - J0) <= 1e-10 * abs(J0)
    assert abs(r["cd"] - f0["cd"]) <= 1e-10 * abs(f0["cd"]) and abs(r["cl"] - f0["cl"]) <= 1e-10 * abs(f0["cl"])
    grad = np.concatenate([[r["dalpha"], r["dratio"]], r["dwall"]])
    steps = [1e-5, 1e-4, 1e-6, 1e-6]
    for q, h in enumerate(steps):
        e = np.zeros_like(p0)
        e[q] = h
        fd = (_oracle_J(model, p0 + e, w)[0] - _oracle_J(model, p0 - e, w)[0]) / (2 * h)
        if not sst and q == 1:
            assert grad[q] == 0.0 and abs(fd) < 1e-12   # no SST: the ratio does not enter
            continue
        assert abs(grad[q] - fd) <= 1e-5 * abs(fd) + 1e-10, (q, grad[q], fd)


def test_adjoint_params_without_wall_nodes_and_bad_arguments():
    model = _model(False)
    p0 = np.array([math.radians(3.0), 1.0, 0.0, 0.0])
    s = fvlbm.Solver(model.case_at(p0), precision=fvlbm.FVLBM_FP64, device=0, kernel_path=1)
    r = s.adjoint_params(5, w_cd=1.0, w_cl=0.0)
    assert r["dwall"].shape == (0,) and np.isfinite(r["dalpha"])
    with pytest.raises(fvlbm.FvlbmError) as ei:
        s.adjoint_params(5, 1.0, 0.0, wall_nodes=[10 ** 8], wall_normals=[[0.0, 1.0]])
    assert ei.value.code == fvlbm.FVLBM_ERR_BAD_PARAM
    s.close()
    s32 = fvlbm.Solver(model.case_at(p0), precision=fvlbm.FVLBM_FP32_DEV, device=0)
    with pytest.raises(fvlbm.FvlbmError) as ei:
        s32.adjoint_params(2, 1.0, 0.0)
    assert ei.value.code == fvlbm.FVLBM_ERR_NOT_SUPPORTED
    s32.close()
