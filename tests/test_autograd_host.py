"""CPU checks of the parameter map behind the autograd wrapper (``AirfoilForces``): no GPU is
needed to build the model, to form the case at given parameters, or to form the directions that
the backward pass projects the adjoint on.

  - At the base parameters the case is the base case.
  - d(boundary values)/d alpha and d(boundary values)/d ratio, as the backward pass uses them,
    equal central differences of the map p -> boundary values.
  - The node displacements move exactly the chosen wall nodes along their outward unit normals.
"""
import dataclasses
import math

import numpy as np

from paper_1812_00394_gb300 import autograd as fa, fvlbm, meshgen as mg


def _model():
    base = mg.naca0012_cmesh(n_target=2500, re_c=1e4, alpha_deg=4.0)
    m = base.mesh.normalized()
    wall = np.unique(m.bedge_nodes[m.bedge_type == mg.BC_WALL])
    upper = wall[m.xy[wall, 1] > 0]
    picks = [int(upper[np.argmin(np.abs(m.xy[upper, 0] - x))]) for x in (0.2, 0.6)]
    return fa.AirfoilForces(base, picks, steps=10), m


def test_base_parameters_give_the_base_case():
    model, m = _model()
    p0 = np.array([math.radians(4.0), 1.0, 0.0, 0.0])
    case = model.case_at(p0)
    np.testing.assert_allclose(case.mesh.bedge_val, m.bedge_val, rtol=1e-14, atol=1e-17)
    assert np.array_equal(case.mesh.xy, m.xy)
    assert case.dt == model.dt and model.dt == fvlbm.check_case(model.base)[1]


def test_boundary_value_directions_match_central_differences():
    model, _ = _model()
    p0 = np.array([math.radians(4.0), 1.3, 0.0, 0.0])
    d_alpha, d_ratio = model._bval_directions(model.case_at(p0), p0)
    for q, d in ((0, d_alpha), (1, d_ratio)):
        h = 1e-6
        e = np.zeros_like(p0)
        e[q] = h
        fd = (model.case_at(p0 + e).mesh.bedge_val - model.case_at(p0 - e).mesh.bedge_val) / (2 * h)
        assert np.abs(fd - d).max() <= 1e-7 * np.abs(d).max(), q
        assert np.abs(d).max() > 0


def test_displacements_move_the_chosen_wall_nodes_along_outward_normals():
    model, m = _model()
    n = model.normals
    np.testing.assert_allclose(np.linalg.norm(n, axis=1), 1.0, rtol=1e-14)
    wall = np.unique(m.bedge_nodes[m.bedge_type == mg.BC_WALL])
    centre = m.xy[wall].mean(0)
    assert np.all(np.einsum("jc,jc->j", n, m.xy[model.wall_nodes] - centre) > 0)
    p = np.array([math.radians(4.0), 1.0, 1e-4, -2e-4])
    xy = model.case_at(p).mesh.xy
    moved = np.flatnonzero(np.any(xy != m.xy, axis=1))
    assert sorted(moved) == sorted(model.wall_nodes)
    np.testing.assert_allclose(xy[model.wall_nodes] - m.xy[model.wall_nodes], p[2:, None] * n,
                               rtol=1e-9, atol=1e-18)
    assert fvlbm.check_case(dataclasses.replace(model.case_at(p)))[0] == 0
