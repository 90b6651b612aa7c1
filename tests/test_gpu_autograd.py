"""GPU check of the autograd wrapper: gradients of (C_L, C_D) with respect to the free-stream
angle, the inflow eddy-viscosity ratio and wall-node normal displacements, taken by
torch.autograd through the tangent-mode backward (SST case) and through the adjoint backward
(laminar case), against central differences of the forward map and against each other."""
import math

import numpy as np
import pytest
import torch

from paper_1812_00394_gb300 import autograd as fa, meshgen as mg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", ["tangent", "adjoint"])
def test_autograd_gradients_match_central_differences(mode):
    base = mg.naca0012_cmesh(n_target=2500, re_c=1e4, alpha_deg=4.0)
    m = base.mesh.normalized()
    wall = np.unique(m.bedge_nodes[m.bedge_type == mg.BC_WALL])
    upper = wall[m.xy[wall, 1] > 0]
    picks = [int(upper[np.argmin(np.abs(m.xy[upper, 0] - x))]) for x in (0.1, 0.4, 0.8)]
    model = fa.AirfoilForces(base, picks, steps=30, device=0, mode=mode)
    p0 = np.array([math.radians(4.0), 1.0, 0.0, 0.0, 0.0])
    p = torch.tensor(p0, requires_grad=True)
    out = fa.forces(model, p)
    loss = out[0] + 0.5 * out[1]
    loss.backward()
    g = p.grad.numpy()
    steps = [1e-5, 1e-5, 1e-6, 1e-6, 1e-6]
    for q, h in enumerate(steps):
        e = np.zeros_like(p0)
        e[q] = h
        vp, vm = model.value(p0 + e), model.value(p0 - e)
        fd = ((vp[0] + 0.5 * vp[1]) - (vm[0] + 0.5 * vm[1])) / (2 * h)
        tol = 1e-5 if q < 2 else 1e-4
        assert abs(g[q] - fd) <= tol * abs(fd) + 1e-9, (q, g[q], fd)
    # the forward value is the FP64 step of the base case at p0
    np.testing.assert_allclose(out.detach().numpy(), model.value(p0), rtol=0, atol=0)


def _laminar_model(mode):
    import dataclasses
    base = dataclasses.replace(mg.naca0012_cmesh(n_target=2500, re_c=2000.0, alpha_deg=3.0),
                               sst=False)
    m = base.mesh.normalized()
    wall = np.unique(m.bedge_nodes[m.bedge_type == mg.BC_WALL])
    upper = wall[m.xy[wall, 1] > 0]
    lower = wall[m.xy[wall, 1] < 0]
    picks = [int(upper[np.argmin(np.abs(m.xy[upper, 0] - 0.3))]),
             int(lower[np.argmin(np.abs(m.xy[lower, 0] - 0.6))])]
    return fa.AirfoilForces(base, picks, steps=25, device=0, mode=mode)


def test_autograd_adjoint_backward_matches_tangent_and_fd():
    p0 = np.array([math.radians(3.0), 1.0, 0.0, 0.0])
    grads = {}
    for mode in ("adjoint", "tangent"):
        model = _laminar_model(mode)
        assert model.mode == mode
        p = torch.tensor(p0, requires_grad=True)
        out = fa.forces(model, p)
        (0.8 * out[0] - 2.0 * out[1]).backward()
        grads[mode] = p.grad.numpy().copy()
    ga, gt = grads["adjoint"], grads["tangent"]
    assert ga[1] == 0.0 and abs(gt[1]) <= 1e-14   # omega_b does not enter a laminar step
    for q in (0, 2, 3):
        assert abs(ga[q] - gt[q]) <= 1e-8 * abs(gt[q]), (q, ga[q], gt[q])
    model = _laminar_model("auto")
    assert model.mode == "adjoint"
    for q, h in ((0, 1e-5), (2, 1e-6)):
        e = np.zeros_like(p0)
        e[q] = h
        vp, vm = model.value(p0 + e), model.value(p0 - e)
        fd = ((0.8 * vp[0] - 2.0 * vp[1]) - (0.8 * vm[0] - 2.0 * vm[1])) / (2 * h)
        assert abs(ga[q] - fd) <= 1e-5 * abs(fd), (q, ga[q], fd)


def test_autograd_sst_adjoint_backward_matches_tangent():
    """SST NACA 0012 with alpha, the inflow ratio and two wall nodes: the default backward is the
    adjoint, and it equals the tangent backward."""
    base = mg.naca0012_cmesh(n_target=2500, re_c=1e4, alpha_deg=4.0)
    m = base.mesh.normalized()
    wall = np.unique(m.bedge_nodes[m.bedge_type == mg.BC_WALL])
    upper = wall[m.xy[wall, 1] > 0]
    picks = [int(upper[np.argmin(np.abs(m.xy[upper, 0] - x))]) for x in (0.2, 0.6)]
    p0 = np.array([math.radians(4.0), 1.0, 0.0, 0.0])
    grads = {}
    for mode in ("auto", "tangent"):
        model = fa.AirfoilForces(base, picks, steps=30, device=0, mode=mode)
        assert model.mode == ("adjoint" if mode == "auto" else "tangent")
        p = torch.tensor(p0, requires_grad=True)
        out = fa.forces(model, p)
        (out[0] + 0.5 * out[1]).backward()
        grads[mode] = p.grad.numpy().copy()
    for q in range(4):
        assert abs(grads["auto"][q] - grads["tangent"][q]) <= 1e-8 * abs(grads["tangent"][q]) + 1e-14, q


def test_step_forces_gradients_match_central_differences():
    """The full-input autograd function: a loss of (C_D, C_L) after 20 FP64 steps of a laminar
    airfoil, differentiated by one adjoint solve with respect to f0, the boundary values and the
    node positions, against central differences along a direction of each input."""
    import dataclasses
    base = dataclasses.replace(mg.naca0012_cmesh(n_target=1500, re_c=2000.0, alpha_deg=4.0), sst=False)
    model = fa.StepForces(base, steps=20, device=0)
    f0, bv, xy = (t.requires_grad_(True) for t in model.inputs())
    out = fa.step_forces(model, f0, bv, xy)
    (1.5 * out[0] - out[1]).backward()
    rng = np.random.default_rng(17)
    # node direction: a dilation about the centroid of the nodes.  It keeps every face normal,
    # so no upwind choice on an e.n = 0 face (the quads of the boundary layer) changes sides
    # within the differences, where the derivative is one-sided
    xy0 = xy.detach().numpy()
    dirs = [1e-3 * rng.standard_normal(tuple(f0.shape)), np.zeros(tuple(bv.shape)),
            1e-3 * (xy0 - xy0.mean(0))]
    dirs[1][:, :3] = 1e-2 * rng.standard_normal((bv.shape[0], 3))
    base_in = [t.detach().numpy() for t in (f0, bv, xy)]
    for q, grad in enumerate((f0.grad, bv.grad, xy.grad)):
        h = (1e-5, 1e-5, 1e-4)[q]
        vals = []
        for sgn in (1.0, -1.0):
            args = [a.copy() for a in base_in]
            args[q] = args[q] + sgn * h * dirs[q]
            s = model.solver(*args)
            s.step(model.steps)
            f = s.forces()
            s.close()
            vals.append(1.5 * f["cd"] - f["cl"])
        fd = (vals[0] - vals[1]) / (2 * h)
        adj = float(np.sum(grad.numpy() * dirs[q]))
        assert abs(adj - fd) <= 1e-5 * abs(fd), (q, adj, fd)
