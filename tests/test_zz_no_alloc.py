"""Allocation-free statistics entry point (fvlbm_stats_reduce_static).

It serves callers that cannot allocate device memory; it must give the same FP64 residual and
mass as fvlbm_step's own statistics.  This file is collected last so that a failure here never
hides another test.
"""
import numpy as np
import pytest

from paper_1812_00394_gb300 import fvlbm, meshgen as mg

pytestmark = pytest.mark.gpu


def _areas(mesh):
    out = np.empty(mesh.n_cells)
    for i in range(mesh.n_cells):
        q = mesh.xy[mesh.cell_nodes[mesh.cell_ptr[i]:mesh.cell_ptr[i + 1]]]
        out[i] = 0.5 * np.sum(q[:, 0] * np.roll(q[:, 1], -1) - np.roll(q[:, 0], -1) * q[:, 1])
    return out


def test_static_stats_match_step_stats_twice():
    torch = pytest.importorskip("torch")
    lib = fvlbm.load()
    case = mg.cavity_delaunay(h_boundary=1 / 60, n_target=9000, re=400.0, z=5.0, seed=11)
    s = fvlbm.Solver(case, precision=fvlbm.FVLBM_FP64, device=0)
    area = torch.tensor(_areas(case.mesh), dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    s.step(5)
    for _ in range(2):                                   # two calls in a row
        before = s.fields()
        st = s.step(1, stats=True)
        after = s.fields()
        dev = {k: torch.tensor(v, dtype=torch.float64, device="cuda")
               for k, v in (("uo", before["u"]), ("vo", before["v"]), ("un", after["u"]),
                            ("vn", after["v"]), ("rho", after["rho"]))}
        torch.cuda.synchronize()
        rc = lib.fvlbm_stats_reduce_static(dev["uo"].data_ptr(), dev["vo"].data_ptr(),
                                           dev["un"].data_ptr(), dev["vn"].data_ptr(),
                                           dev["rho"].data_ptr(), area.data_ptr(),
                                           case.mesh.n_cells, out.data_ptr(), None)
        assert rc == 0
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        residual = np.sqrt(o[0]) / np.sqrt(o[1])
        assert abs(residual - st["residual"]) <= 1e-10 * st["residual"]
        assert abs(o[2] - st["mass"]) <= 1e-12 * st["mass"]
        assert o[3] == 0.0


def test_static_stats_rejects_oversize():
    """Sizes beyond the static scratch capacity are rejected before any launch."""
    torch = pytest.importorskip("torch")
    lib = fvlbm.load()
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = x.data_ptr()
    rc = lib.fvlbm_stats_reduce_static(p, p, p, p, p, p, 4194304 + 1, p, None)
    assert rc == -3
