"""A mesh split into parts on one GPU: one handle per part, ghosts exchanged through the C ABI
(fvlbm_get_cells / fvlbm_set_cells) after every step, against the whole-mesh handle.

All parts share the GPU and run one after another (no kernel waits on another part), so this
checks the library side of the partition -- the cell-list calls, the whole mesh's wall distance
and time step in every part, the per-edge wall force -- while the multi-rank exchange itself is
covered on CPU ranks.  FP64 on both sides: the owned cells match the whole mesh to rounding
(the ghosts pass through the double interface, f - w rho0 -> f -> f - w rho0).
"""
import dataclasses

import numpy as np
import pytest

from paper_1812_00394_gb300 import fvlbm, meshgen as mg
from paper_1812_00394_gb300.partition import LocalPartitionedRun, MeshPartition

pytestmark = pytest.mark.gpu

FP64, FP32 = fvlbm.FVLBM_FP64, fvlbm.FVLBM_FP32_DEV


def _perturbed(case, seed):
    rho, u, v, k, w = case.init_arrays()
    n = rho.shape[0]
    r = [mg.splitmix64_uniform(seed + j, n) for j in range(5)]
    du = 0.02 * case.uref
    return dataclasses.replace(case, rho=rho * (1 + 0.01 * r[0]), u=u + du * r[1], v=v + du * r[2],
                               k=k * (1 + 0.3 * r[3]), omega=w * (1 + 0.3 * r[4]))


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _split(case, nparts):
    _, wd = fvlbm.case_geometry(case)
    rc, dt, why = fvlbm.check_case(case)
    assert rc == 0, why
    return MeshPartition(case, nparts, dt=dt, wdist=wd if case.sst else None)


@pytest.mark.parametrize("path", [0, 1, 2], ids=["fused", "twopass", "facevalue"])
@pytest.mark.parametrize("name,nparts", [("naca_sst", 3), ("cavity", 2)])
def test_parts_on_one_gpu_match_the_whole_mesh(name, nparts, path):
    case = {"naca_sst": lambda: mg.naca0012_cmesh(n_target=6000, re_c=1e4, alpha_deg=4.0),
            "cavity": lambda: mg.cavity_delaunay(h_boundary=1 / 40, n_target=4000, re=400.0,
                                                 z=5.0, seed=3)}[name]()
    case = _perturbed(case, 21)
    pt = _split(case, nparts)
    run = LocalPartitionedRun(pt, lambda c: fvlbm.Solver(c, precision=FP64, device=0, kernel_path=path))
    whole = fvlbm.Solver(case, precision=FP64, device=0, kernel_path=path)
    run.step(8)
    whole.step(8)
    assert _rel(run.get_f(), whole.get_f()) < 1e-12
    fl, fw = run.fields(), whole.fields()
    for key in ("u", "v", "k", "omega", "nut"):
        assert _rel(fl[key] + 1.0, fw[key] + 1.0) < 1e-12, key
    fr, fo = run.forces(), whole.forces()
    scale = max(abs(fo["cd"]), abs(fo["cl"]), 1e-300)
    assert abs(fr["cd"] - fo["cd"]) <= 1e-10 * scale and abs(fr["cl"] - fo["cl"]) <= 1e-10 * scale
    run.close()
    whole.close()


def test_cell_list_calls_and_wall_distance():
    """get_cells / set_cells move exactly the listed cells (FP32 handle: the deviation values
    pass unchanged); an id outside the instance is refused; fvlbm_forces_edges adds up to
    fvlbm_forces; a wall distance set from the whole mesh changes the SST step exactly as the
    one create computed when they are equal."""
    case = mg.naca0012_cmesh(n_target=4000, re_c=1e4, alpha_deg=4.0)
    s = fvlbm.Solver([mg.cavity_quad(12, re=400.0), case], precision=FP32, device=0)
    s.step(5)
    n = s.cells[1]
    cells = np.array([0, 7, n - 1, 123], np.int32)
    f, k, w, nt = s.get_cells(cells, i=1)
    full = s.get_f(1)
    np.testing.assert_array_equal(f, full[cells])
    fl = s.fields(1)
    np.testing.assert_array_equal(k, fl["k"][cells])
    np.testing.assert_array_equal(nt, fl["nut"][cells])
    other = s.get_f(0)
    s.set_cells(cells, f * 1.0, k * 2.0, w, nt, i=1)
    np.testing.assert_array_equal(s.get_f(1), full)
    k2 = s.fields(1)["k"]
    np.testing.assert_array_equal(k2[cells], 2.0 * k)
    mask = np.ones(n, bool)
    mask[cells] = False
    np.testing.assert_array_equal(k2[mask], fl["k"][mask])
    np.testing.assert_array_equal(s.get_f(0), other)
    with pytest.raises(fvlbm.FvlbmError) as ei:
        s.get_cells(np.array([n], np.int32), i=1)
    assert ei.value.code == fvlbm.FVLBM_ERR_BAD_PARAM
    with pytest.raises(fvlbm.FvlbmError):
        s.set_cells(cells, k=k, i=1)          # k without omega and nu_t
    fe = s.forces_edges(1)
    fo = s.forces(1)
    assert abs(fe[:, 0].sum() - fo["fx"]) <= 1e-12 * abs(fo["fx"])
    assert abs(fe[:, 1].sum() - fo["fy"]) <= 1e-12 * max(abs(fo["fy"]), abs(fo["fx"]))
    s.close()
    # the wall distance create computes, set again, changes nothing; a different one does
    _, wd = fvlbm.case_geometry(case)
    a = fvlbm.Solver(case, precision=FP64, device=0)
    b = fvlbm.Solver(case, precision=FP64, device=0)
    c = fvlbm.Solver(case, precision=FP64, device=0)
    b.set_wall_distance(wd)
    c.set_wall_distance(wd * 1.5)
    for x in (a, b, c):
        x.step(4)
    np.testing.assert_array_equal(a.get_f(), b.get_f())
    assert _rel(c.fields()["nut"], a.fields()["nut"]) > 1e-6
    with pytest.raises(fvlbm.FvlbmError):
        a.set_wall_distance(np.zeros(a.cells[0]))


@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_device_buffer_exchange_equals_host_exchange(prec):
    """The ghost rows moved through device buffers (fvlbm_set_exchange_list, then
    fvlbm_pack_cells_dev / fvlbm_unpack_cells_dev on the handles' streams) give bit for bit what
    the host path (fvlbm_get_cells / fvlbm_set_cells) gives; bad lists and ids are refused."""
    case = _perturbed(mg.naca0012_cmesh(n_target=6000, re_c=1e4, alpha_deg=4.0), 22)
    pt = _split(case, 3)
    make = lambda c: fvlbm.Solver(c, precision=prec, device=0, kernel_path=2)  # noqa: E731
    host = LocalPartitionedRun(pt, make)
    dev = LocalPartitionedRun(pt, make, device_buffers=True)
    host.step(6)
    dev.step(6)
    np.testing.assert_array_equal(dev.get_f(), host.get_f())
    fd, fh = dev.fields(), host.fields()
    for key in ("k", "omega", "nut"):
        np.testing.assert_array_equal(fd[key], fh[key])
    s = dev.solvers[0]
    with pytest.raises(fvlbm.FvlbmError) as ei:
        s.set_exchange_list(np.array([0, s.cells[0]], np.int32))
    assert ei.value.code == fvlbm.FVLBM_ERR_BAD_PARAM
    with pytest.raises(fvlbm.FvlbmError):
        s.pack_cells_dev(10 ** 6, 0)
    host.close()
    dev.close()
