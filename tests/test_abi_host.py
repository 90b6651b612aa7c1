"""CPU checks of the C ABI: the library builds, loads and exports every declared entry point,
and the host-side validation rejects bad input before any device work (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1812_00394_gb300 import fvlbm, meshgen as mg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            with open(os.path.join(ROOT, "include", fn)) as fh:
                names |= set(re.findall(r"\b(fvlbm_[a-z_0-9]+)\s*\(", fh.read()))
    return names


def test_library_exports_every_declared_symbol():
    lib = fvlbm.load()
    declared = _declared()
    assert declared, "no declarations found"
    for name in sorted(declared):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert declared <= set(fvlbm.EXPORTS) | declared


def test_strerror_codes():
    assert fvlbm.strerror(0) == "ok"
    assert "diverged" in fvlbm.strerror(-6)
    assert fvlbm.strerror(12345) == "unknown error"


def _create(case, **kw):
    pack = fvlbm._Pack(case, fvlbm.FVLBM_FP64)
    for k, v in kw.items():
        setattr(pack.params, k, v)
    h = C.c_void_p()
    rc = fvlbm.load().fvlbm_create(C.byref(pack.mesh), C.byref(pack.bc), C.byref(pack.params), 0,
                                   None, C.byref(h))
    return rc


def test_rejects_clockwise_cell():
    case = mg.cavity_quad(4)
    m = case.mesh
    cn = m.cell_nodes.copy().reshape(-1, 4)
    cn[5] = cn[5][::-1]
    bad = mg.Mesh(m.xy, m.cell_ptr, cn.ravel(), m.bedge_nodes, m.bedge_type, m.bedge_val)
    assert _create(mg.Case(bad, nu=1e-3, dt=1e-3)) == -1


def test_rejects_missing_boundary_edge():
    case = mg.cavity_quad(4)
    m = case.mesh
    bad = mg.Mesh(m.xy, m.cell_ptr, m.cell_nodes, m.bedge_nodes[1:], m.bedge_type[1:],
                  m.bedge_val[1:])
    assert _create(mg.Case(bad, nu=1e-3, dt=1e-3)) == -2


def test_rejects_interior_edge_as_boundary():
    case = mg.cavity_quad(4)
    m = case.mesh
    bn = m.bedge_nodes.copy()
    bn[0] = [5, 6]   # an interior edge of the 4x4 grid (nodes 5-6 lie inside)
    bad = mg.Mesh(m.xy, m.cell_ptr, m.cell_nodes, bn, m.bedge_type, m.bedge_val)
    assert _create(mg.Case(bad, nu=1e-3, dt=1e-3)) == -2


@pytest.mark.parametrize("kw", [{"nu": 0.0}, {"dt": 0.0, "cfl": 0.0}, {"precision": 7}])
def test_rejects_bad_params(kw):
    case = mg.cavity_quad(4)
    case.dt = 1e-3
    assert _create(case, **kw) == -3


def test_oracle_not_imported_by_product():
    for fn in ("fvlbm.py", "build.py", "__init__.py", "meshgen.py"):
        with open(os.path.join(ROOT, "paper_1812_00394_gb300", fn)) as fh:
            src = fh.read()
            assert "import oracle" not in src and "from oracle" not in src, fn


def test_splitmix64_reference_values():
    """SplitMix64 with seed 0: the first outputs of the published generator are
    0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F."""
    u = mg.splitmix64_uniform(0, 3)
    words = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    expect = np.array([2.0 * ((w >> 11) * 2.0 ** -53) - 1.0 for w in words])
    assert np.array_equal(u, expect)


def test_rejects_empty_mesh():
    m = mg.Mesh(np.zeros((3, 2)), np.zeros(1, np.int32), np.zeros(0, np.int32),
                np.zeros((0, 2), np.int32), np.zeros(0, np.int32), np.zeros((0, 5)))
    assert _create(mg.Case(m, nu=1e-3, dt=1e-3)) == -1


def test_rejects_polygon_with_five_nodes():
    xy = np.array([[0, 0], [1, 0], [1.5, 0.8], [0.5, 1.4], [-0.4, 0.8]], float)
    cells = np.arange(5, dtype=np.int32)
    bn = np.stack([np.arange(5), (np.arange(5) + 1) % 5], 1).astype(np.int32)
    m = mg.Mesh(xy, np.array([0, 5], np.int32), cells, bn, np.zeros(5, np.int32),
                np.tile([1.0, 0, 0, 0, 0], (5, 1)))
    assert _create(mg.Case(m, nu=1e-3, dt=1e-3)) == -1


def test_derivative_entry_points_reject_a_null_handle():
    """The adjoint and tangent entry points check their handle before any device work."""
    lib = fvlbm.load()
    w = np.array([1.0, 0.0])
    out = np.zeros(4)
    assert lib.fvlbm_adjoint(None, 0, 1, w.ctypes.data_as(C.c_void_p), None, None, None, None) \
        == fvlbm.FVLBM_ERR_BAD_PARAM
    assert lib.fvlbm_set_adjoint_budget(None, 0) == fvlbm.FVLBM_ERR_BAD_PARAM
    assert lib.fvlbm_forces_tangent(None, 0, 0.0, out.ctypes.data_as(C.c_void_p),
                                    out.ctypes.data_as(C.c_void_p)) == fvlbm.FVLBM_ERR_BAD_PARAM
    assert lib.fvlbm_tangent_seed(None, 0, None, None) == fvlbm.FVLBM_ERR_BAD_PARAM
