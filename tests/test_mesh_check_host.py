"""CPU checks of the host-side mesh validation (``fvlbm_check_mesh`` and the consistency checks
that ``fvlbm_create`` runs on every prepared instance).

  - A small native program (tests/native/prepared_check.cpp) built here with g++ from the
    library's host sources preprocesses a mesh and passes the checks.  Then, one at a time, it
    plants mistakes in the prepared arrays and shows that each is caught:
      - an index out of range, and a link that is not mutual;
      - a flipped or shifted normal;
      - swapped least-squares components;
      - a wrong offset or area;
      - a bad time step.
  - Through the C ABI, with no GPU: the generated meshes of every workload pass.  The CFL step
    of a uniform quad grid is cfl h / 2: the diagonal velocities leave through two faces.
  - A periodic pair whose edges are not translates by the shift is rejected.
  - The error code of a bad input equals the one ``fvlbm_create`` returns for it.
  - What the preprocessing hands the kernels matches the oracle's own, independent geometry:
    areas, wall distances, the CFL step and least-squares gradients (a second native program,
    tests/native/prepared_geometry_dump.cpp).
"""
import ctypes as C
import dataclasses
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from paper_1812_00394_gb300 import fvlbm, meshgen as mg

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1812_00394_gb300", "csrc")

# planted mistake -> words of the message that names the check that must catch it
PLANTS = {
    "nbr_out_of_range": "link is not mutual", "back_slot": "link is not mutual",
    "link_not_mutual": "link is not mutual", "open_face": "open face",
    "bowner": "boundary face link", "bface_twice": "boundary face link",
    "padding_face": "padding cell", "padding_slot": "slot past the faces",
    "slot_past_faces": "slot past the faces", "perm_duplicate": "permutation",
    "bedge_order": "input edge index", "btype_periodic": "type", "array_size": "array sizes",
    "area": "area disagrees", "gq_shift": "relative to the centroid",
    "gq_node_order": "outward normal", "sn_sign": "outward normal", "sn_slot": "outward normal",
    "rown_shift": "face midpoint", "rnbr_own": "neighbour-side face offset",
    "dvec_not_reversed": "reverse of the neighbour", "dinv": "1/|d|",
    "boundary_dvec": "boundary face offsets", "lsq_swap": "least-squares",
    "lsq_dropped_face": "least-squares", "bnrm_sign": "normal or length",
    "blen": "normal or length", "wdist_nan": "wall distance", "dt_zero": "time step",
    "dt_cell_negative": "local time step",
}


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("prepcheck") / "prepared_check")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fopenmp", "-I", os.path.join(ROOT, "include"),
                           "-I", CSRC, os.path.join(HERE, "native", "prepared_check.cpp"),
                           os.path.join(CSRC, "fvlbm_host.cpp"), "-o", out])
    return out


def _run(checker, path, m):
    m = m.normalized()
    with open(path, "wb") as fh:
        fh.write(struct.pack("<i", m.n_nodes)); fh.write(m.xy.astype("<f8").tobytes())
        fh.write(struct.pack("<i", m.n_cells)); fh.write(m.cell_ptr.astype("<i4").tobytes())
        fh.write(m.cell_nodes.astype("<i4").tobytes())
        fh.write(struct.pack("<i", m.n_bedges)); fh.write(m.bedge_nodes.astype("<i4").tobytes())
        fh.write(m.bedge_type.astype("<i4").tobytes()); fh.write(m.bedge_val.astype("<f8").tobytes())
        fh.write(struct.pack("<i", m.periodic_pairs.shape[0]))
        fh.write(m.periodic_pairs.astype("<i4").tobytes()); fh.write(m.periodic_shift.astype("<f8").tobytes())
    res = subprocess.run([checker, path], capture_output=True, text=True, check=True).stdout
    out = {}
    for ln in res.splitlines():
        name, rc, *msg = ln.split(" ")
        out[name] = (int(rc), " ".join(msg))
    return out


@pytest.mark.parametrize("name", ["jittered_quads", "periodic_triangles"])
def test_planted_mistakes_are_caught(checker, tmp_path, name):
    if name == "jittered_quads":   # 400 cells: padding cells follow
        m = mg.cavity_quad(20, re=400.0, jitter=0.2, seed=3).mesh
    else:                          # triangles, periodic in x, walls above and below
        m = mg.couette_channel(12, 10, kind="tri", jitter=0.2, seed=4)
    out = _run(checker, str(tmp_path / "mesh.bin"), m)
    assert out["valid"] == (0, ""), out["valid"]
    assert out["valid_dual"] == (0, ""), out["valid_dual"]
    for plant, words in PLANTS.items():
        rc, msg = out[plant]
        assert rc < 0, (plant, rc, msg)
        assert words in msg, (plant, msg)


def _cases():
    return {
        "cavity_quad_64": mg.cavity_quad(64),
        "cavity_delaunay": mg.cavity_delaunay(n_target=3000),
        "bfs_hybrid": mg.bfs_hybrid(8000),
        "naca0012_sst": mg.naca0012_cmesh(n_target=5000),
        "naca0012_laminar": dataclasses.replace(mg.naca0012_cmesh(n_target=2500, re_c=2000.0), sst=False),
        "periodic_box_tri": mg.Case(mg.periodic_box(12, kind="tri", jitter=0.2, seed=2), nu=1e-3, cfl=0.5),
        "couette_stretched": mg.Case(mg.couette_channel(6, 40, stretch=1.08), nu=0.01, cfl=0.5),
    }


@pytest.mark.parametrize("name", list(_cases()))
def test_generated_meshes_pass(name):
    case = _cases()[name]
    for prec in (fvlbm.FVLBM_FP64, fvlbm.FVLBM_FP32_DEV, fvlbm.FVLBM_FP64_TANGENT):
        rc, dt, why = fvlbm.check_case(case, precision=prec)
        assert rc == 0 and why == "", (name, prec, rc, why)
        assert dt > 0.0


def test_cfl_step_of_a_uniform_quad_grid():
    """Upwind outflow rate max_alpha sum_m max(e_alpha . n_m, 0) dl_m / A on an h x h square:
    2 / h (a diagonal velocity leaves through two faces), so dt = cfl h / 2."""
    for n, cfl in ((16, 0.5), (64, 0.5), (40, 0.9)):
        case = dataclasses.replace(mg.cavity_quad(n), cfl=cfl, dt=0.0)
        rc, dt, why = fvlbm.check_case(case)
        assert rc == 0, why
        assert abs(dt - cfl * (1.0 / n) / 2.0) <= 1e-14, (n, dt)


def test_periodic_pair_must_be_a_translate():
    m = mg.periodic_box(8, kind="quad")
    case = mg.Case(m, nu=1e-3, cfl=0.5)
    assert fvlbm.check_case(case)[0] == 0
    bad = m.periodic_shift.copy()
    bad[0, 0] += 1e-3
    rc, _, why = fvlbm.check_case(mg.Case(dataclasses.replace(m, periodic_shift=bad), nu=1e-3, cfl=0.5))
    assert rc == fvlbm.FVLBM_ERR_BAD_BC and "moved by the shift" in why, (rc, why)
    pairs = m.periodic_pairs.copy()
    pairs[0, 1], pairs[1, 1] = pairs[1, 1], pairs[0, 1]   # two edges glued to the wrong partners
    rc, _, why = fvlbm.check_case(mg.Case(dataclasses.replace(m, periodic_pairs=pairs), nu=1e-3, cfl=0.5))
    assert rc == fvlbm.FVLBM_ERR_BAD_BC, (rc, why)


def _create_rc(case, **kw):
    pack = fvlbm._Pack(case, fvlbm.FVLBM_FP64)
    for k, v in kw.items():
        setattr(pack.params, k, v)
    h = C.c_void_p()
    return fvlbm.load().fvlbm_create(C.byref(pack.mesh), C.byref(pack.bc), C.byref(pack.params), 0,
                                     None, C.byref(h)), pack


def test_error_codes_match_create():
    base = mg.cavity_quad(4)
    m = base.mesh
    cw = m.cell_nodes.copy().reshape(-1, 4)
    cw[5] = cw[5][::-1]
    bad_cases = [
        (mg.Case(mg.Mesh(m.xy, m.cell_ptr, cw.ravel(), m.bedge_nodes, m.bedge_type, m.bedge_val),
                 nu=1e-3, dt=1e-3), {}),
        (mg.Case(mg.Mesh(m.xy, m.cell_ptr, m.cell_nodes, m.bedge_nodes[1:], m.bedge_type[1:],
                         m.bedge_val[1:]), nu=1e-3, dt=1e-3), {}),
        (mg.Case(m, nu=1e-3, dt=1e-3), {"nu": 0.0}),
        (mg.Case(m, nu=1e-3, dt=1e-3), {"precision": 7}),
    ]
    for case, kw in bad_cases:
        rc_create, _ = _create_rc(case, **kw)
        pack = fvlbm._Pack(case, fvlbm.FVLBM_FP64)
        for k, v in kw.items():
            setattr(pack.params, k, v)
        rc, _, why = fvlbm.fvlbm_check_mesh(pack.mesh, pack.bc, pack.params)
        assert rc == rc_create and rc < 0 and why, (kw, rc, rc_create, why)
    # fvlbm_create checks the scheme after it has selected the device; the host check alone
    pack = fvlbm._Pack(mg.Case(m, nu=1e-3, dt=1e-3), fvlbm.FVLBM_FP64, scheme=3)
    assert fvlbm.fvlbm_check_mesh(pack.mesh, pack.bc, pack.params)[0] == fvlbm.FVLBM_ERR_BAD_PARAM


def test_create_error_names_the_instance_and_reason():
    """A refused create raises FvlbmError with the code, the failing instance and the reason that
    the host validation gives (no device work happens before the refusal)."""
    m = mg.cavity_quad(4).mesh
    cw = m.cell_nodes.copy().reshape(-1, 4)
    cw[5] = cw[5][::-1]
    bad = mg.Case(mg.Mesh(m.xy, m.cell_ptr, cw.ravel(), m.bedge_nodes, m.bedge_type, m.bedge_val),
                  nu=1e-3, dt=1e-3)
    with pytest.raises(fvlbm.FvlbmError) as e:
        fvlbm.Solver(bad, precision=fvlbm.FVLBM_FP64, device=0)
    assert e.value.code == fvlbm.FVLBM_ERR_BAD_MESH
    assert "instance 0" in str(e.value) and "non-positive area" in str(e.value)
    good = mg.Case(m, nu=1e-3, dt=1e-3)
    with pytest.raises(fvlbm.FvlbmError) as e:
        fvlbm.Solver([good, bad], precision=fvlbm.FVLBM_FP64, device=0)
    assert e.value.code == fvlbm.FVLBM_ERR_BAD_MESH and "instance 1" in str(e.value)


@pytest.fixture(scope="module")
def dumper(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("prepdump") / "prepared_geometry_dump")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fopenmp", "-I", os.path.join(ROOT, "include"),
                           "-I", CSRC, os.path.join(HERE, "native", "prepared_geometry_dump.cpp"),
                           os.path.join(CSRC, "fvlbm_host.cpp"), "-o", out])
    return out


@pytest.mark.parametrize("name", ["cavity_delaunay", "bfs_hybrid", "naca0012_sst", "periodic_box_tri"])
def test_host_geometry_matches_the_oracle(dumper, tmp_path, name):
    """What the library's host preprocessing hands the kernels, against the oracle's own,
    independent geometry (both FP64, no GPU):
      - cell areas;
      - wall distances;
      - the CFL time step;
      - the least-squares gradient of a random field with random boundary values, formed from
        the library's stored weights as the kernels form it."""
    from oracle.oracle import Oracle
    case = dataclasses.replace(_cases()[name], dt=0.0, cfl=0.5)
    m = case.mesh.normalized()
    rng = np.random.default_rng(8)
    phi = rng.standard_normal(m.n_cells)
    phib = rng.standard_normal(m.n_bedges)
    path = str(tmp_path / "mesh.bin")
    _run_write(path, m, phi, phib)
    out = str(tmp_path / "dump.bin")
    subprocess.run([dumper, path, out], check=True)
    d = np.fromfile(out, dtype="<f8")
    dt, cells = d[0], d[1:].reshape(m.n_cells, 5)
    o = Oracle(dataclasses.replace(case, mesh=m))
    geo = o.geometry()
    np.testing.assert_allclose(cells[:, 0], geo["area"], rtol=1e-13, atol=0)
    walls = geo["wdist"] < 1e29
    np.testing.assert_allclose(cells[walls, 1], geo["wdist"][walls], rtol=1e-13, atol=0)
    assert np.all(cells[~walls, 1] >= 1e29)
    assert abs(dt - o.dt) <= 1e-14 * o.dt
    g = o.gradient(phi, phib)
    scale = np.abs(g).max()
    assert np.abs(cells[:, 2:4] - g).max() <= 1e-12 * scale, np.abs(cells[:, 2:4] - g).max() / scale


def _run_write(path, m, phi=None, phib=None):
    with open(path, "wb") as fh:
        fh.write(struct.pack("<i", m.n_nodes)); fh.write(m.xy.astype("<f8").tobytes())
        fh.write(struct.pack("<i", m.n_cells)); fh.write(m.cell_ptr.astype("<i4").tobytes())
        fh.write(m.cell_nodes.astype("<i4").tobytes())
        fh.write(struct.pack("<i", m.n_bedges)); fh.write(m.bedge_nodes.astype("<i4").tobytes())
        fh.write(m.bedge_type.astype("<i4").tobytes()); fh.write(m.bedge_val.astype("<f8").tobytes())
        fh.write(struct.pack("<i", m.periodic_pairs.shape[0]))
        fh.write(m.periodic_pairs.astype("<i4").tobytes()); fh.write(m.periodic_shift.astype("<f8").tobytes())
        if phi is not None:
            fh.write(np.asarray(phi, "<f8").tobytes()); fh.write(np.asarray(phib, "<f8").tobytes())


@pytest.mark.parametrize("name", ["bfs_hybrid", "naca0012_laminar"])
def test_host_local_time_steps_match_the_oracle(dumper, tmp_path, name):
    """Local time stepping: every cell's dt_i = cfl / max_alpha sum_m max(e_alpha . n_m, 0)
    dl_m / A_i from the library's preprocessing equals the oracle's, and the global dt is the
    smallest of them."""
    from oracle.oracle import Oracle
    case = dataclasses.replace(_cases()[name], dt=0.0, cfl=0.5, local_dt=True)
    m = case.mesh.normalized()
    path = str(tmp_path / "mesh.bin")
    _run_write(path, m, np.zeros(m.n_cells), np.zeros(m.n_bedges))
    out = str(tmp_path / "dump.bin")
    subprocess.run([dumper, path, out, "local"], check=True)
    d = np.fromfile(out, dtype="<f8")
    dt, dti = d[0], d[1:].reshape(m.n_cells, 5)[:, 4]
    want = Oracle(dataclasses.replace(case, mesh=m)).dt_cells()
    np.testing.assert_allclose(dti, want, rtol=1e-14, atol=0)
    assert dt == dti.min() and dti.max() > 10 * dti.min()


def test_periodic_mesh_read_with_six_digits_is_accepted():
    """A periodic mesh whose node coordinates were written with 6 decimals (as a mesh file
    might hold them) still glues: the edges agree to about 1e-5 of their length, within the
    1e-4 tolerance.  A shift that is wrong by a tenth of an edge is still refused."""
    m = mg.periodic_box(16, kind="tri", jitter=0.2, seed=9)
    rounded = dataclasses.replace(m, xy=np.round(m.xy, 6))
    assert fvlbm.check_case(mg.Case(rounded, nu=1e-3, cfl=0.5))[0] == 0
    bad = m.periodic_shift.copy()
    bad[:, 0] += 0.1 / 16
    rc, _, why = fvlbm.check_case(mg.Case(dataclasses.replace(rounded, periodic_shift=bad), nu=1e-3, cfl=0.5))
    assert rc == fvlbm.FVLBM_ERR_BAD_BC, (rc, why)
