"""CPU checks of the host side of the derivative paths: the dual-number geometry of the tangent
and the reverse-mode geometry of the adjoint.

The tangent (FVLBM_FP64_TANGENT) differentiates the mesh preprocessing with respect to node
positions by running it with dual numbers.  A small native program (tests/native) built here
with g++ from the library's own host sources compares those derivatives with central
differences of the double-precision preprocessing, for an interior node of a jittered cavity
and for a wall node of an airfoil C-mesh (where the wall distance and the boundary normals
move too).  A second one checks the adjoint's reverse-mode geometry (geometry_adjoint) against
that forward mode by the dot-product identity <A, J v> = <J^T A, v> for random A and v, and a
third the adjoint's binomial checkpoint schedule (revolve_schedule)."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

from paper_1812_00394_gb300 import meshgen as mg

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1812_00394_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("dualcheck") / "dual_geometry_check")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fopenmp", "-I", os.path.join(ROOT, "include"),
                           "-I", CSRC, os.path.join(HERE, "native", "dual_geometry_check.cpp"),
                           os.path.join(CSRC, "fvlbm_host.cpp"), "-o", out])
    return out


def _run(checker, tmp_path, m, node, d, h):
    path = str(tmp_path / "mesh.bin")
    with open(path, "wb") as fh:
        fh.write(struct.pack("<i", m.n_nodes)); fh.write(m.xy.astype("<f8").tobytes())
        fh.write(struct.pack("<i", m.n_cells)); fh.write(m.cell_ptr.astype("<i4").tobytes())
        fh.write(m.cell_nodes.astype("<i4").tobytes())
        fh.write(struct.pack("<i", m.n_bedges)); fh.write(m.bedge_nodes.astype("<i4").tobytes())
        fh.write(m.bedge_type.astype("<i4").tobytes()); fh.write(m.bedge_val.astype("<f8").tobytes())
        fh.write(struct.pack("<iddd", node, d[0], d[1], h))
    res = subprocess.run([checker, path], capture_output=True, text=True, check=True).stdout
    return {ln.split()[0]: (float(ln.split()[1]), float(ln.split()[2])) for ln in res.splitlines()}


def test_dual_geometry_interior_node(checker, tmp_path):
    m = mg.cavity_quad(16, re=400.0, jitter=0.2, seed=7).mesh.normalized()
    node = int(np.argmin(np.linalg.norm(m.xy - 0.5, axis=1)))
    out = _run(checker, tmp_path, m, node, (0.6, 0.8), 1e-6)
    for name in ("sn", "lsq", "rown", "rnbr", "dinv", "area", "wdist"):
        fd, err = out[name]
        assert fd > 0 and err <= 1e-6 * fd, (name, fd, err)
    assert out["bnrm"][0] == 0 and out["blen"][0] == 0   # the node is not on the boundary


def test_dual_geometry_wall_node(checker, tmp_path):
    m = mg.naca0012_cmesh(n_target=2500, re_c=1e4, alpha_deg=4.0).mesh.normalized()
    wall = np.unique(m.bedge_nodes[m.bedge_type == mg.BC_WALL])
    node = int(wall[np.argmin(np.abs(m.xy[wall, 0] - 0.4) + 10 * (m.xy[wall, 1] < 0))])
    out = _run(checker, tmp_path, m, node, (0.0, 1.0), 1e-7)
    for name in ("sn", "lsq", "rown", "rnbr", "dinv", "area", "wdist", "bnrm", "blen"):
        fd, err = out[name]
        assert fd > 0 and err <= 1e-5 * fd, (name, fd, err)


def test_dual_number_operations(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "dual_ops_check")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-I", CSRC,
                           os.path.join(HERE, "native", "dual_ops_check.cpp"), "-o", exe])
    res = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    out = {ln.split()[0]: float(ln.split()[1]) for ln in res.splitlines()}
    for name in ("mul_add", "div", "sqrt", "tanh", "fmin_fmax", "neg_sub"):
        assert out[name] < 1e-8, (name, out[name])
    assert out["sqrt0"] == 0.0


@pytest.fixture(scope="module")
def adjoint_checker(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("geoadj") / "geometry_adjoint_check")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fopenmp", "-I", os.path.join(ROOT, "include"),
                           "-I", CSRC, os.path.join(HERE, "native", "geometry_adjoint_check.cpp"),
                           os.path.join(CSRC, "fvlbm_host.cpp"), "-o", out])
    return out


@pytest.mark.parametrize("which", ["cavity_jitter", "naca", "bfs"])
def test_geometry_adjoint_dot_product(adjoint_checker, tmp_path, which):
    if which == "cavity_jitter":
        m = mg.cavity_quad(12, re=400.0, jitter=0.2, seed=7).mesh.normalized()
    elif which == "naca":
        m = mg.naca0012_cmesh(n_target=1500, re_c=1e4, alpha_deg=4.0).mesh.normalized()
    else:
        m = mg.bfs_hybrid(n_target=1500).mesh.normalized()
    path = str(tmp_path / "mesh.bin")
    with open(path, "wb") as fh:
        fh.write(struct.pack("<i", m.n_nodes)); fh.write(m.xy.astype("<f8").tobytes())
        fh.write(struct.pack("<i", m.n_cells)); fh.write(m.cell_ptr.astype("<i4").tobytes())
        fh.write(m.cell_nodes.astype("<i4").tobytes())
        fh.write(struct.pack("<i", m.n_bedges)); fh.write(m.bedge_nodes.astype("<i4").tobytes())
        fh.write(m.bedge_type.astype("<i4").tobytes()); fh.write(m.bedge_val.astype("<f8").tobytes())
        fh.write(struct.pack("<Q", 12345))
    res = subprocess.run([adjoint_checker, path], capture_output=True, text=True, check=True).stdout
    out = {ln.split()[0]: float(ln.split()[1]) for ln in res.splitlines()}
    assert abs(out["forward"]) > 0
    assert abs(out["forward"] - out["reverse"]) <= 1e-10 * abs(out["forward"]), out


def test_revolve_schedule(tmp_path):
    """The adjoint's binomial checkpoint schedule (host code): every unit reversed once, last to
    first, from a snapshot holding its start; snapshot indices within the count; forward work
    within (r + 1) units; refused without snapshots for two units or more.  Pass counts of a few
    cases pin the schedule (17 units with a snapshot each: 2 x 17 - 1)."""
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "revolve_check")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fopenmp", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                           os.path.join(HERE, "native", "revolve_check.cpp"),
                           os.path.join(CSRC, "fvlbm_host.cpp"), "-o", exe])
    res = subprocess.run([exe], capture_output=True, text=True)
    assert res.returncode == 0, res.stdout
    passes = {(int(a), int(b)): int(c) for _, a, b, c in
              (ln.split() for ln in res.stdout.splitlines() if ln.startswith("passes"))}
    assert passes[(17, 16)] == 33
    assert passes[(100, 3)] == 595
    assert passes[(1000, 5)] == 7368
