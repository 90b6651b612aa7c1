"""Python binding of the C ABI in include/fvlbm.h (argument marshalling only).

Every entry point of the library is exposed under its C name (``fvlbm_create``,
``fvlbm_step``, ...); ``Solver`` is a small convenience wrapper around them.  All arithmetic
of the time step runs in the CUDA library; this module only converts numpy arrays to
pointers.  It raises if the compiled library is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

FVLBM_OK = 0
FVLBM_ERR_BAD_MESH = -1
FVLBM_ERR_BAD_BC = -2
FVLBM_ERR_BAD_PARAM = -3
FVLBM_ERR_OOM = -4
FVLBM_ERR_CUDA = -5
FVLBM_ERR_DIVERGED = -6
FVLBM_ERR_NOT_SUPPORTED = -7
FVLBM_ERR_TIMEOUT = -8
FVLBM_FP64 = 0
FVLBM_FP32_DEV = 1
FVLBM_FP64_TANGENT = 2
SCHEME_IMEX = 0
SCHEME_EULER = 1
Q = 9


class FvlbmError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


class fvlbm_mesh(C.Structure):
    _fields_ = [("n_nodes", C.c_int), ("xy", C.c_void_p), ("n_cells", C.c_int),
                ("cell_ptr", C.c_void_p), ("cell_nodes", C.c_void_p)]


class fvlbm_bc(C.Structure):
    _fields_ = [("n_bedges", C.c_int), ("bedge_nodes", C.c_void_p), ("bedge_type", C.c_void_p),
                ("bedge_val", C.c_void_p), ("n_periodic", C.c_int), ("periodic_pairs", C.c_void_p),
                ("periodic_shift", C.c_void_p)]


class fvlbm_params(C.Structure):
    _fields_ = [("nu", C.c_double), ("rho0", C.c_double), ("dt", C.c_double), ("cfl", C.c_double),
                ("sst", C.c_int), ("precision", C.c_int), ("uref", C.c_double),
                ("lref", C.c_double), ("alpha_deg", C.c_double), ("rho_init", C.c_void_p),
                ("u_init", C.c_void_p), ("v_init", C.c_void_p), ("k_init", C.c_void_p),
                ("omega_init", C.c_void_p), ("kernel_path", C.c_int), ("scheme", C.c_int),
                ("local_dt", C.c_int), ("variant", C.c_int)]


class fvlbm_stats(C.Structure):
    _fields_ = [("steps", C.c_longlong), ("residual", C.c_double), ("mass", C.c_double),
                ("diverged", C.c_int)]


EXPORTS = ["fvlbm_create", "fvlbm_create_batch", "fvlbm_step", "fvlbm_forces", "fvlbm_get_f",
           "fvlbm_set_f", "fvlbm_get_fields", "fvlbm_info", "fvlbm_footprint",
           "fvlbm_profile_kernels", "fvlbm_autotune", "fvlbm_destroy", "fvlbm_strerror",
           "fvlbm_stats_reduce_static", "fvlbm_tangent_seed", "fvlbm_tangent_seed_nodes",
           "fvlbm_get_f_tangent", "fvlbm_forces_tangent", "fvlbm_adjoint",
           "fvlbm_set_adjoint_budget", "fvlbm_state_bytes", "fvlbm_save_state",
           "fvlbm_load_state", "fvlbm_set_rollback", "fvlbm_set_f_async",
           "fvlbm_get_fields_async", "fvlbm_wait", "fvlbm_get_fdev_f32", "fvlbm_set_fdev_f32_async",
           "fvlbm_check_mesh", "fvlbm_adjoint_params", "fvlbm_set_wait_limit",
           "fvlbm_get_cells", "fvlbm_set_cells", "fvlbm_set_wall_distance", "fvlbm_cell_geometry",
           "fvlbm_forces_edges", "fvlbm_set_exchange_list", "fvlbm_pack_cells_dev",
           "fvlbm_unpack_cells_dev", "fvlbm_fp64_peak", "fvlbm_fv_items"]

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load libfvlbm.so (building it in-tree first if allowed and missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise FileNotFoundError(f"libfvlbm.so not built at {path}")
        _build.build()
    lib = C.CDLL(path)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    P = C.POINTER
    lib.fvlbm_create.argtypes = [P(fvlbm_mesh), P(fvlbm_bc), P(fvlbm_params), i, vp, P(vp)]
    lib.fvlbm_create_batch.argtypes = [i, P(fvlbm_mesh), P(fvlbm_bc), P(fvlbm_params), i, vp, P(vp)]
    lib.fvlbm_step.argtypes = [vp, i, P(fvlbm_stats)]
    lib.fvlbm_forces.argtypes = [vp, i, vp, vp]
    lib.fvlbm_get_f.argtypes = [vp, i, vp]
    lib.fvlbm_set_f.argtypes = [vp, i, vp]
    lib.fvlbm_get_fields.argtypes = [vp, i, vp, vp, vp, vp, vp, vp]
    lib.fvlbm_info.argtypes = [vp, i, P(i), P(i), P(d)]
    lib.fvlbm_footprint.argtypes = [vp, P(C.c_longlong), P(i)]
    lib.fvlbm_profile_kernels.argtypes = [vp, i, i, vp, vp, vp]
    lib.fvlbm_autotune.argtypes = [vp, i, P(i), vp]
    lib.fvlbm_set_f_async.argtypes = [vp, i, vp]
    lib.fvlbm_get_fields_async.argtypes = [vp, i, vp, vp, vp, vp, vp, vp]
    lib.fvlbm_wait.argtypes = [vp]
    lib.fvlbm_get_fdev_f32.argtypes = [vp, i, vp]
    lib.fvlbm_set_fdev_f32_async.argtypes = [vp, i, vp]
    lib.fvlbm_state_bytes.argtypes = [vp, P(C.c_longlong)]
    lib.fvlbm_save_state.argtypes = [vp, vp, C.c_longlong]
    lib.fvlbm_load_state.argtypes = [vp, vp, C.c_longlong]
    lib.fvlbm_set_rollback.argtypes = [vp, i]
    lib.fvlbm_tangent_seed.argtypes = [vp, i, vp, vp]
    lib.fvlbm_get_f_tangent.argtypes = [vp, i, vp]
    lib.fvlbm_tangent_seed_nodes.argtypes = [vp, i, vp]
    lib.fvlbm_forces_tangent.argtypes = [vp, i, d, vp, vp]
    lib.fvlbm_adjoint.argtypes = [vp, i, i, vp, vp, vp, vp, vp]
    lib.fvlbm_set_adjoint_budget.argtypes = [vp, C.c_longlong]
    lib.fvlbm_adjoint_params.argtypes = [vp, i, i, vp, i, vp, vp, vp, vp, vp, vp, vp]
    lib.fvlbm_set_wait_limit.argtypes = [vp, C.c_longlong]
    lib.fvlbm_fv_items.argtypes = [vp, vp, vp, vp]
    lib.fvlbm_destroy.argtypes = [vp]
    lib.fvlbm_destroy.restype = None
    lib.fvlbm_strerror.argtypes = [i]
    lib.fvlbm_strerror.restype = C.c_char_p
    lib.fvlbm_stats_reduce_static.argtypes = [vp] * 6 + [i, vp, vp]
    lib.fvlbm_check_mesh.argtypes = [P(fvlbm_mesh), P(fvlbm_bc), P(fvlbm_params), P(d), C.c_char_p, i]
    lib.fvlbm_get_cells.argtypes = [vp, i, i, vp, vp, vp, vp, vp]
    lib.fvlbm_set_cells.argtypes = [vp, i, i, vp, vp, vp, vp, vp]
    lib.fvlbm_set_wall_distance.argtypes = [vp, i, vp]
    lib.fvlbm_cell_geometry.argtypes = [P(fvlbm_mesh), P(fvlbm_bc), P(fvlbm_params), vp, vp]
    lib.fvlbm_forces_edges.argtypes = [vp, i, vp]
    lib.fvlbm_set_exchange_list.argtypes = [vp, i, i, vp, P(i)]
    lib.fvlbm_pack_cells_dev.argtypes = [vp, i, vp]
    lib.fvlbm_unpack_cells_dev.argtypes = [vp, i, vp]
    lib.fvlbm_fp64_peak.argtypes = [i, P(d)]
    for name in EXPORTS:
        if name not in ("fvlbm_destroy", "fvlbm_strerror"):
            getattr(lib, name).restype = i
    _lib = lib
    return lib


def strerror(code: int) -> str:
    try:
        return load().fvlbm_strerror(int(code)).decode()
    except Exception:  # noqa: BLE001 -- message only
        return "unknown"


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise FvlbmError(rc, what)
    return rc


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------------ C-named wrappers
def _create_failed(rc: int, what: str, triples) -> None:
    """Raise FvlbmError for a failed create; for an input error the message names the first
    instance that fvlbm_check_mesh refuses and its reason."""
    if rc in (FVLBM_ERR_BAD_MESH, FVLBM_ERR_BAD_BC, FVLBM_ERR_BAD_PARAM):
        for i, (m, b, p) in enumerate(triples):
            rc_i, _, why = fvlbm_check_mesh(m, b, p)
            if rc_i < 0:
                what = f"{what}: instance {i}: {why}"
                break
    raise FvlbmError(rc, what)


def fvlbm_create(mesh: fvlbm_mesh, bc: fvlbm_bc, params: fvlbm_params, device: int = -1,
                 stream: int | None = None) -> C.c_void_p:
    h = C.c_void_p()
    rc = load().fvlbm_create(C.byref(mesh), C.byref(bc), C.byref(params), device,
                             C.c_void_p(stream) if stream else None, C.byref(h))
    if rc < 0:
        _create_failed(rc, "fvlbm_create", [(mesh, bc, params)])
    return h


def fvlbm_check_mesh(mesh: fvlbm_mesh, bc: fvlbm_bc, params: fvlbm_params) -> tuple[int, float, str]:
    """(return code, time step, message) of the host-only validation; no GPU is touched."""
    dt = C.c_double(0.0)
    why = C.create_string_buffer(512)
    rc = load().fvlbm_check_mesh(C.byref(mesh), C.byref(bc), C.byref(params), C.byref(dt), why, 512)
    return rc, dt.value, why.value.decode()


def fvlbm_create_batch(meshes, bcs, params, device: int = -1, stream: int | None = None):
    n = len(meshes)
    M = (fvlbm_mesh * n)(*meshes)
    B = (fvlbm_bc * n)(*bcs)
    Pm = (fvlbm_params * n)(*params)
    h = C.c_void_p()
    rc = load().fvlbm_create_batch(n, M, B, Pm, device, C.c_void_p(stream) if stream else None,
                                   C.byref(h))
    if rc < 0:
        _create_failed(rc, "fvlbm_create_batch", list(zip(meshes, bcs, params)))
    return h


def fvlbm_step(h, n_steps: int, stats: bool = False):
    st = fvlbm_stats() if stats else None
    rc = load().fvlbm_step(h, int(n_steps), C.byref(st) if st is not None else None)
    if rc == FVLBM_ERR_DIVERGED and st is not None:
        return {"steps": st.steps, "residual": st.residual, "mass": st.mass, "diverged": 1}
    _check(rc, "fvlbm_step")
    if st is None:
        return None
    return {"steps": st.steps, "residual": st.residual, "mass": st.mass, "diverged": st.diverged}


def fvlbm_info(h, instance: int = 0):
    n, b, dt = C.c_int(), C.c_int(), C.c_double()
    _check(load().fvlbm_info(h, instance, C.byref(n), C.byref(b), C.byref(dt)), "fvlbm_info")
    return n.value, b.value, dt.value


def fvlbm_get_f(h, instance: int, out: np.ndarray | None = None) -> np.ndarray:
    n, _, _ = fvlbm_info(h, instance)
    f = np.empty((n, Q)) if out is None else out
    _check(load().fvlbm_get_f(h, instance, _p(f)), "fvlbm_get_f")
    return f


def fvlbm_set_f(h, instance: int, f: np.ndarray) -> None:
    f = np.ascontiguousarray(f, np.float64)
    _check(load().fvlbm_set_f(h, instance, _p(f)), "fvlbm_set_f")


def fvlbm_get_fields(h, instance: int = 0) -> dict:
    n, _, _ = fvlbm_info(h, instance)
    out = {key: np.empty(n) for key in ("rho", "u", "v", "k", "omega", "nut")}
    _check(load().fvlbm_get_fields(h, instance, *(_p(out[k]) for k in
                                                  ("rho", "u", "v", "k", "omega", "nut"))),
           "fvlbm_get_fields")
    return out


def fvlbm_forces(h, instance: int = 0, with_cp: bool = False) -> dict:
    _, nb, _ = fvlbm_info(h, instance)
    out = np.zeros(4)
    cp = np.zeros(nb) if with_cp else None
    _check(load().fvlbm_forces(h, instance, _p(out), _p(cp)), "fvlbm_forces")
    res = {"fx": out[0], "fy": out[1], "cd": out[2], "cl": out[3]}
    if with_cp:
        res["cp"] = cp
    return res


def fvlbm_get_cells(h, instance: int, cells) -> tuple:
    """(f [n, 9], k, omega, nu_t) of the listed cells (input ids of the instance)."""
    cells = np.ascontiguousarray(cells, np.int32)
    n = cells.shape[0]
    f, k, w, nt = np.empty((n, Q)), np.empty(n), np.empty(n), np.empty(n)
    _check(load().fvlbm_get_cells(h, instance, n, _p(cells), _p(f), _p(k), _p(w), _p(nt)),
           "fvlbm_get_cells")
    return f, k, w, nt


def fvlbm_set_cells(h, instance: int, cells, f=None, k=None, omega=None, nut=None) -> None:
    cells = np.ascontiguousarray(cells, np.int32)
    arr = [None if a is None else np.ascontiguousarray(a, np.float64) for a in (f, k, omega, nut)]
    _check(load().fvlbm_set_cells(h, instance, cells.shape[0], _p(cells), *(_p(a) for a in arr)),
           "fvlbm_set_cells")


def fvlbm_set_wall_distance(h, instance: int, d) -> None:
    d = np.ascontiguousarray(d, np.float64)
    _check(load().fvlbm_set_wall_distance(h, instance, _p(d)), "fvlbm_set_wall_distance")


def fvlbm_forces_edges(h, instance: int = 0) -> np.ndarray:
    """[n_bedges, 2] wall force (Fx, Fy) per boundary edge (0 off the walls)."""
    _, nb, _ = fvlbm_info(h, instance)
    out = np.zeros((nb, 2))
    _check(load().fvlbm_forces_edges(h, instance, _p(out)), "fvlbm_forces_edges")
    return out


def fvlbm_set_exchange_list(h, instance: int, cells) -> int:
    """Register a cell list for the device-buffer ghost exchange; returns its id."""
    cells = np.ascontiguousarray(cells, np.int32)
    lid = C.c_int()
    _check(load().fvlbm_set_exchange_list(h, instance, cells.shape[0], _p(cells), C.byref(lid)),
           "fvlbm_set_exchange_list")
    return lid.value


def fvlbm_pack_cells_dev(h, list_id: int, vals_ptr: int) -> None:
    """Enqueue the packing of a list into a DEVICE buffer of n * 12 doubles (address)."""
    _check(load().fvlbm_pack_cells_dev(h, list_id, C.c_void_p(vals_ptr)), "fvlbm_pack_cells_dev")


def fvlbm_unpack_cells_dev(h, list_id: int, vals_ptr: int) -> None:
    _check(load().fvlbm_unpack_cells_dev(h, list_id, C.c_void_p(vals_ptr)), "fvlbm_unpack_cells_dev")


def fvlbm_fp64_peak(device: int = -1) -> float:
    """Measured FP64 FMA throughput of the device in TFLOP/s."""
    t = C.c_double()
    _check(load().fvlbm_fp64_peak(device, C.byref(t)), "fvlbm_fp64_peak")
    return t.value


def fvlbm_footprint(h):
    b, lps = C.c_longlong(), C.c_int()
    _check(load().fvlbm_footprint(h, C.byref(b), C.byref(lps)), "fvlbm_footprint")
    return b.value, lps.value


def fvlbm_profile_kernels(h, n_steps: int) -> dict:
    maxk = 16
    names = C.create_string_buffer(32 * maxk)
    ms = np.zeros(maxk)
    launches = np.zeros(maxk, np.int32)
    nk = _check(load().fvlbm_profile_kernels(h, int(n_steps), maxk, names, _p(ms), _p(launches)),
                "fvlbm_profile_kernels")
    raw = names.raw
    res = {}
    for k in range(nk):
        nm = raw[32 * k:32 * (k + 1)].split(b"\0", 1)[0].decode()
        res[nm] = {"ms": float(ms[k]), "launches": int(launches[k])}
    return res


def fvlbm_stats_reduce_static(u_old: int, v_old: int, u_new: int, v_new: int, rho: int,
                              area: int, n: int, out: int, stream: int | None = None) -> None:
    """Allocation-free FP64 statistics over caller-owned DEVICE arrays (raw pointers); writes 4
    doubles to the device pointer ``out``.  For callers that cannot allocate device memory."""
    _check(load().fvlbm_stats_reduce_static(u_old, v_old, u_new, v_new, rho, area, int(n), out,
                                            stream), "fvlbm_stats_reduce_static")


def fvlbm_autotune(h, trial_steps: int = 5):
    """Time the available kernel configurations on a snapshot and keep the fastest.
    Returns (chosen, {name: ms_per_step})."""
    chosen = C.c_int()
    ms = np.zeros(4)
    _check(load().fvlbm_autotune(h, int(trial_steps), C.byref(chosen), _p(ms)), "fvlbm_autotune")
    names = ("fused256", "fused128", "twopass", "facevalue")
    return names[chosen.value], {names[k]: float(ms[k]) for k in range(4) if ms[k] >= 0}


def fvlbm_tangent_seed(h, instance: int, dbedge_val: np.ndarray | None = None,
                       df: np.ndarray | None = None) -> None:
    """Seed d/dp of the boundary values ([n_bedges, 5], input edge order) and/or of f
    ([n_cells, 9]) on a FVLBM_FP64_TANGENT handle."""
    bv = None if dbedge_val is None else np.ascontiguousarray(dbedge_val, np.float64)
    f = None if df is None else np.ascontiguousarray(df, np.float64)
    _check(load().fvlbm_tangent_seed(h, instance, _p(bv), _p(f)), "fvlbm_tangent_seed")


def fvlbm_tangent_seed_nodes(h, instance: int, dxy: np.ndarray) -> None:
    """Seed d(x, y)/dp of every mesh node ([n_nodes, 2]) on a FVLBM_FP64_TANGENT handle."""
    d = np.ascontiguousarray(dxy, np.float64)
    _check(load().fvlbm_tangent_seed_nodes(h, instance, _p(d)), "fvlbm_tangent_seed_nodes")


def fvlbm_get_f_tangent(h, instance: int = 0) -> np.ndarray:
    n, _, _ = fvlbm_info(h, instance)
    df = np.empty((n, Q))
    _check(load().fvlbm_get_f_tangent(h, instance, _p(df)), "fvlbm_get_f_tangent")
    return df


def fvlbm_forces_tangent(h, instance: int = 0, dalpha: float = 0.0) -> tuple[dict, dict]:
    """(forces, d forces / dp); dalpha = d(alpha in radians)/dp."""
    out, dout = np.zeros(4), np.zeros(4)
    _check(load().fvlbm_forces_tangent(h, instance, float(dalpha), _p(out), _p(dout)),
           "fvlbm_forces_tangent")
    keys = ("fx", "fy", "cd", "cl")
    return dict(zip(keys, out)), dict(zip(keys, dout))


def fvlbm_adjoint(h, instance: int, n_steps: int, w_cd: float = 0.0, w_cl: float = 0.0,
                  n_nodes: int | None = None):
    """Reverse-mode gradient of J = w_cd C_D + w_cl C_L after n_steps FP64 steps from the
    current state: (J, dJ/df [n_cells, 9], dJ/dbedge_val [n_bedges, 5], dJ/dxy [n_nodes, 2] or
    None).  dJ/dxy is computed when n_nodes (the instance's node count) is given.  The handle's
    state is unchanged."""
    n, nb, _ = fvlbm_info(h, instance)
    w = np.array([w_cd, w_cl], np.float64)
    J = C.c_double()
    df = np.empty((n, Q))
    db = np.empty((nb, 5))
    dxy = None if n_nodes is None else np.empty((int(n_nodes), 2))
    _check(load().fvlbm_adjoint(h, instance, int(n_steps), _p(w), C.byref(J), _p(df), _p(db),
                                _p(dxy)), "fvlbm_adjoint")
    return J.value, df, db, dxy


def fvlbm_adjoint_params(h, instance: int, n_steps: int, w_cd: float, w_cl: float,
                         wall_nodes=None, wall_normals=None) -> dict:
    """Gradient of J = w_cd C_D + w_cl C_L after n_steps FP64 steps with respect to the
    free-stream angle (radians), the inflow eddy-viscosity ratio and the displacement of each
    node ``wall_nodes[j]`` along ``wall_normals[j]`` (see fvlbm_adjoint_params in the header).
    Returns {"J", "cd", "cl", "dalpha", "dratio", "dwall"}."""
    nodes = np.zeros(0, np.int32) if wall_nodes is None else np.ascontiguousarray(wall_nodes, np.int32)
    nw = int(nodes.shape[0])
    normals = (np.zeros((0, 2)) if wall_normals is None
               else np.ascontiguousarray(wall_normals, np.float64).reshape(nw, 2))
    w = np.array([w_cd, w_cl], np.float64)
    J, da, dr = C.c_double(), C.c_double(), C.c_double()
    cdcl = np.zeros(2)
    dwall = np.zeros(nw)
    _check(load().fvlbm_adjoint_params(h, instance, int(n_steps), _p(w), nw,
                                       _p(nodes) if nw else None, _p(normals) if nw else None,
                                       C.byref(J), _p(cdcl), C.byref(da), C.byref(dr),
                                       _p(dwall) if nw else None), "fvlbm_adjoint_params")
    return {"J": J.value, "cd": float(cdcl[0]), "cl": float(cdcl[1]), "dalpha": da.value,
            "dratio": dr.value, "dwall": dwall}


def fvlbm_save_state(h) -> bytes:
    """The handle's state as an opaque blob (checkpoint)."""
    n = C.c_longlong()
    _check(load().fvlbm_state_bytes(h, C.byref(n)), "fvlbm_state_bytes")
    buf = C.create_string_buffer(n.value)
    _check(load().fvlbm_save_state(h, buf, n.value), "fvlbm_save_state")
    return buf.raw


def fvlbm_load_state(h, blob: bytes) -> None:
    """Restore a blob written by fvlbm_save_state (same meshes and parameters)."""
    buf = C.create_string_buffer(blob, len(blob))
    _check(load().fvlbm_load_state(h, buf, len(blob)), "fvlbm_load_state")


def fvlbm_set_wait_limit(h, polls: int) -> None:
    """Diagnostic: polls of the fused kernels' first staging wait (see the header)."""
    _check(load().fvlbm_set_wait_limit(h, int(polls)), "fvlbm_set_wait_limit")


def fvlbm_fv_items(h) -> tuple:
    """Diagnostic: (items, blocks split, items using the halo overflow) of the face-value stages."""
    v = (C.c_int * 3)()
    _check(load().fvlbm_fv_items(h, C.byref(v, 0), C.byref(v, 4), C.byref(v, 8)), "fvlbm_fv_items")
    return tuple(int(x) for x in v)


def fvlbm_set_rollback(h, every: int) -> None:
    _check(load().fvlbm_set_rollback(h, int(every)), "fvlbm_set_rollback")


def forces_gradient(case, directions, steps: int, device: int = -1):
    """Derivatives of the wall force of ``case`` after ``steps`` steps along several parameter
    directions at once: one FVLBM_FP64_TANGENT batch with one instance per direction, so that
    every kernel launch of a step advances all directions.  Each direction is a dict with any
    of ``dbedge_val`` ([n_bedges, 5]), ``dxy`` ([n_nodes, 2]), ``df`` ([n_cells, 9]) and
    ``dalpha`` (d alpha / dp in radians).  Returns (forces, [d forces / dp_k])."""
    k = len(directions)
    if k == 0:
        raise ValueError("forces_gradient needs at least one direction")
    s = Solver([case] * k, precision=FVLBM_FP64_TANGENT, device=device)
    for i, d in enumerate(directions):
        if d.get("dxy") is not None:
            s.tangent_seed_nodes(d["dxy"], i=i)
        if d.get("dbedge_val") is not None or d.get("df") is not None:
            s.tangent_seed(d.get("dbedge_val"), d.get("df"), i=i)
    s.step(steps)
    grads = []
    val = None
    for i, d in enumerate(directions):
        v, g = s.forces_tangent(i, float(d.get("dalpha", 0.0)))
        val = v if val is None else val
        grads.append(g)
    s.close()
    return val, grads


def fvlbm_destroy(h) -> None:
    if h:
        load().fvlbm_destroy(h)


def fvlbm_strerror(code: int) -> str:
    return strerror(code)


# ------------------------------------------------------------------ convenience wrapper
class _Pack:
    """Keeps the numpy arrays alive that a (mesh, bc, params) triple points into."""

    def __init__(self, case, precision: int, kernel_path: int = 0, scheme: int = 0):
        m = case.mesh.normalized()
        rho, u, v, k, w = case.init_arrays()
        self.keep = (m, rho, u, v, k, w)
        self.mesh = fvlbm_mesh(m.n_nodes, _p(m.xy), m.n_cells, _p(m.cell_ptr), _p(m.cell_nodes))
        self.bc = fvlbm_bc(m.n_bedges, _p(m.bedge_nodes), _p(m.bedge_type), _p(m.bedge_val),
                           m.periodic_pairs.shape[0], _p(m.periodic_pairs), _p(m.periodic_shift))
        self.params = fvlbm_params(case.nu, case.rho0, case.dt, case.cfl, int(bool(case.sst)),
                                   precision, case.uref, case.lref, case.alpha_deg, _p(rho), _p(u),
                                   _p(v), _p(k), _p(w), kernel_path, scheme,
                                   int(bool(getattr(case, "local_dt", False))),
                                   int(getattr(case, "variant", 0)))


def check_case(case, precision: int = FVLBM_FP64, kernel_path: int = 0,
               scheme: int = 0) -> tuple[int, float, str]:
    """``fvlbm_check_mesh`` on a ``meshgen.Case``: (return code, time step, message)."""
    pk = _Pack(case, precision, kernel_path, scheme)
    return fvlbm_check_mesh(pk.mesh, pk.bc, pk.params)


def case_geometry(case) -> tuple[np.ndarray, np.ndarray]:
    """(area, wall distance) per cell of ``case`` as create computes them (host only)."""
    pk = _Pack(case, FVLBM_FP64)
    n = case.mesh.n_cells
    area, wd = np.empty(n), np.empty(n)
    _check(load().fvlbm_cell_geometry(C.byref(pk.mesh), C.byref(pk.bc), C.byref(pk.params), _p(area),
                                      _p(wd)), "fvlbm_cell_geometry")
    return area, wd


class Solver:
    """One handle over one case or a batch of cases (``meshgen.Case``)."""

    def __init__(self, cases, precision: int = FVLBM_FP64, device: int = -1,
                 stream: int | None = None, kernel_path: int = 0, scheme: int = 0):
        if not isinstance(cases, (list, tuple)):
            cases = [cases]
        packs = [_Pack(c, precision, kernel_path, scheme) for c in cases]
        if len(packs) == 1:
            self.h = fvlbm_create(packs[0].mesh, packs[0].bc, packs[0].params, device, stream)
        else:
            self.h = fvlbm_create_batch([p.mesh for p in packs], [p.bc for p in packs],
                                        [p.params for p in packs], device, stream)
        self.n = len(cases)
        self.n_nodes = [int(c.mesh.n_nodes) for c in cases]
        self.cells = [fvlbm_info(self.h, i)[0] for i in range(self.n)]

    def close(self):
        if getattr(self, "h", None):
            fvlbm_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def dt(self, i: int = 0) -> float:
        return fvlbm_info(self.h, i)[2]

    def step(self, n: int = 1, stats: bool = False):
        return fvlbm_step(self.h, n, stats)

    def get_f(self, i: int = 0) -> np.ndarray:
        return fvlbm_get_f(self.h, i)

    def set_f(self, f: np.ndarray, i: int = 0) -> None:
        fvlbm_set_f(self.h, i, f)

    def get_cells(self, cells, i: int = 0):
        return fvlbm_get_cells(self.h, i, cells)

    def set_cells(self, cells, f=None, k=None, omega=None, nut=None, i: int = 0) -> None:
        fvlbm_set_cells(self.h, i, cells, f, k, omega, nut)

    def set_exchange_list(self, cells, i: int = 0) -> int:
        return fvlbm_set_exchange_list(self.h, i, cells)

    def pack_cells_dev(self, list_id: int, vals_ptr: int) -> None:
        fvlbm_pack_cells_dev(self.h, list_id, vals_ptr)

    def unpack_cells_dev(self, list_id: int, vals_ptr: int) -> None:
        fvlbm_unpack_cells_dev(self.h, list_id, vals_ptr)

    def set_wall_distance(self, d, i: int = 0) -> None:
        fvlbm_set_wall_distance(self.h, i, d)

    def forces_edges(self, i: int = 0) -> np.ndarray:
        return fvlbm_forces_edges(self.h, i)

    def fields(self, i: int = 0) -> dict:
        return fvlbm_get_fields(self.h, i)

    def forces(self, i: int = 0, with_cp: bool = False) -> dict:
        return fvlbm_forces(self.h, i, with_cp)

    def footprint(self):
        return fvlbm_footprint(self.h)

    def autotune(self, trial_steps: int = 5):
        return fvlbm_autotune(self.h, trial_steps)

    def profile_kernels(self, n_steps: int) -> dict:
        return fvlbm_profile_kernels(self.h, n_steps)

    def save_state(self) -> bytes:
        return fvlbm_save_state(self.h)

    def load_state(self, blob: bytes) -> None:
        fvlbm_load_state(self.h, blob)

    def set_rollback(self, every: int) -> None:
        fvlbm_set_rollback(self.h, every)

    def tangent_seed(self, dbedge_val=None, df=None, i: int = 0) -> None:
        fvlbm_tangent_seed(self.h, i, dbedge_val, df)

    def tangent_seed_nodes(self, dxy, i: int = 0) -> None:
        fvlbm_tangent_seed_nodes(self.h, i, dxy)

    def get_f_tangent(self, i: int = 0) -> np.ndarray:
        return fvlbm_get_f_tangent(self.h, i)

    def forces_tangent(self, i: int = 0, dalpha: float = 0.0):
        return fvlbm_forces_tangent(self.h, i, dalpha)

    def set_adjoint_budget(self, nbytes: int) -> None:
        _check(load().fvlbm_set_adjoint_budget(self.h, int(nbytes)), "fvlbm_set_adjoint_budget")

    def adjoint(self, n_steps: int, w_cd: float = 0.0, w_cl: float = 0.0, i: int = 0,
                shape: bool = False):
        """(J, dJ/df, dJ/dbedge_val, dJ/dxy or None); see fvlbm_adjoint."""
        nn = self.n_nodes[i] if shape else None
        return fvlbm_adjoint(self.h, i, n_steps, w_cd, w_cl, nn)

    def adjoint_params(self, n_steps: int, w_cd: float = 0.0, w_cl: float = 0.0, i: int = 0,
                       wall_nodes=None, wall_normals=None) -> dict:
        """See fvlbm_adjoint_params."""
        return fvlbm_adjoint_params(self.h, i, n_steps, w_cd, w_cl, wall_nodes, wall_normals)
