"""ctypes wrapper of the FP64 CPU oracle (oracle/fvlbm_oracle.c).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg import this module.  The product path (the CUDA library and its binding)
never imports it, and this module imports nothing from the product package except what a
caller passes in (a ``meshgen.Case``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fvlbm_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")
LIB_CS = os.path.join(BUILD, "liboracle_cs.so")   # complex-step build (the oracle's tangent)
_lock = threading.Lock()
_lib = None
_lib_cs = None

Q = 9
_D = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_I = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False, complex_step: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so that every product is rounded as
    written; OpenMP for its optional multi-threaded per-cell loops); with ``complex_step`` the
    same source in complex arithmetic (the oracle's own tangent by the complex-step method)."""
    os.makedirs(BUILD, exist_ok=True)
    lib = LIB_CS if complex_step else LIB
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(SRC):
        tmp = lib + f".tmp{os.getpid()}"
        # the double build runs its per-cell loops on oracle_set_threads() threads (1 unless
        # asked; results are bitwise the same for any count)
        flags = ["-DORACLE_COMPLEX_STEP"] if complex_step else ["-fopenmp"]
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               *flags, "-o", tmp, SRC, "-lm"])
        os.replace(tmp, lib)
    return lib


def _common(lib):
    vp = C.c_void_p
    opt_d = C.c_void_p  # nullable double*
    lib.oracle_create.restype = vp
    lib.oracle_create.argtypes = [C.c_int, _D, C.c_int, _I, _I, C.c_int, _I, _I, _D, C.c_int,
                                  _I, _D, opt_d, opt_d, opt_d, opt_d, opt_d, _D]
    lib.oracle_destroy.argtypes = [vp]
    lib.oracle_step.argtypes = [vp, C.c_int]
    lib.oracle_step.restype = C.c_int
    for name in ("oracle_dt", "oracle_residual", "oracle_moment_defect", "oracle_mass"):
        getattr(lib, name).argtypes = [vp]
        getattr(lib, name).restype = C.c_double
    lib.oracle_dt_cells.argtypes = [vp, _D]
    lib.oracle_n_cells.argtypes = [vp]
    lib.oracle_n_cells.restype = C.c_int
    lib.oracle_get_f.argtypes = [vp, _D]
    lib.oracle_set_f.argtypes = [vp, _D]
    lib.oracle_get_fields.argtypes = [vp, _D, _D, _D, _D, _D, _D]
    lib.oracle_set_turb.argtypes = [vp, _D, _D, _D]
    lib.oracle_set_wdist.argtypes = [vp, _D]
    lib.oracle_geometry.argtypes = [vp, _D, _D, _D, _D]
    lib.oracle_forces.argtypes = [vp, _D, opt_d, opt_d, opt_d]


def _load_cs():
    global _lib_cs
    with _lock:
        if _lib_cs is not None:
            return _lib_cs
        lib = C.CDLL(build(complex_step=True))
        _common(lib)
        lib.oracle_cs_seed.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double]
        lib.oracle_cs_forces.argtypes = [C.c_void_p, C.c_double, _D, _D]
        _lib_cs = lib
        return lib


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        _common(lib)
        vp = C.c_void_p
        lib.oracle_limiter.argtypes = [vp, _D, _D, _D]
        lib.oracle_gradient.argtypes = [vp, _D, _D, _D]
        lib.oracle_bj_limiter.argtypes = [vp, _D, _D, _D]
        lib.oracle_set_threads.argtypes = [C.c_int]
        lib.oracle_sst_bvals.argtypes = [vp, _D]
        lib.oracle_convection.argtypes = [vp, _D, _D]
        lib.oracle_feq.argtypes = [C.c_double, C.c_double, C.c_double, _D]
        lib.oracle_sst_point.argtypes = [C.c_double] * 9 + [_D]
        _lib = lib
        return lib


def set_threads(n: int) -> None:
    """Threads of the oracle's per-cell loops (default 1).  The results do not depend on it."""
    _load().oracle_set_threads(int(n))


def feq(rho: float, u: float, v: float) -> np.ndarray:
    out = np.zeros(Q)
    _load().oracle_feq(rho, u, v, out)
    return out


def sst_point(k, w, d, gk, gw, S, nu) -> dict:
    out = np.zeros(4)
    _load().oracle_sst_point(k, w, d, gk[0], gk[1], gw[0], gw[1], S, nu, out)
    return {"f1": out[0], "f2": out[1], "cdkw": out[2], "nut": out[3]}


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Oracle:
    """One oracle instance for a ``meshgen.Case``; arrays are in the mesh's cell order and
    f is cell-major [n_cells, 9]."""

    def __init__(self, case, dt: float | None = None, sst: bool | None = None,
                 scheme: int = 0, complex_step: bool = False):
        lib = _load_cs() if complex_step else _load()
        m = case.mesh.normalized()
        rho, u, v, k, w = case.init_arrays()
        self._keep = (m, rho, u, v, k, w)
        params = np.array([case.nu, case.rho0, case.dt if dt is None else dt, case.cfl,
                           float(case.sst if sst is None else sst), case.uref, case.lref,
                           case.alpha_deg, float(scheme), float(case.local_dt),
                           float(case.variant)], np.float64)
        self._h = lib.oracle_create(m.n_nodes, m.xy.ravel(), m.n_cells, m.cell_ptr, m.cell_nodes,
                                    m.n_bedges, m.bedge_nodes.ravel(), m.bedge_type,
                                    m.bedge_val.ravel(), m.periodic_pairs.shape[0],
                                    m.periodic_pairs.ravel(), m.periodic_shift.ravel(),
                                    _ptr(rho), _ptr(u), _ptr(v), _ptr(k), _ptr(w), params)
        if not self._h:
            raise ValueError("oracle_create rejected the mesh")
        self.lib = lib
        self.n_cells = m.n_cells
        self.n_bedges = m.n_bedges

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self.lib.oracle_destroy(h)
            self._h = None

    @property
    def dt(self) -> float:
        return self.lib.oracle_dt(self._h)

    def dt_cells(self) -> np.ndarray:
        """dt of every cell (the global dt unless the case asks for local time stepping)."""
        out = np.zeros(self.n_cells)
        self.lib.oracle_dt_cells(self._h, out)
        return out

    def step(self, n: int = 1) -> None:
        if self.lib.oracle_step(self._h, int(n)) != 0:
            raise FloatingPointError("oracle step produced NaN")

    def residual(self) -> float:
        return self.lib.oracle_residual(self._h)

    def moment_defect(self) -> float:
        return self.lib.oracle_moment_defect(self._h)

    def mass(self) -> float:
        return self.lib.oracle_mass(self._h)

    def get_f(self) -> np.ndarray:
        f = np.zeros(self.n_cells * Q)
        self.lib.oracle_get_f(self._h, f)
        return f.reshape(self.n_cells, Q)

    def set_f(self, f: np.ndarray) -> None:
        self.lib.oracle_set_f(self._h, np.ascontiguousarray(f, np.float64).ravel())

    def set_turb(self, k: np.ndarray, omega: np.ndarray, nut: np.ndarray) -> None:
        self.lib.oracle_set_turb(self._h, *(np.ascontiguousarray(a, np.float64) for a in (k, omega, nut)))

    def set_wdist(self, d: np.ndarray) -> None:
        self.lib.oracle_set_wdist(self._h, np.ascontiguousarray(d, np.float64))

    def fields(self) -> dict:
        n = self.n_cells
        out = {key: np.zeros(n) for key in ("rho", "u", "v", "k", "omega", "nut")}
        self.lib.oracle_get_fields(self._h, out["rho"], out["u"], out["v"], out["k"],
                                   out["omega"], out["nut"])
        return out

    def geometry(self) -> dict:
        n = self.n_cells
        out = {key: np.zeros(n) for key in ("area", "cx", "cy", "wdist")}
        self.lib.oracle_geometry(self._h, out["area"], out["cx"], out["cy"], out["wdist"])
        return out

    def gradient(self, phi: np.ndarray, phib: np.ndarray) -> np.ndarray:
        g = np.zeros(2 * self.n_cells)
        self.lib.oracle_gradient(self._h, np.ascontiguousarray(phi, np.float64),
                                 np.ascontiguousarray(phib, np.float64), g)
        return g.reshape(self.n_cells, 2)

    def limiter(self, phi: np.ndarray, phib: np.ndarray) -> np.ndarray:
        """Limiter value per cell of the reconstruction of a scalar field (variant 1)."""
        psi = np.zeros(self.n_cells)
        self.lib.oracle_limiter(self._h, np.ascontiguousarray(phi, np.float64),
                                np.ascontiguousarray(phib, np.float64), psi)
        return psi

    def bj_limiter(self, phi: np.ndarray, phib: np.ndarray) -> np.ndarray:
        """Barth-Jespersen limiter value per cell of the SST reconstruction of a scalar field
        with boundary values phib [n_bedges], at its least-squares gradient."""
        psi = np.zeros(self.n_cells)
        self.lib.oracle_bj_limiter(self._h, np.ascontiguousarray(phi, np.float64),
                                   np.ascontiguousarray(phib, np.float64), psi)
        return psi

    def sst_bvals(self) -> np.ndarray:
        """[n_bedges, 4] boundary values (u, v, k, omega) the SST update uses at the current
        state (zeros on periodic edges)."""
        out = np.zeros(4 * self.n_bedges)
        self.lib.oracle_sst_bvals(self._h, out)
        return out.reshape(self.n_bedges, 4)

    def convection(self, f: np.ndarray) -> np.ndarray:
        ga = np.zeros(self.n_cells * Q)
        self.lib.oracle_convection(self._h, np.ascontiguousarray(f, np.float64).ravel(), ga)
        return ga.reshape(self.n_cells, Q)

    def cs_seed(self, dbedge_val=None, df=None, h: float = 1e-30) -> None:
        """Complex-step build only: seed d(boundary values) [n_bedges, 5] and / or df [n_cells, 9]
        as imaginary parts h * d."""
        bv = None if dbedge_val is None else np.ascontiguousarray(dbedge_val, np.float64)
        f = None if df is None else np.ascontiguousarray(df, np.float64)
        self.lib.oracle_cs_seed(self._h, _ptr(bv), _ptr(f), float(h))

    def cs_forces(self, h: float = 1e-30):
        """Complex-step build only: (forces, d forces / dp along the seeded direction)."""
        val, der = np.zeros(4), np.zeros(4)
        self.lib.oracle_cs_forces(self._h, float(h), val, der)
        keys = ("fx", "fy", "cd", "cl")
        return dict(zip(keys, val)), dict(zip(keys, der))

    def forces(self, per_edge: bool = False):
        """Total wall force and C_D, C_L; with ``per_edge`` also Cp and the force per edge."""
        out = np.zeros(4)
        nb = self.n_bedges
        cp, fxe, fye = (np.zeros(nb), np.zeros(nb), np.zeros(nb)) if per_edge else (None,) * 3
        self.lib.oracle_forces(self._h, out, _ptr(cp), _ptr(fxe), _ptr(fye))
        res = {"fx": out[0], "fy": out[1], "cd": out[2], "cl": out[3]}
        if per_edge:
            res.update(cp=cp, fx_edge=fxe, fy_edge=fye)
        return res
