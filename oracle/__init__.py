"""CPU oracle for the batched octree hydro step (ctypes binding of hydro_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
CPU-baseline / reference leg of the benchmark.  The CUDA library and its Python
binding never import it, and it imports nothing from them.

``build()`` compiles ``hydro_oracle.c`` with gcc (-O2 -ffp-contract=off, OpenMP
when available) into ``liboracle.so`` next to this file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hydro_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

NF, NP = 11, 14
RK3_BETA = (1.0, 0.25, 2.0 / 3.0)  # Shu-Osher SSP-RK3 stage weights beta (alpha = 1 - beta)


def build(force: bool = False) -> str:
    """Compile the oracle shared library; returns its path."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "hydro_oracle.h"))):
        return _LIB
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c99", _SRC, "-o", _LIB,
            "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    return _LIB


class _Grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("gamma", ctypes.c_double), ("de_switch", ctypes.c_double),
                ("flux_form", ctypes.c_int32), ("dx", ctypes.c_void_p), ("neighbor", ctypes.c_void_p),
                ("neighbor_rel", ctypes.c_void_p), ("octant", ctypes.c_void_p), ("reflux", ctypes.c_int32),
                ("cw84", ctypes.c_int32)]

# CW84 PPM extensions (Oracle(cw84=...)): shock flattening, contact steepening of the density
CW84_FLATTEN, CW84_STEEPEN = 1, 2


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        L.oracle_ppm_pencil.argtypes = [dp, dp, dp]
        L.oracle_face_eos.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp, dp]
        L.oracle_face_flux.argtypes = [dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp]
        L.oracle_face_flux.restype = ctypes.c_double
        L.oracle_stage.argtypes = [ctypes.POINTER(_Grid), ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_void_p, dp, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        L.oracle_fill_ghosts.argtypes = [ctypes.POINTER(_Grid), ctypes.c_void_p]
        L.oracle_totals.argtypes = [ctypes.POINTER(_Grid), ctypes.c_void_p, dp]
        L.oracle_diagnostics.argtypes = [ctypes.POINTER(_Grid), ctypes.c_void_p, ctypes.c_void_p, dp]
        L.oracle_tau_resync.argtypes = [ctypes.POINTER(_Grid), ctypes.c_void_p]
        L.oracle_tau_resync.restype = ctypes.c_long
        L.oracle_margin_cells.argtypes = [ctypes.POINTER(_Grid), ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                          ctypes.c_double, ctypes.c_void_p]
        L.oracle_margin_cells.restype = ctypes.c_long
        L.oracle_ghost_cell.argtypes = [ctypes.POINTER(_Grid), ctypes.c_void_p] + [ctypes.c_int] * 6
        L.oracle_ghost_cell.restype = ctypes.c_double
        L.oracle_fill_ghosts_full.argtypes = [ctypes.POINTER(_Grid), ctypes.c_void_p]
        L.oracle_simpson_flux.argtypes = [dp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp]
        L.oracle_simpson_flux.restype = ctypes.c_double
        L.oracle_stage3d.argtypes = [ctypes.POINTER(_Grid), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_void_p, dp, ctypes.c_int]
        L.oracle_margin_cells3d.argtypes = [ctypes.POINTER(_Grid), ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]
        L.oracle_margin_cells3d.restype = ctypes.c_long
        _lib = L
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def ppm_pencil(q: Sequence[float]) -> Tuple[np.ndarray, np.ndarray]:
    q = np.ascontiguousarray(q, np.float64)
    assert q.shape == (NP,)
    aL = np.full(NP, np.nan)
    aR = np.full(NP, np.nan)
    lib().oracle_ppm_pencil(_dptr(q), _dptr(aL), _dptr(aR))
    return aL, aR


def face_eos(U, d, gamma=5.0 / 3.0, eta=1e-3):
    U = np.ascontiguousarray(U, np.float64)
    u, p, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().oracle_face_eos(_dptr(U), d, gamma, eta, ctypes.byref(u), ctypes.byref(p), ctypes.byref(c))
    return u.value, p.value, c.value


def simpson_flux(AL, AR, d, gamma=5.0 / 3.0, eta=1e-3, form=0):
    """Simpson flux of one face from the face averages [3][3][11] (left, right) of
    the 3 x 3 faces around it.  Returns (F[11], speed)."""
    AL = np.ascontiguousarray(AL, np.float64)
    AR = np.ascontiguousarray(AR, np.float64)
    assert AL.shape == (3, 3, NF) and AR.shape == (3, 3, NF)
    F = np.zeros(NF)
    a = lib().oracle_simpson_flux(_dptr(AL), _dptr(AR), int(d), float(gamma), float(eta), int(form), _dptr(F))
    return F, a


def face_flux(UL, UR, d, gamma=5.0 / 3.0, eta=1e-3, form=0):
    UL = np.ascontiguousarray(UL, np.float64)
    UR = np.ascontiguousarray(UR, np.float64)
    F = np.zeros(NF)
    a = lib().oracle_face_flux(_dptr(UL), _dptr(UR), d, gamma, eta, form, _dptr(F))
    return F, a


class Oracle:
    """Oracle bound to one grid descriptor (see ``paper_2210_06437_gb300.workloads.Grid``)."""

    def __init__(self, grid, flux_form: int = 0, gamma: Optional[float] = None, de_switch: Optional[float] = None,
                 reflux: bool = True, cw84: int = 0):
        self.grid = grid
        self._dx = np.ascontiguousarray(grid.dx, np.float64)
        self._nb = np.ascontiguousarray(grid.neighbor, np.int32)
        self._rel = np.ascontiguousarray(grid.neighbor_rel, np.int8)
        self._oct = np.ascontiguousarray(grid.octant, np.int8)
        self._g = _Grid(grid.n, grid.gamma if gamma is None else gamma,
                        grid.de_switch if de_switch is None else de_switch, flux_form,
                        self._dx.ctypes.data, self._nb.ctypes.data, self._rel.ctypes.data, self._oct.ctypes.data,
                        1 if reflux else 0, int(cw84))

    def _check(self, U):
        assert U.dtype == np.float64 and U.flags.c_contiguous and U.shape == (self.grid.n, NF, NP, NP, NP)

    def fill_ghosts(self, U: np.ndarray) -> np.ndarray:
        self._check(U)
        lib().oracle_fill_ghosts(ctypes.byref(self._g), U.ctypes.data)
        return U

    def stage(self, Uin: np.ndarray, dt: float, U0: Optional[np.ndarray] = None, beta: float = 1.0,
              Uout: Optional[np.ndarray] = None, ids=None, nthreads: int = 0,
              sub_amax: Optional[np.ndarray] = None, batch_all: bool = False):
        """One RK stage Uout = U0 + beta (U* - U0), U* = Uin + dt/dx dU; returns
        (Uout, max_speed[2], status).  Uout defaults to a copy of Uin.  The
        coarse-fine flux correction uses the finer neighbours advanced by the
        same call: those in `ids`, or every sub-grid with batch_all (a call on
        the whole grid of which only `ids` are computed here)."""
        self._check(Uin)
        if Uout is None:
            Uout = Uin.copy()
        self._check(Uout)
        if U0 is not None:
            self._check(U0)
        ms = np.zeros(2)
        if ids is not None:
            ids = np.ascontiguousarray(ids, np.int32)
        st = lib().oracle_stage(ctypes.byref(self._g), None if ids is None else ids.ctypes.data,
                                0 if ids is None else len(ids), Uin.ctypes.data,
                                None if U0 is None else U0.ctypes.data, beta, dt, Uout.ctypes.data,
                                _dptr(ms), None if sub_amax is None else sub_amax.ctypes.data, nthreads,
                                1 if batch_all else 0)
        return Uout, ms, st

    def rk3_step(self, U: np.ndarray, dt: float, nthreads: int = 0, tau_resync: bool = False):
        """One SSP-RK3 step from U (ghosts filled); returns (U_new with ghosts filled,
        max_speed of the first stage, worst status).  tau_resync: reset the
        entropy tracer from the internal energy at the end of the step."""
        st_all = 0
        U1, ms, st = self.stage(U, dt, nthreads=nthreads)
        st_all = min(st_all, st)
        self.fill_ghosts(U1)
        U2, _, st = self.stage(U1, dt, U0=U, beta=RK3_BETA[1], nthreads=nthreads)
        st_all = min(st_all, st)
        self.fill_ghosts(U2)
        U3, _, st = self.stage(U2, dt, U0=U, beta=RK3_BETA[2], nthreads=nthreads)
        st_all = min(st_all, st)
        if tau_resync:
            self.tau_resync(U3)
        self.fill_ghosts(U3)
        return U3, ms, st_all

    def tau_resync(self, U: np.ndarray) -> int:
        """Dual-energy reset tau = e_i^(1/gamma) where e_i >= eta E (interior
        cells, in place); returns the number of cells reset."""
        self._check(U)
        return int(lib().oracle_tau_resync(ctypes.byref(self._g), U.ctypes.data))

    def margin_cells(self, U: np.ndarray, eps: float, ids=None, mask: Optional[np.ndarray] = None):
        """Interior cells near a branch decision of the scheme on input U (ghosts
        filled): tests within 64 eps of their threshold, spread 3 cells along
        their pencil.  Returns (mask [n, 8, 8, 8] bool, OR-ed into `mask` when
        given, number of near decisions)."""
        self._check(U)
        m = np.zeros((self.grid.n, 8, 8, 8), np.uint8) if mask is None else mask
        assert m.dtype == np.uint8 and m.flags.c_contiguous and m.shape == (self.grid.n, 8, 8, 8)
        if ids is not None:
            ids = np.ascontiguousarray(ids, np.int32)
        k = lib().oracle_margin_cells(ctypes.byref(self._g), None if ids is None else ids.ctypes.data,
                                      0 if ids is None else len(ids), U.ctypes.data, 64.0 * eps, m.ctypes.data)
        return m, int(k)

    def ghost_cell(self, U: np.ndarray, s: int, face: int, ga: int, c1: int, c2: int, f: int) -> float:
        """The ghost value of field f of sub-grid s across face at interior
        coordinate ga along its axis (any depth) by the ghost-fill rules."""
        self._check(U)
        return float(lib().oracle_ghost_cell(ctypes.byref(self._g), U.ctypes.data, int(s), int(face), int(ga),
                                             int(c1), int(c2), int(f)))

    def fill_ghosts_full(self, U: np.ndarray) -> np.ndarray:
        """Every ghost cell of the padded cubes (faces, edges, corners) of a grid of one level."""
        self._check(U)
        if lib().oracle_fill_ghosts_full(ctypes.byref(self._g), U.ctypes.data) != 0:
            raise ValueError("the 3D reconstruction needs a grid of one level")
        return U

    def stage3d(self, Uin: np.ndarray, dt: float, U0: Optional[np.ndarray] = None, beta: float = 1.0,
                Uout: Optional[np.ndarray] = None, nthreads: int = 0):
        """One RK stage with the 3D reconstruction and Simpson face quadrature
        (every sub-grid; ghosts filled by fill_ghosts_full).  Returns (Uout,
        max_speed[2], status)."""
        self._check(Uin)
        if U0 is not None:
            self._check(U0)
        Uout = Uin.copy() if Uout is None else Uout
        ms = np.zeros(2)
        st = lib().oracle_stage3d(ctypes.byref(self._g), Uin.ctypes.data, None if U0 is None else U0.ctypes.data,
                                  float(beta), float(dt), Uout.ctypes.data, _dptr(ms), int(nthreads))
        return Uout, ms, st

    def margin_cells3d(self, U: np.ndarray, eps: float, mask: Optional[np.ndarray] = None):
        """Interior cells beside faces whose 3D-reconstruction point states sit
        within 64 eps of a transverse test or of the dual-energy test (U: any
        padded state; its ghosts are filled on a copy).  Returns (mask [n, 8,
        8, 8] uint8, OR-ed into `mask` when given, number of marked faces)."""
        self._check(U)
        Uf = self.fill_ghosts_full(U.copy())
        m = np.zeros((self.grid.n, 8, 8, 8), np.uint8) if mask is None else mask
        assert m.dtype == np.uint8 and m.flags.c_contiguous and m.shape == (self.grid.n, 8, 8, 8)
        k = lib().oracle_margin_cells3d(ctypes.byref(self._g), Uf.ctypes.data, 64.0 * eps, m.ctypes.data)
        if k < 0:
            raise ValueError("the 3D reconstruction needs a grid of one level")
        return m, int(k)

    def rk3_step3d(self, U: np.ndarray, dt: float, nthreads: int = 0):
        """One SSP-RK3 step with stage3d (ghosts refilled before each stage)."""
        self.fill_ghosts_full(U)
        U1, ms, st1 = self.stage3d(U, dt, nthreads=nthreads)
        self.fill_ghosts_full(U1)
        U2, _, st2 = self.stage3d(U1, dt, U0=U, beta=0.25, nthreads=nthreads)
        self.fill_ghosts_full(U2)
        U3, _, st3 = self.stage3d(U2, dt, U0=U, beta=2.0 / 3.0, nthreads=nthreads)
        return U3, ms, st1 | st2 | st3

    def totals(self, U: np.ndarray) -> np.ndarray:
        self._check(U)
        t = np.zeros(NF)
        lib().oracle_totals(ctypes.byref(self._g), U.ctypes.data, _dptr(t))
        return t

    def diagnostics(self, U: np.ndarray, origin: Optional[np.ndarray] = None) -> np.ndarray:
        """[M, Lx, Ly, Lz, M1, X1, Y1, Z1, M2, X2, Y2, Z2] (Section V-B.1 diagnostics)."""
        self._check(U)
        o = np.ascontiguousarray(self.grid.origin if origin is None else origin, np.float64)
        assert o.shape == (self.grid.n, 3)
        out = np.zeros(12)
        lib().oracle_diagnostics(ctypes.byref(self._g), U.ctypes.data, o.ctypes.data, _dptr(out))
        return out
