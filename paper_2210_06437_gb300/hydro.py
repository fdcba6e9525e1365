"""Python binding of the C ABI in include/hydro.h (ctypes; argument marshalling only).

PyTorch provides device memory and streams; every step of the hydro path runs
in the CUDA library ``libhydro.so`` built in-tree by ``build.py``.  There is no
CPU fallback: if the library or a GPU is missing, constructing a HydroGrid
raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhydro.so")

NF, NP, NX, NG = 11, 14, 8, 3
HYDRO_FP64, HYDRO_MIXED = 0, 1
HYDRO_FLUX_KNP, HYDRO_FLUX_KT = 0, 1
PARAM_STAGE_CTAS_PER_SM, PARAM_GHOST_THREADS, PARAM_REFLUX, PARAM_TAU_RESYNC = 0, 1, 2, 3
PARAM_WAIT_LIMIT, PARAM_QUEUE_ORDER, PARAM_STAGE_GRID = 4, 5, 6
PARAM_PREFETCH_PASS, PARAM_REFLUX_SHAPE, PARAM_FUSED_RK3, PARAM_CW84, PARAM_RECON3D = 7, 8, 9, 10, 11
CW84_FLATTEN, CW84_STEEPEN = 1, 2
ITEM_FLUX_ONLY = 0x40000000   # batch id flag: export the sub-grid's coarse-fine fluxes, do not advance it
RK3_BETA = (1.0, 0.25, 2.0 / 3.0)

STATUS = {0: "HYDRO_OK", -1: "HYDRO_ERR_INVALID", -2: "HYDRO_ERR_CUDA", -3: "HYDRO_ERR_NOMEM",
          -4: "HYDRO_ERR_NONFINITE", -5: "HYDRO_ERR_TIMEOUT", -6: "HYDRO_ERR_STATE"}

# every symbol include/hydro.h declares
EXPORTS = ("hydro_create", "hydro_step", "hydro_shadow", "hydro_step_shadowed", "hydro_fill_ghosts", "hydro_rk3_step",
           "hydro_rk3_step_cfl", "hydro_rk3_run_cfl", "hydro_rk3_run_prepare", "hydro_totals", "hydro_diagnostics",
           "hydro_tau_resync", "hydro_totals_noalloc", "hydro_pack_interiors", "hydro_unpack_interiors",
           "hydro_pack_interiors_range", "hydro_unpack_interiors_range", "hydro_sync",
           "hydro_last_error", "hydro_launch_count", "hydro_set_param", "hydro_destroy")
SHADOW_FIELD = NX * NX * NX + (NX // 2) ** 3   # interior, then its 4^3 restriction
TOTALS_NOALLOC_MAX_SUBGRIDS = 65536
RK3_RUN_MAX_STEPS = 1024


class HydroError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


class GridDesc(ctypes.Structure):
    _fields_ = [("n_subgrids", ctypes.c_int32), ("n_fields", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("ghost", ctypes.c_int32), ("gamma", ctypes.c_double), ("de_switch", ctypes.c_double),
                ("precision", ctypes.c_int32), ("flux_form", ctypes.c_int32), ("dx", ctypes.c_void_p),
                ("neighbor", ctypes.c_void_p), ("neighbor_rel", ctypes.c_void_p), ("octant", ctypes.c_void_p)]


class Batch(ctypes.Structure):
    _fields_ = [("subgrid_ids", ctypes.c_void_p), ("n_items", ctypes.c_int32),
                ("batch_offsets", ctypes.c_void_p), ("n_batches", ctypes.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libhydro.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libhydro.so is missing: run paper_2210_06437_gb300.build.build() (nvcc, sm_103a)")
    L = ctypes.CDLL(path)
    vp, i32, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    L.hydro_create.argtypes = [ctypes.POINTER(GridDesc), ctypes.POINTER(vp)]
    L.hydro_step.argtypes = [vp, ctypes.POINTER(Batch), vp, vp, dbl, dbl, vp, vp, vp]
    L.hydro_shadow.argtypes = [vp, vp, vp, vp]
    L.hydro_step_shadowed.argtypes = [vp, ctypes.POINTER(Batch), vp, vp, vp, dbl, dbl, vp, vp, vp, vp]
    L.hydro_fill_ghosts.argtypes = [vp, vp, vp]
    L.hydro_pack_interiors.argtypes = [vp, vp, vp, vp]
    L.hydro_unpack_interiors.argtypes = [vp, vp, vp, vp]
    L.hydro_pack_interiors_range.argtypes = [vp, vp, vp, i32, i32, vp]
    L.hydro_unpack_interiors_range.argtypes = [vp, vp, vp, i32, i32, vp]
    L.hydro_rk3_step.argtypes = [vp, ctypes.POINTER(Batch), vp, vp, vp, dbl, vp, vp]
    L.hydro_rk3_step_cfl.argtypes = [vp, ctypes.POINTER(Batch), vp, vp, vp, dbl, vp, vp, vp]
    L.hydro_rk3_run_cfl.argtypes = [vp, ctypes.POINTER(Batch), vp, vp, vp, dbl, i32, vp, vp, vp, vp]
    L.hydro_rk3_run_prepare.argtypes = [vp, ctypes.POINTER(Batch), vp, vp, vp, dbl, i32, vp, vp, vp]
    L.hydro_totals.argtypes = [vp, vp, vp, vp]
    L.hydro_diagnostics.argtypes = [vp, vp, vp, vp, vp]
    L.hydro_totals_noalloc.argtypes = [vp, vp, i32, vp, vp]
    L.hydro_tau_resync.argtypes = [vp, vp, vp, vp]
    L.hydro_sync.argtypes = [vp]
    L.hydro_last_error.argtypes = [vp]
    L.hydro_last_error.restype = ctypes.c_char_p
    L.hydro_launch_count.argtypes = [vp]
    L.hydro_launch_count.restype = ctypes.c_int64
    L.hydro_set_param.argtypes = [vp, i32, i32]
    L.hydro_destroy.argtypes = [vp]
    L.hydro_destroy.restype = None
    for name in EXPORTS:
        if name not in ("hydro_last_error", "hydro_launch_count", "hydro_destroy"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class HydroGrid:
    """A grid handle on the current CUDA device.

    ``grid`` is a workloads.Grid-like object with arrays dx, neighbor,
    neighbor_rel, octant and attributes n, gamma, de_switch."""

    def __init__(self, grid, precision: str = "fp64", flux_form: int = HYDRO_FLUX_KNP,
                 gamma: Optional[float] = None, de_switch: Optional[float] = None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("HydroGrid needs a CUDA device; there is no CPU path")
        self.lib = load_library()
        self.n = int(grid.n)
        self.precision = precision
        self._dx = np.ascontiguousarray(grid.dx, np.float64)
        self._origin = getattr(grid, "origin", None)
        self._origin_dev = None
        self._nb = np.ascontiguousarray(grid.neighbor, np.int32)
        self._rel = np.ascontiguousarray(grid.neighbor_rel, np.int8)
        self._oct = np.ascontiguousarray(grid.octant, np.int8)
        d = GridDesc(self.n, NF, NX, NG, grid.gamma if gamma is None else gamma,
                     grid.de_switch if de_switch is None else de_switch,
                     HYDRO_MIXED if precision == "mixed" else HYDRO_FP64, flux_form,
                     self._dx.ctypes.data, self._nb.ctypes.data, self._rel.ctypes.data, self._oct.ctypes.data)
        h = ctypes.c_void_p()
        rc = self.lib.hydro_create(ctypes.byref(d), ctypes.byref(h))
        if rc != 0:
            raise HydroError(rc, "hydro_create")
        self.h = h
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._all = torch.arange(self.n, dtype=torch.int32, device=self.device)
        self._ms = torch.zeros(2, dtype=torch.float64, device=self.device)

    # -- helpers ------------------------------------------------------------
    def _check(self, rc):
        if rc != 0:
            raise HydroError(rc, self.lib.hydro_last_error(self.h).decode())

    def _batch(self, ids, offsets):
        import torch
        if ids is None:
            ids = self._all
        elif not isinstance(ids, torch.Tensor) or ids.device.type != "cuda":
            ids = torch.as_tensor(np.asarray(ids, np.int32), device=self.device)
        assert ids.dtype == torch.int32 and ids.is_contiguous()
        b = Batch(ids.data_ptr() if ids.numel() else None, ids.numel(), None, 0)
        keep = [ids]
        if offsets is not None:
            off = np.ascontiguousarray(offsets, np.int32)
            b.batch_offsets = off.ctypes.data
            b.n_batches = len(off) - 1
            keep.append(off)
        return b, keep

    def empty_state(self):
        import torch
        return torch.empty((self.n, NF, NP, NP, NP), dtype=torch.float64, device=self.device)

    def _state(self, U):
        import torch
        assert isinstance(U, torch.Tensor) and U.dtype == torch.float64 and U.is_cuda and U.is_contiguous()
        assert tuple(U.shape) == (self.n, NF, NP, NP, NP)
        return U

    # -- ABI calls ----------------------------------------------------------
    def step(self, U_in, dt, U0=None, beta=1.0, U_out=None, ids=None, batch_offsets=None, max_speed=None,
             stream=None):
        """One RK stage (hydro_step).  Returns (U_out, max_speed tensor[2])."""
        self._state(U_in)
        if U_out is None:
            U_out = U_in.clone()
        self._state(U_out)
        ms = self._ms if max_speed is None else max_speed
        b, keep = self._batch(ids, batch_offsets)
        self._check(self.lib.hydro_step(self.h, ctypes.byref(b), _ptr(U_in), _ptr(U0), float(beta), float(dt),
                                        _ptr(U_out), _ptr(ms), _stream_ptr(stream)))
        return U_out, ms

    def empty_shadow(self):
        import torch
        return torch.empty((self.n, NF, SHADOW_FIELD), dtype=torch.float32, device=self.device)

    def _shadow_buf(self, S):
        import torch
        assert isinstance(S, torch.Tensor) and S.dtype == torch.float32 and S.is_cuda and S.is_contiguous()
        assert S.numel() == self.n * NF * SHADOW_FIELD
        return S

    def shadow(self, U, S=None, stream=None):
        """FP32 shadow of U's interiors (hydro_shadow).  Returns S [n, 11, 512]."""
        self._state(U)
        S = self.empty_shadow() if S is None else self._shadow_buf(S)
        self._check(self.lib.hydro_shadow(self.h, _ptr(U), _ptr(S), _stream_ptr(stream)))
        return S

    def step_shadowed(self, U_in, S_in, dt, U0=None, beta=1.0, U_out=None, S_out=None, ids=None, batch_offsets=None,
                      max_speed=None, stream=None):
        """One RK stage from a caller-held shadow (hydro_step_shadowed, mixed
        precision).  Returns (U_out, max_speed tensor[2])."""
        self._state(U_in)
        self._shadow_buf(S_in)
        if S_out is not None:
            self._shadow_buf(S_out)
        if U_out is None:
            U_out = U_in.clone()
        self._state(U_out)
        ms = self._ms if max_speed is None else max_speed
        b, keep = self._batch(ids, batch_offsets)
        self._check(self.lib.hydro_step_shadowed(self.h, ctypes.byref(b), _ptr(U_in), _ptr(S_in), _ptr(U0),
                                                 float(beta), float(dt), _ptr(U_out), _ptr(S_out), _ptr(ms),
                                                 _stream_ptr(stream)))
        return U_out, ms

    def empty_interiors(self, pin_memory=False, device=None):
        """A packed-interior array [n, 11, 512] float64 (device, or pinned host)."""
        import torch
        if device == "cpu" or pin_memory:
            return torch.empty((self.n, NF, NX ** 3), dtype=torch.float64, pin_memory=pin_memory)
        return torch.empty((self.n, NF, NX ** 3), dtype=torch.float64, device=self.device)

    def _packed(self, P):
        import torch
        assert isinstance(P, torch.Tensor) and P.dtype == torch.float64 and P.is_cuda and P.is_contiguous()
        assert P.numel() == self.n * NF * NX ** 3
        return P

    def pack(self, U, P=None, stream=None, first=None, count=None):
        """Interiors of U into the packed array P (hydro_pack_interiors); with
        first/count, only those sub-grids (hydro_pack_interiors_range)."""
        self._state(U)
        P = self.empty_interiors() if P is None else self._packed(P)
        if first is None:
            self._check(self.lib.hydro_pack_interiors(self.h, _ptr(U), _ptr(P), _stream_ptr(stream)))
        else:
            self._check(self.lib.hydro_pack_interiors_range(self.h, _ptr(U), _ptr(P), first, count,
                                                            _stream_ptr(stream)))
        return P

    def unpack(self, P, U, stream=None, first=None, count=None):
        """Interiors of U from the packed array P (hydro_unpack_interiors); with
        first/count, only those sub-grids (hydro_unpack_interiors_range)."""
        self._state(U)
        self._packed(P)
        if first is None:
            self._check(self.lib.hydro_unpack_interiors(self.h, _ptr(P), _ptr(U), _stream_ptr(stream)))
        else:
            self._check(self.lib.hydro_unpack_interiors_range(self.h, _ptr(P), _ptr(U), first, count,
                                                              _stream_ptr(stream)))
        return U

    def upload(self, P_host, U, P_dev, stream=None):
        """Host packed interiors (pinned) -> device state U: copy into P_dev, unpack."""
        P_dev.copy_(P_host, non_blocking=True)
        return self.unpack(P_dev, U, stream)

    def download(self, U, P_dev, P_host, stream=None):
        """Device state U -> host packed interiors (pinned): pack into P_dev, copy."""
        self.pack(U, P_dev, stream)
        P_host.copy_(P_dev, non_blocking=True)
        return P_host

    def fill_ghosts(self, U, stream=None):
        self._state(U)
        self._check(self.lib.hydro_fill_ghosts(self.h, _ptr(U), _stream_ptr(stream)))
        return U

    def rk3_step(self, U, dt, scratch1, scratch2, ids=None, batch_offsets=None, max_speed=None, stream=None):
        """One SSP-RK3 step in place on U (hydro_rk3_step, graph replay).  Returns max_speed[2]."""
        for t in (U, scratch1, scratch2):
            self._state(t)
        ms = self._ms if max_speed is None else max_speed
        b, keep = self._batch(ids, batch_offsets)
        self._keep = keep  # the captured graph refers to these device ids
        self._check(self.lib.hydro_rk3_step(self.h, ctypes.byref(b), _ptr(U), _ptr(scratch1), _ptr(scratch2),
                                            float(dt), _ptr(ms), _stream_ptr(stream)))
        return ms

    def rk3_step_cfl(self, U, cfl, scratch1, scratch2, max_speed, ids=None, batch_offsets=None, dt_out=None,
                     stream=None):
        """One SSP-RK3 step with dt = cfl / max_speed[1] chosen on the device
        (hydro_rk3_step_cfl).  max_speed must hold the previous first-stage
        speeds on entry; it holds this step's on exit."""
        for t in (U, scratch1, scratch2):
            self._state(t)
        b, keep = self._batch(ids, batch_offsets)
        self._keep = keep
        self._check(self.lib.hydro_rk3_step_cfl(self.h, ctypes.byref(b), _ptr(U), _ptr(scratch1), _ptr(scratch2),
                                                float(cfl), _ptr(max_speed), _ptr(dt_out), _stream_ptr(stream)))
        return max_speed

    def rk3_run_cfl(self, U, cfl, scratch1, scratch2, max_speed, n_steps, ids=None, batch_offsets=None,
                    dt_out=None, totals=None, stream=None):
        """n_steps SSP-RK3 steps with device-chosen dt in one graph launch
        (hydro_rk3_run_cfl); dt_out [n_steps] and totals [n_steps, 11] are
        optional device outputs.  Returns max_speed."""
        for t in (U, scratch1, scratch2):
            self._state(t)
        b, keep = self._batch(ids, batch_offsets)
        self._keep = keep
        self._check(self.lib.hydro_rk3_run_cfl(self.h, ctypes.byref(b), _ptr(U), _ptr(scratch1), _ptr(scratch2),
                                               float(cfl), int(n_steps), _ptr(max_speed), _ptr(dt_out),
                                               _ptr(totals), _stream_ptr(stream)))
        return max_speed

    def rk3_run_prepare(self, U, cfl, scratch1, scratch2, max_speed, n_steps, ids=None, batch_offsets=None,
                        dt_out=None, totals=None):
        """Capture the graph of the matching rk3_run_cfl call without running it."""
        for t in (U, scratch1, scratch2):
            self._state(t)
        b, keep = self._batch(ids, batch_offsets)
        self._keep = keep
        self._check(self.lib.hydro_rk3_run_prepare(self.h, ctypes.byref(b), _ptr(U), _ptr(scratch1),
                                                   _ptr(scratch2), float(cfl), int(n_steps), _ptr(max_speed),
                                                   _ptr(dt_out), _ptr(totals)))

    def totals(self, U, out=None, stream=None):
        import torch
        self._state(U)
        out = torch.empty(NF, dtype=torch.float64, device=self.device) if out is None else out
        self._check(self.lib.hydro_totals(self.h, _ptr(U), _ptr(out), _stream_ptr(stream)))
        return out

    def diagnostics(self, U, out=None, stream=None):
        """[M, Lx, Ly, Lz, M1, X1, Y1, Z1, M2, X2, Y2, Z2] (hydro_diagnostics);
        needs the grid's sub-grid origins."""
        import torch
        self._state(U)
        if self._origin_dev is None:
            if self._origin is None:
                raise ValueError("the grid descriptor has no sub-grid origins")
            self._origin_dev = torch.as_tensor(np.ascontiguousarray(self._origin, np.float64), device=self.device)
        out = torch.empty(12, dtype=torch.float64, device=self.device) if out is None else out
        self._check(self.lib.hydro_diagnostics(self.h, _ptr(U), _ptr(self._origin_dev), _ptr(out),
                                               _stream_ptr(stream)))
        return out

    def tau_resync(self, U, S=None, stream=None):
        """Dual-energy reset of the entropy tracer in place (hydro_tau_resync);
        S (mixed handles) is a shadow of U whose tau field is refreshed."""
        self._state(U)
        if S is not None:
            self._shadow_buf(S)
        self._check(self.lib.hydro_tau_resync(self.h, _ptr(U), _ptr(S), _stream_ptr(stream)))
        return U

    def sync(self):
        """Wait and return the device status; raises HydroError on a device-side error."""
        self._check(self.lib.hydro_sync(self.h))

    def set_param(self, key, value):
        self._check(self.lib.hydro_set_param(self.h, key, value))

    @property
    def launches(self) -> int:
        return int(self.lib.hydro_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.hydro_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
