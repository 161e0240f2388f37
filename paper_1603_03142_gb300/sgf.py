"""Thin ctypes binding of libsgf (C ABI in include/sgf.h).

Argument marshalling only: every step of the force computation runs in the
CUDA kernels of libsgf.so.  PyTorch supplies device memory and streams.  There
is no fallback: importing this module raises if the native library is missing
(build it with ``__graft_entry__.build()`` or ``python -m paper_1603_03142_gb300._build``).
"""
from __future__ import annotations

import ctypes
from pathlib import Path
from typing import List, Optional, Sequence

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "libsgf.so"
if not _LIB_PATH.exists():
    raise ImportError(f"libsgf.so not built at {_LIB_PATH}: run __graft_entry__.build() first")
_lib = ctypes.CDLL(str(_LIB_PATH))

SGF_MAX_LEVELS = 8
SGF_MAX_PATCHES = 16
SGF_OK, SGF_EINVAL, SGF_ENOMEM, SGF_ECUDA, SGF_ETIMEOUT, SGF_EUNSUPPORTED = range(6)
STATUS_NAMES = {0: "SGF_OK", 1: "SGF_EINVAL", 2: "SGF_ENOMEM", 3: "SGF_ECUDA", 4: "SGF_ETIMEOUT",
                5: "SGF_EUNSUPPORTED"}
FP64, FP32, BF16X = 0, 1, 2
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16x": BF16X}

# every symbol include/sgf.h declares
EXPORTS = ["sgf_plan_create", "sgf_plan_create_ex", "sgf_plan_check", "sgf_plan_share", "sgf_plan_stats_get",
           "sgf_solve", "sgf_solve_host", "sgf_solve_batched", "sgf_plan_destroy", "sgf_last_error", "sgf_version",
           "sgf_plan_profile", "sgf_plan_profile_read", "sgf_solve_noalloc", "sgf_batch_create",
           "sgf_batch_solve", "sgf_batch_info", "sgf_batch_destroy", "sgf_plan_estimate", "sgf_server_create",
           "sgf_server_clock", "sgf_server_submit", "sgf_server_progress", "sgf_server_stats_get",
           "sgf_server_destroy", "sgf_plan_schedule_get", "sgf_plan_schedule_set", "sgf_plan_autotune",
           "sgf_plan_share_ex", "sgf_solve_potential", "sgf_plan_create_forest", "sgf_plan_estimate_forest",
           "sgf_plan_footprint", "sgf_plan_inject_timeout", "sgf_solve_host_many"]
BATCH_NO_GRAPH = 0x1
PLAN_ZERO_RIM = 0x1
PLAN_POTENTIAL = 0x2
NOALLOC_SCRATCH_BYTES = 32 << 20
AUTOTUNE_TIMES = 18
KERNELS = ["restrict", "row_fwd", "col", "row_inv"]


class NestDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("levels", ctypes.c_int32), ("x0", ctypes.c_double),
                ("y0", ctypes.c_double), ("h0", ctypes.c_double),
                ("off", (ctypes.c_int32 * 2) * SGF_MAX_LEVELS)]


class ForestDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("patches", ctypes.c_int32), ("x0", ctypes.c_double),
                ("y0", ctypes.c_double), ("h0", ctypes.c_double),
                ("level", ctypes.c_int32 * SGF_MAX_PATCHES),
                ("org", (ctypes.c_int32 * 2) * SGF_MAX_PATCHES)]


class PlanStats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("levels", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("forward_slabs", ctypes.c_int32), ("outputs", ctypes.c_int32),
                ("spectra_sets", ctypes.c_int32), ("launches_per_solve", ctypes.c_int32),
                ("workspace_bytes", ctypes.c_size_t), ("spectra_bytes", ctypes.c_size_t),
                ("algorithmic_bytes", ctypes.c_size_t), ("plan_ms", ctypes.c_double),
                ("spectra_sets_streamed", ctypes.c_int32), ("spectra_waves", ctypes.c_int32),
                ("spectra_window_bytes", ctypes.c_size_t)]


class KernelTimes(ctypes.Structure):
    _fields_ = [("solves", ctypes.c_int32), ("launches", ctypes.c_int32 * 4), ("ms", ctypes.c_double * 4)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("max_inflight", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("simulate_gbs", ctypes.c_double), ("max_shape_bytes", ctypes.c_size_t)]


class Request(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("desc", NestDesc), ("precision", ctypes.c_int), ("plan_flags", ctypes.c_uint32),
                ("sigma", ctypes.c_void_p * SGF_MAX_LEVELS), ("fx", ctypes.c_void_p * SGF_MAX_LEVELS),
                ("fy", ctypes.c_void_p * SGF_MAX_LEVELS)]


class Completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("slot", ctypes.c_int32),
                ("built_shape", ctypes.c_int32), ("pad", ctypes.c_int32), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("queued", ctypes.c_int32), ("inflight", ctypes.c_int32),
                ("inflight_peak", ctypes.c_int32), ("slots", ctypes.c_int32), ("shapes_resident", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("shapes_built", ctypes.c_int64), ("slots_evicted", ctypes.c_int64),
                ("bytes_used", ctypes.c_size_t), ("bytes_peak", ctypes.c_size_t), ("hbm_budget", ctypes.c_size_t)]


class Schedule(ctypes.Structure):
    _fields_ = [("col_pass", ctypes.c_int32), ("row_inv0", ctypes.c_int32), ("col_case3", ctypes.c_int32),
                ("col_radix", ctypes.c_int32), ("inv_radix", ctypes.c_int32), ("row_fwd", ctypes.c_int32)]


SERVER_SIMULATE = 0x1
SERVER_NO_AUTOTUNE = 0x2
SERVER_STREAM = 0x4
INJECT_TMA_GATHER = 0x1
INJECT_TC_COMMIT = 0x2
_vpp = ctypes.POINTER(ctypes.c_void_p)
_szp = ctypes.POINTER(ctypes.c_size_t)
_lib.sgf_plan_create.argtypes = [ctypes.POINTER(NestDesc), ctypes.c_int, ctypes.c_size_t,
                                 ctypes.POINTER(ctypes.c_void_p)]
_lib.sgf_plan_footprint.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]
_lib.sgf_plan_inject_timeout.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int64]
_lib.sgf_plan_create_ex.argtypes = [ctypes.POINTER(NestDesc), ctypes.c_int, ctypes.c_uint32,
                                    ctypes.POINTER(ctypes.c_void_p)]
_lib.sgf_plan_check.argtypes = [ctypes.c_void_p]
_lib.sgf_plan_share.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
_lib.sgf_plan_share_ex.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
_lib.sgf_plan_stats_get.argtypes = [ctypes.c_void_p, ctypes.POINTER(PlanStats)]
_lib.sgf_solve.argtypes = [ctypes.c_void_p, _vpp, _vpp, _vpp, ctypes.c_void_p]
_lib.sgf_solve_host.argtypes = [ctypes.c_void_p, _vpp, _vpp, _vpp, ctypes.c_void_p]
_lib.sgf_solve_host_many.argtypes = [ctypes.c_void_p, ctypes.c_int32, _vpp, _vpp, _vpp, ctypes.c_void_p]
_lib.sgf_solve_noalloc.argtypes = [ctypes.c_void_p, _vpp, _vpp, _vpp, ctypes.c_void_p]
_lib.sgf_solve_potential.argtypes = [ctypes.c_void_p, _vpp, _vpp, ctypes.c_void_p]
_lib.sgf_batch_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, ctypes.c_uint32,
                                  ctypes.POINTER(ctypes.c_void_p)]
_lib.sgf_batch_solve.argtypes = [ctypes.c_void_p, ctypes.POINTER(_vpp), ctypes.POINTER(_vpp), ctypes.POINTER(_vpp),
                                 ctypes.c_void_p]
_lib.sgf_batch_info.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
_lib.sgf_batch_destroy.argtypes = [ctypes.c_void_p]
_lib.sgf_solve_batched.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32,
                                   ctypes.POINTER(_vpp), ctypes.POINTER(_vpp), ctypes.POINTER(_vpp),
                                   ctypes.c_void_p]
_lib.sgf_plan_destroy.argtypes = [ctypes.c_void_p]
_lib.sgf_plan_profile.argtypes = [ctypes.c_void_p, ctypes.c_int32]
_lib.sgf_plan_profile_read.argtypes = [ctypes.c_void_p, ctypes.POINTER(KernelTimes)]
_lib.sgf_plan_estimate.argtypes = [ctypes.POINTER(NestDesc), ctypes.c_int, ctypes.c_uint32, _szp, _szp, _szp]
_lib.sgf_plan_create_forest.argtypes = [ctypes.POINTER(ForestDesc), ctypes.c_int, ctypes.c_uint32,
                                        ctypes.POINTER(ctypes.c_void_p)]
_lib.sgf_plan_estimate_forest.argtypes = [ctypes.POINTER(ForestDesc), ctypes.c_int, ctypes.c_uint32, _szp, _szp,
                                          _szp]
_lib.sgf_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(ctypes.c_void_p)]
_lib.sgf_server_clock.argtypes = [ctypes.c_void_p]
_lib.sgf_server_clock.restype = ctypes.c_double
_lib.sgf_server_submit.argtypes = [ctypes.c_void_p, ctypes.POINTER(Request)]
_lib.sgf_server_progress.argtypes = [ctypes.c_void_p, ctypes.POINTER(Completion), ctypes.c_int32,
                                     ctypes.POINTER(ctypes.c_int32)]
_lib.sgf_server_stats_get.argtypes = [ctypes.c_void_p, ctypes.POINTER(ServerStats)]
_lib.sgf_server_destroy.argtypes = [ctypes.c_void_p]
_lib.sgf_plan_schedule_get.argtypes = [ctypes.c_void_p, ctypes.POINTER(Schedule)]
_lib.sgf_plan_schedule_set.argtypes = [ctypes.c_void_p, ctypes.POINTER(Schedule)]
_lib.sgf_plan_autotune.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(Schedule),
                                   ctypes.POINTER(ctypes.c_double)]
_lib.sgf_last_error.restype = ctypes.c_char_p
_lib.sgf_version.restype = ctypes.c_char_p
for _f in ("sgf_plan_create", "sgf_plan_create_ex", "sgf_plan_check", "sgf_plan_share", "sgf_plan_stats_get", "sgf_solve", "sgf_solve_host",
           "sgf_solve_batched", "sgf_plan_destroy", "sgf_plan_profile", "sgf_plan_profile_read",
           "sgf_solve_noalloc", "sgf_batch_create", "sgf_batch_solve", "sgf_batch_info", "sgf_batch_destroy",
           "sgf_plan_estimate", "sgf_server_create", "sgf_server_submit", "sgf_server_progress",
           "sgf_server_stats_get", "sgf_server_destroy", "sgf_plan_schedule_get", "sgf_plan_schedule_set",
           "sgf_plan_autotune", "sgf_plan_share_ex", "sgf_solve_potential", "sgf_plan_create_forest",
           "sgf_plan_estimate_forest", "sgf_plan_footprint", "sgf_plan_inject_timeout", "sgf_solve_host_many"):
    getattr(_lib, _f).restype = ctypes.c_int


class SgfError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)}: {last_error()}")


def last_error() -> str:
    return _lib.sgf_last_error().decode()


def version() -> str:
    return _lib.sgf_version().decode()


def library_path() -> Path:
    return _LIB_PATH


def _check(status: int, what: str):
    if status != SGF_OK:
        raise SgfError(status, what)


def is_forest(geom) -> bool:
    """A forest (several patches per level) has per-patch ``level`` and ``org`` lists."""
    return hasattr(geom, "org") and hasattr(geom, "level")


def make_forest_desc(forest) -> ForestDesc:
    d = ForestDesc()
    K = len(forest.level)
    if K > SGF_MAX_PATCHES:
        raise ValueError(f"{K} patches, at most {SGF_MAX_PATCHES}")
    d.n, d.patches = int(forest.n), K
    d.x0, d.y0, d.h0 = float(forest.x0), float(forest.y0), float(forest.h0)
    for p in range(K):
        d.level[p] = int(forest.level[p])
        d.org[p][0], d.org[p][1] = int(forest.org[p][0]), int(forest.org[p][1])
    return d


def make_desc(nest) -> NestDesc:
    d = NestDesc()
    d.n, d.levels = int(nest.n), int(nest.levels)
    d.x0, d.y0, d.h0 = float(nest.x0), float(nest.y0), float(nest.h0)
    for l in range(1, min(int(nest.levels), SGF_MAX_LEVELS, len(nest.off))):
        d.off[l][0], d.off[l][1] = int(nest.off[l][0]), int(nest.off[l][1])
    return d


def _ptrs(ptrs: Sequence[int]):
    return (ctypes.c_void_p * len(ptrs))(*[ctypes.c_void_p(int(p)) for p in ptrs])


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


class Plan:
    """A solve plan: nest geometry + precision, resident kernel spectra, workspace."""

    def __init__(self, nest, precision="fp32", zero_rim: bool = False, potential: bool = False, _handle=None,
                 spectra_budget: int = 0):
        self.nest = nest
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.n, self.levels = int(nest.n), int(nest.levels)
        self.zero_rim = bool(zero_rim)
        self.potential = bool(potential)
        if _handle is not None:
            self._h = _handle
            return
        h = ctypes.c_void_p()
        flags = (PLAN_ZERO_RIM if zero_rim else 0) | (PLAN_POTENTIAL if potential else 0)
        if spectra_budget:  # sgf_plan_create: nests, force plans (spectra over the budget regenerated per solve)
            if is_forest(nest) or flags:
                raise ValueError("a spectra budget takes a nest force plan without options")
            _check(_lib.sgf_plan_create(ctypes.byref(make_desc(nest)), self.precision, int(spectra_budget),
                                        ctypes.byref(h)), "sgf_plan_create")
        elif is_forest(nest):  # per-patch arrays stand where a nest has per-level ones
            _check(_lib.sgf_plan_create_forest(ctypes.byref(make_forest_desc(nest)), self.precision, flags,
                                               ctypes.byref(h)), "sgf_plan_create_forest")
        else:
            _check(_lib.sgf_plan_create_ex(ctypes.byref(make_desc(nest)), self.precision, flags, ctypes.byref(h)),
                   "sgf_plan_create_ex")
        self._h = h

    def check(self):
        """Wait for the last solve and raise SgfError if the device recorded a violation."""
        _check(_lib.sgf_plan_check(self._h), "sgf_plan_check")

    def check_status(self) -> int:
        return int(_lib.sgf_plan_check(self._h))

    @property
    def handle(self):
        return self._h

    @property
    def dtype_name(self) -> str:
        return "float64" if self.precision == FP64 else "float32"

    def share(self, precision=None) -> "Plan":
        """A plan with its own workspace on these spectra (precision: this plan's, or
        fp32 / bf16x for each other)."""
        h = ctypes.c_void_p()
        if precision is None:
            _check(_lib.sgf_plan_share(self._h, ctypes.byref(h)), "sgf_plan_share")
            prec = self.precision
        else:
            prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
            _check(_lib.sgf_plan_share_ex(self._h, prec, ctypes.byref(h)), "sgf_plan_share_ex")
        return Plan(self.nest, prec, zero_rim=self.zero_rim, potential=self.potential, _handle=h)

    def stats(self) -> dict:
        st = PlanStats()
        _check(_lib.sgf_plan_stats_get(self._h, ctypes.byref(st)), "sgf_plan_stats_get")
        return {name: getattr(st, name) for name, _ in PlanStats._fields_}

    def inject_timeout(self, which: int, wait_cycles: int):
        """sgf_plan_inject_timeout (testing): the next solve withholds the producers of
        the waits in `which` and bounds every device wait by wait_cycles."""
        _check(_lib.sgf_plan_inject_timeout(self._h, int(which), int(wait_cycles)), "sgf_plan_inject_timeout")

    def footprint(self) -> dict:
        """sgf_plan_footprint: device bytes of the plan's workspace and of its spectra."""
        ws, sp = ctypes.c_size_t(), ctypes.c_size_t()
        _check(_lib.sgf_plan_footprint(self._h, ctypes.byref(ws), ctypes.byref(sp)), "sgf_plan_footprint")
        return {"workspace_bytes": ws.value, "spectra_bytes": sp.value}

    def solve_noalloc_ptrs(self, sigma_ptrs, fx_ptrs, fy_ptrs, stream=None):
        """sgf_solve_noalloc: the solve with the library's fixed scratch array (no allocation)."""
        _check(_lib.sgf_solve_noalloc(self._h, _ptrs(sigma_ptrs), _ptrs(fx_ptrs), _ptrs(fy_ptrs),
                                      ctypes.c_void_p(_stream_handle(stream))), "sgf_solve_noalloc")

    def schedule(self) -> dict:
        sc = Schedule()
        _check(_lib.sgf_plan_schedule_get(self._h, ctypes.byref(sc)), "sgf_plan_schedule_get")
        return {"col_pass": sc.col_pass, "row_inv0": sc.row_inv0, "col_case3": sc.col_case3,
                "col_radix": sc.col_radix, "inv_radix": sc.inv_radix, "row_fwd": sc.row_fwd}

    def set_schedule(self, col_pass: int = 0, row_inv0: int = 0, col_case3: int = 0, col_radix: int = 0,
                     inv_radix: int = 0, row_fwd: int = 0):
        sc = Schedule(int(col_pass), int(row_inv0), int(col_case3), int(col_radix), int(inv_radix), int(row_fwd))
        _check(_lib.sgf_plan_schedule_set(self._h, ctypes.byref(sc)), "sgf_plan_schedule_set")

    def autotune(self, reps: int = 5, stream=None) -> dict:
        """sgf_plan_autotune: time every schedule candidate, keep the fastest."""
        sc = Schedule()
        ms = (ctypes.c_double * AUTOTUNE_TIMES)()
        _check(_lib.sgf_plan_autotune(self._h, int(reps), ctypes.c_void_p(_stream_handle(stream)), ctypes.byref(sc),
                                      ms), "sgf_plan_autotune")
        return {"chosen": {"col_pass": sc.col_pass, "row_inv0": sc.row_inv0, "col_case3": sc.col_case3,
                           "col_radix": sc.col_radix, "inv_radix": sc.inv_radix, "row_fwd": sc.row_fwd},
                "ms": {"col_pass0": ms[0], "col_pass1": ms[1], "col_pass2": ms[2], "row_inv0_0": ms[3],
                       "row_inv0_1": ms[4], "row_inv0_2": ms[5], "col_case3_0": ms[6], "col_case3_1": ms[7],
                       "row_inv0_3": ms[8], "col_pass3": ms[9], "row_inv0_4": ms[10],
                       "col_pass3_radix1": ms[11], "row_inv0_4_radix1": ms[12], "row_fwd0": ms[13],
                       "row_fwd1": ms[14], "row_inv0_5": ms[15], "row_inv0_5_radix1": ms[16],
                       "row_fwd2": ms[17]}}

    def profile(self, enable: bool = True):
        _check(_lib.sgf_plan_profile(self._h, 1 if enable else 0), "sgf_plan_profile")

    def profile_read(self) -> dict:
        kt = KernelTimes()
        _check(_lib.sgf_plan_profile_read(self._h, ctypes.byref(kt)), "sgf_plan_profile_read")
        return {"solves": kt.solves,
                "kernels": {KERNELS[k]: {"launches": kt.launches[k], "ms": kt.ms[k]} for k in range(4)}}

    def solve_ptrs(self, sigma_ptrs, fx_ptrs, fy_ptrs, stream=None):
        _check(_lib.sgf_solve(self._h, _ptrs(sigma_ptrs), _ptrs(fx_ptrs), _ptrs(fy_ptrs),
                              ctypes.c_void_p(_stream_handle(stream))), "sgf_solve")

    def _device_levels(self, sigma):
        import torch
        sig = list(sigma)
        if len(sig) != self.levels:
            raise ValueError(f"need {self.levels} sigma levels")
        dt = torch.float64 if self.precision == FP64 else torch.float32
        for s in sig:
            if not (s.is_cuda and s.is_contiguous() and s.dtype == dt and tuple(s.shape) == (self.n, self.n)):
                raise ValueError(f"sigma levels must be contiguous CUDA {dt} tensors of shape ({self.n}, {self.n})")
        return sig

    def solve_potential_ptrs(self, sigma_ptrs, phi_ptrs, stream=None):
        _check(_lib.sgf_solve_potential(self._h, _ptrs(sigma_ptrs), _ptrs(phi_ptrs),
                                        ctypes.c_void_p(_stream_handle(stream))), "sgf_solve_potential")

    def solve_potential(self, sigma, phi=None, stream=None):
        """Potential plans: sigma as for solve(); returns the per-level potential list."""
        import torch
        sig = self._device_levels(sigma)
        if phi is None:
            phi = [torch.empty_like(s) for s in sig]
        self.solve_potential_ptrs([s.data_ptr() for s in sig], [t.data_ptr() for t in phi], stream)
        return phi

    def solve(self, sigma, fx=None, fy=None, stream=None):
        """sigma: list of per-level contiguous CUDA tensors (n, n). Returns (fx, fy) lists."""
        import torch
        sig = self._device_levels(sigma)
        if fx is None:
            fx = [torch.empty_like(s) for s in sig]
        if fy is None:
            fy = [torch.empty_like(s) for s in sig]
        self.solve_ptrs([s.data_ptr() for s in sig], [t.data_ptr() for t in fx], [t.data_ptr() for t in fy], stream)
        return fx, fy

    def solve_host(self, sigma: Sequence[np.ndarray], fx=None, fy=None, stream=None):
        """Host-buffer solve (copies inside the library; returns when done)."""
        dt = np.float64 if self.precision == FP64 else np.float32
        sig = [np.ascontiguousarray(s, dtype=dt) for s in sigma]
        if fx is None:
            fx = [np.empty((self.n, self.n), dtype=dt) for _ in range(self.levels)]
        if fy is None:
            fy = [np.empty((self.n, self.n), dtype=dt) for _ in range(self.levels)]
        sp = [a.ctypes.data for a in sig]
        xp = [a.ctypes.data for a in fx]
        yp = [a.ctypes.data for a in fy]
        self.solve_host_ptrs(sp, xp, yp, stream)
        return fx, fy

    def solve_host_ptrs(self, sigma_ptrs, fx_ptrs, fy_ptrs, stream=None):
        _check(_lib.sgf_solve_host(self._h, _ptrs(sigma_ptrs), _ptrs(fx_ptrs), _ptrs(fy_ptrs),
                                   ctypes.c_void_p(_stream_handle(stream))), "sgf_solve_host")

    def solve_host_many_ptrs(self, count, sigma_ptrs, fx_ptrs, fy_ptrs, stream=None):
        """sgf_solve_host_many: `count` problems in host memory, problem k's level l at
        index k * levels + l of each pointer list; copies overlap the transforms."""
        _check(_lib.sgf_solve_host_many(self._h, int(count), _ptrs(sigma_ptrs), _ptrs(fx_ptrs), _ptrs(fy_ptrs),
                                        ctypes.c_void_p(_stream_handle(stream))), "sgf_solve_host_many")

    def close(self):
        if getattr(self, "_h", None):
            _lib.sgf_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batched(plans: Sequence[Plan], sigma, fx, fy, stream=None):
    """plans[k] solves sigma[k] -> fx[k], fy[k] (per-level CUDA tensors) in one batched call."""
    n = len(plans)
    ph = (ctypes.c_void_p * n)(*[p.handle for p in plans])
    keep = []

    def table(lists):
        arrs = []
        for lst in lists:
            a = _ptrs([t.data_ptr() for t in lst])
            keep.append(a)
            arrs.append(ctypes.cast(a, _vpp))
        return (_vpp * n)(*arrs)

    _check(_lib.sgf_solve_batched(ph, n, table(sigma), table(fx), table(fy),
                                  ctypes.c_void_p(_stream_handle(stream))), "sgf_solve_batched")


def _ptr_table(lists, keep):
    arrs = []
    for lst in lists:
        a = _ptrs([t.data_ptr() if hasattr(t, "data_ptr") else int(t) for t in lst])
        keep.append(a)
        arrs.append(ctypes.cast(a, _vpp))
    return (_vpp * len(arrs))(*arrs)


class Batch:
    """Fused solve of many independent nests (sgf_batch_*): one launch per pass and
    per group of equal N, replayed as a CUDA graph."""

    def __init__(self, plans: Sequence[Plan], graph: bool = True):
        self.plans = list(plans)
        n = len(self.plans)
        ph = (ctypes.c_void_p * n)(*[p.handle for p in self.plans])
        h = ctypes.c_void_p()
        _check(_lib.sgf_batch_create(ph, n, 0 if graph else BATCH_NO_GRAPH, ctypes.byref(h)), "sgf_batch_create")
        self._h = h

    def info(self) -> dict:
        g, l = ctypes.c_int32(), ctypes.c_int32()
        _check(_lib.sgf_batch_info(self._h, ctypes.byref(g), ctypes.byref(l)), "sgf_batch_info")
        return {"groups": g.value, "launches_per_solve": l.value}

    def solve(self, sigma, fx, fy, stream=None):
        """sigma[k], fx[k], fy[k]: per-level CUDA tensors (or device pointers) of nest k."""
        keep = []
        _check(_lib.sgf_batch_solve(self._h, _ptr_table(sigma, keep), _ptr_table(fx, keep), _ptr_table(fy, keep),
                                    ctypes.c_void_p(_stream_handle(stream))), "sgf_batch_solve")

    def close(self):
        if getattr(self, "_h", None):
            _lib.sgf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def create_status(nest, precision, flags: int = 0) -> int:
    """Status of sgf_plan_create_ex without keeping the plan (validation probes)."""
    h = ctypes.c_void_p()
    desc = make_desc(nest)
    st = _lib.sgf_plan_create_ex(ctypes.byref(desc), PRECISIONS.get(precision, precision), flags, ctypes.byref(h))
    if st == SGF_OK:
        _lib.sgf_plan_destroy(h)
    return st


def estimate(nest, precision="fp32", flags: int = 0) -> dict:
    """sgf_plan_estimate: device bytes of a plan for this nest, without creating it (host only)."""
    ws, sp, bb = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    prec = PRECISIONS.get(precision, precision)
    if is_forest(nest):
        _check(_lib.sgf_plan_estimate_forest(ctypes.byref(make_forest_desc(nest)), prec, flags, ctypes.byref(ws),
                                             ctypes.byref(sp), ctypes.byref(bb)), "sgf_plan_estimate_forest")
    else:
        _check(_lib.sgf_plan_estimate(ctypes.byref(make_desc(nest)), prec, flags,
                                      ctypes.byref(ws), ctypes.byref(sp), ctypes.byref(bb)), "sgf_plan_estimate")
    return {"workspace_bytes": ws.value, "spectra_bytes": sp.value, "build_bytes": bb.value}


class Server:
    """The request loop (sgf_server_*): continuous admission of force requests with
    host buffers onto concurrent streams under an HBM budget.

    submit() queues a request; progress() collects finished ones and admits
    waiting ones; both return at once.  The numpy arrays of a request are kept
    referenced here until its completion has been returned.
    """

    def __init__(self, hbm_budget: int = 0, max_inflight: int = 4, simulate_gbs: Optional[float] = None,
                 max_shape_bytes: int = 0, autotune: bool = True, stream_large: bool = False):
        cfg = ServerConfig()
        cfg.hbm_budget = int(hbm_budget)
        cfg.max_shape_bytes = int(max_shape_bytes)
        cfg.max_inflight = int(max_inflight)
        cfg.flags = ((SERVER_SIMULATE if simulate_gbs is not None else 0) | (0 if autotune else SERVER_NO_AUTOTUNE) |
                     (SERVER_STREAM if stream_large else 0))
        cfg.simulate_gbs = float(simulate_gbs or 0.0)
        h = ctypes.c_void_p()
        _check(_lib.sgf_server_create(ctypes.byref(cfg), ctypes.byref(h)), "sgf_server_create")
        self._h = h
        self._held = {}
        self._buf = (Completion * 256)()

    def clock(self) -> float:
        return float(_lib.sgf_server_clock(self._h))

    def submit(self, rid: int, nest, precision, sigma, fx, fy, plan_flags: int = 0) -> int:
        """Queue request rid (sigma, fx, fy: per-level contiguous host arrays of the
        precision's dtype).  Returns the sgf status (SGF_ENOMEM: rejected)."""
        prec = PRECISIONS.get(precision, precision)
        dt = np.float64 if prec == FP64 else np.float32
        L = int(nest.levels)
        arrays = (list(sigma), list(fx), list(fy))
        for lst in arrays:
            if len(lst) != L:
                raise ValueError(f"need {L} arrays per field")
            for a in lst:
                if a.dtype != dt or not a.flags["C_CONTIGUOUS"] or a.shape != (nest.n, nest.n):
                    raise ValueError(f"request arrays must be C-contiguous {np.dtype(dt).name} ({nest.n}, {nest.n})")
        r = Request()
        r.id = int(rid)
        r.desc = make_desc(nest)
        r.precision = prec
        r.plan_flags = int(plan_flags)
        for l in range(L):
            r.sigma[l] = arrays[0][l].ctypes.data
            r.fx[l] = arrays[1][l].ctypes.data
            r.fy[l] = arrays[2][l].ctypes.data
        st = int(_lib.sgf_server_submit(self._h, ctypes.byref(r)))
        if st == SGF_OK:
            self._held[int(rid)] = arrays
        elif st != SGF_ENOMEM:
            raise SgfError(st, "sgf_server_submit")
        return st

    def progress(self) -> List[dict]:
        done = []
        while True:
            n = ctypes.c_int32()
            st = int(_lib.sgf_server_progress(self._h, self._buf, len(self._buf), ctypes.byref(n)))
            for k in range(n.value):
                c = self._buf[k]
                self._held.pop(int(c.id), None)
                done.append({"id": int(c.id), "status": int(c.status), "slot": int(c.slot),
                             "built_shape": bool(c.built_shape), "t_submit": c.t_submit, "t_admit": c.t_admit,
                             "t_done": c.t_done})
            _check(st, "sgf_server_progress")
            if n.value < len(self._buf):
                return done

    def stats(self) -> dict:
        st = ServerStats()
        _check(_lib.sgf_server_stats_get(self._h, ctypes.byref(st)), "sgf_server_stats_get")
        return {name: getattr(st, name) for name, _ in ServerStats._fields_ if name != "pad"}

    def close(self):
        if getattr(self, "_h", None):
            _lib.sgf_server_destroy(self._h)
            self._h = None
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
