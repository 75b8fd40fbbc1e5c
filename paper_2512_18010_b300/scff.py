"""Thin ctypes binding of the C ABI in include/scff.h.

Argument marshalling only: every step of the form-factor evaluation runs in
the CUDA library ``libscff.so``.  Device memory and streams may come from
PyTorch (CUDA tensors and ``torch.cuda.Stream``); host buffers are numpy
arrays.  If the library is missing the import of this module fails loudly;
there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np

from . import build as _build

FP64, FP32, BF16X3, TF32X3, BF16X2, FP16X2 = 0, 1, 2, 3, 4, 5
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16x3": BF16X3, "tf32x3": TF32X3, "bf16x2": BF16X2, "fp16x2": FP16X2}
# tensor-core W generator variants (scff_set_tc_variant modes, scff_last_path's third entry)
GEN_VARIANTS = {0: "gather", 1: "zstage", 2: "prefetch", 3: "pair", 4: "octant"}
RENORM_CONTRACTED = 1
PURE_D = 2   # d shells are the 5 real solid harmonics
PURE_F = 4   # f shells are the 7 real solid harmonics


def _basis_flags(mol, renorm: bool) -> int:
    return (RENORM_CONTRACTED if renorm else 0) | (int(getattr(mol, "pure", 0)) & (PURE_D | PURE_F))

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED_L", 3: "OOM", 4: "ADMISSION", 5: "CUDA",
          6: "TIMEOUT", 7: "CANCELLED", 8: "NOT_FOUND"}

_SYMBOLS = [
    "scff_create", "scff_destroy", "scff_last_error", "scff_basis", "scff_transitions",
    "scff_qgrid_product", "scff_qgrid_list", "scff_qgrid_size", "scff_form_factor", "scff_sync",
    "scff_kernel_launches", "scff_release_basis", "scff_release_transitions", "scff_release_qgrid",
    "scff_set_timing", "scff_last_timing", "scff_set_tc_drain", "scff_set_tc_variant", "scff_set_tc_zstage", "scff_last_path", "scff_form_factor_static",
    "scff_plan_create", "scff_plan_run", "scff_plan_run_graph", "scff_plan_info", "scff_release_plan",
    "scff_server_create", "scff_submit", "scff_wait", "scff_cancel", "scff_job_times", "scff_server_stats",
    "scff_server_destroy", "scff_set_autotune", "scff_autotune_choice", "scff_set_screening",
    "scff_screening_info", "scff_separable_integral", "scff_spherical", "scff_fft_form_factor", "scff_wait_selftest", "scff_set_hermitian",
    "scff_set_download_bands", "scff_alu_peak",
]


class _ServerOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("slots", ctypes.c_int), ("max_batch_jobs", ctypes.c_int),
                ("arena_bytes", ctypes.c_uint64), ("batch_cost_ratio", ctypes.c_double)]


class _Request(ctypes.Structure):
    _fields_ = [("basis", ctypes.c_void_p), ("trans", ctypes.c_void_p),
                ("qx", ctypes.c_void_p), ("nx", ctypes.c_int), ("qy", ctypes.c_void_p), ("ny", ctypes.c_int),
                ("qz", ctypes.c_void_p), ("nz", ctypes.c_int), ("scale", ctypes.c_double),
                ("f_out", ctypes.c_void_p), ("f2_out", ctypes.c_void_p), ("out_on_device", ctypes.c_int)]


class _SphGrid(ctypes.Structure):
    _fields_ = [("lmax", ctypes.c_int), ("n_q", ctypes.c_int), ("q", ctypes.c_void_p),
                ("n_theta", ctypes.c_int), ("theta", ctypes.c_void_p), ("n_phi", ctypes.c_int),
                ("phi", ctypes.c_void_p)]


class _FftGrid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("dq", ctypes.c_double * 3), ("centre", ctypes.c_double * 3),
                ("threshold", ctypes.c_double)]


class _Job(ctypes.Structure):
    _fields_ = [("basis", ctypes.c_void_p), ("trans", ctypes.c_void_p), ("grid", ctypes.c_void_p),
                ("scale", ctypes.c_double), ("f_out", ctypes.c_void_p), ("f2_out", ctypes.c_void_p)]


class ScffError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libscff.so (building it with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libscff.so not found at {_build.LIB}; build it with "
                          "`python -m paper_2512_18010_b300.build`")
    lib = ctypes.CDLL(_build.LIB)
    P, I32, I64, D, U32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_uint32
    lib.scff_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.c_uint64]
    lib.scff_destroy.argtypes = [P]
    lib.scff_destroy.restype = None
    lib.scff_last_error.restype = ctypes.c_char_p
    lib.scff_basis.argtypes = [P, ctypes.c_int, P, ctypes.c_int, P, P, P, P, P, U32, ctypes.POINTER(P),
                               ctypes.POINTER(I32)]
    lib.scff_transitions.argtypes = [P, P, ctypes.c_int, P, ctypes.c_int, ctypes.POINTER(P)]
    lib.scff_qgrid_product.argtypes = [P, P, ctypes.c_int, P, ctypes.c_int, P, ctypes.c_int, ctypes.POINTER(P)]
    lib.scff_qgrid_list.argtypes = [P, P, I64, ctypes.POINTER(P)]
    lib.scff_qgrid_size.argtypes = [P, P]
    lib.scff_qgrid_size.restype = I64
    lib.scff_form_factor.argtypes = [P, P, P, P, ctypes.c_int, D, P, P, ctypes.c_int, P]
    lib.scff_fft_form_factor.argtypes = [P, P, P, ctypes.POINTER(_FftGrid), ctypes.c_int, D, P, P, P, ctypes.c_int, P]
    lib.scff_wait_selftest.argtypes = [P, I64]
    lib.scff_spherical.argtypes = [P, P, P, ctypes.POINTER(_SphGrid), ctypes.c_int, D, P, P, P, P, ctypes.c_int, P]
    lib.scff_sync.argtypes = [P, P]
    lib.scff_form_factor_static.argtypes = [ctypes.c_int, P, ctypes.c_int, P, P, P, P, P, U32, ctypes.c_int, P,
                                            I64, P, D, P, P, P]
    lib.scff_form_factor_static.restype = I32
    lib.scff_plan_create.argtypes = [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(P)]
    lib.scff_plan_create.restype = I32
    lib.scff_plan_run.argtypes = [P, P, P]
    lib.scff_plan_run.restype = I32
    lib.scff_plan_run_graph.argtypes = [P, P, P]
    lib.scff_plan_run_graph.restype = I32
    lib.scff_plan_info.argtypes = [P, P, P]
    lib.scff_plan_info.restype = I32
    lib.scff_release_plan.argtypes = [P, P]
    lib.scff_release_plan.restype = None
    lib.scff_server_create.argtypes = [P, P, ctypes.POINTER(P)]
    lib.scff_submit.argtypes = [P, P, ctypes.POINTER(I64)]
    lib.scff_wait.argtypes = [P, I64, I64]
    lib.scff_cancel.argtypes = [P, I64]
    lib.scff_job_times.argtypes = [P, I64, P]
    lib.scff_server_stats.argtypes = [P, P]
    for n in ("scff_server_create", "scff_submit", "scff_wait", "scff_cancel", "scff_job_times",
              "scff_server_stats"):
        getattr(lib, n).restype = I32
    lib.scff_server_destroy.argtypes = [P]
    lib.scff_server_destroy.restype = None
    lib.scff_separable_integral.argtypes = [P, P, P, P, P, ctypes.c_int, P, P, ctypes.c_int, P, P, ctypes.c_int,
                                            D, P]
    lib.scff_separable_integral.restype = I32
    lib.scff_set_screening.argtypes = [P, D]
    lib.scff_set_screening.restype = I32
    lib.scff_screening_info.argtypes = [P, P, P, P]
    lib.scff_screening_info.restype = I32
    lib.scff_set_autotune.argtypes = [P, ctypes.c_int]
    lib.scff_set_autotune.restype = I32
    lib.scff_autotune_choice.argtypes = [P, P, P, P, ctypes.c_int, P]
    lib.scff_autotune_choice.restype = I32
    lib.scff_set_timing.argtypes = [P, ctypes.c_int]
    lib.scff_set_tc_drain.argtypes = [P, ctypes.c_int]
    for name in ("scff_set_tc_variant", "scff_set_tc_zstage"):
        getattr(lib, name).argtypes = [P, ctypes.c_int]
        getattr(lib, name).restype = I32
    lib.scff_last_path.argtypes = [P, P]
    lib.scff_last_path.restype = I32
    lib.scff_set_download_bands.argtypes = [P, ctypes.c_int]
    lib.scff_alu_peak.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P]
    lib.scff_alu_peak.restype = I32
    lib.scff_set_download_bands.restype = I32
    lib.scff_last_timing.argtypes = [P, P]
    lib.scff_kernel_launches.argtypes = [P]
    lib.scff_kernel_launches.restype = I64
    for n in ("scff_release_basis", "scff_release_transitions", "scff_release_qgrid"):
        getattr(lib, n).argtypes = [P, P]
        getattr(lib, n).restype = None
    for n in ("scff_create", "scff_basis", "scff_transitions", "scff_qgrid_product", "scff_qgrid_list",
              "scff_form_factor", "scff_sync", "scff_set_timing", "scff_last_timing", "scff_set_tc_drain"):
        getattr(lib, n).restype = I32
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        raise ScffError(rc, _lib.scff_last_error().decode())


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _is_torch_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


class Basis:
    def __init__(self, ctx: "Context", handle, nbf: int):
        self.ctx, self.handle, self.nbf = ctx, handle, nbf


class Transitions:
    def __init__(self, ctx, handle, n_states: int, basis: Basis):
        self.ctx, self.handle, self.n_states, self.basis = ctx, handle, n_states, basis


class QGrid:
    def __init__(self, ctx, handle, n: int, shape: Optional[Tuple[int, int, int]]):
        self.ctx, self.handle, self.n, self.shape = ctx, handle, n, shape


def _stream_ptr(stream):
    if stream is None:
        return ctypes.c_void_p(0)
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class Plan:
    """A fixed batch of jobs evaluated by persistent launches (see scff_plan_create)."""

    def __init__(self, ctx, handle, outputs):
        self.ctx, self.handle, self.outputs = ctx, handle, outputs

    def run(self, stream=None):
        _check(self.ctx.lib.scff_plan_run(self.ctx.h, self.handle, _stream_ptr(stream)))

    def run_graph(self, stream):
        _check(self.ctx.lib.scff_plan_run_graph(self.ctx.h, self.handle, _stream_ptr(stream)))

    def info(self) -> dict:
        out = np.zeros(6, dtype=np.int64)
        _check(self.ctx.lib.scff_plan_info(self.ctx.h, self.handle, _p(out)))
        keys = ("jobs", "tc_jobs", "groups", "tiles", "device_bytes", "launches_per_run")
        return {k: int(v) for k, v in zip(keys, out)}

    def release(self):
        if self.handle:
            self.ctx.lib.scff_release_plan(self.ctx.h, self.handle)
            self.handle = None


class Server:
    """Continuous-batching request loop (see scff_server_create)."""

    def __init__(self, ctx: "Context", precision=TF32X3, slots: int = 2, max_batch_jobs: int = 64,
                 arena_bytes: int = 0, batch_cost_ratio: float = 0.0):
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        self.ctx = ctx
        self.precision = precision
        opt = _ServerOptions(int(precision), int(slots), int(max_batch_jobs), int(arena_bytes),
                             float(batch_cost_ratio))
        h = ctypes.c_void_p()
        _check(ctx.lib.scff_server_create(ctx.h, ctypes.byref(opt), ctypes.byref(h)))
        self.h = h
        self._keep = {}

    def submit(self, basis: Basis, trans: Transitions, qx, qy, qz, f_out, f2_out=None, scale: float = 1.0) -> int:
        """Queues one job; f_out/f2_out are CUDA tensors (device outputs) or numpy/pinned arrays (host)."""
        qx, qy, qz = _np(qx, np.float64), _np(qy, np.float64), _np(qz, np.float64)
        dev = _is_torch_cuda(f_out)
        if dev:
            fp, f2p = f_out.data_ptr(), (f2_out.data_ptr() if f2_out is not None else None)
        elif hasattr(f_out, "data_ptr"):
            fp, f2p = f_out.data_ptr(), (f2_out.data_ptr() if f2_out is not None else None)
        else:
            fp = f_out.ctypes.data
            f2p = f2_out.ctypes.data if f2_out is not None else None
        req = _Request(basis.handle.value, trans.handle.value, qx.ctypes.data, len(qx), qy.ctypes.data, len(qy),
                       qz.ctypes.data, len(qz), float(scale), fp, f2p, 1 if dev else 0)
        jid = ctypes.c_int64()
        _check(self.ctx.lib.scff_submit(self.h, ctypes.byref(req), ctypes.byref(jid)))
        self._keep[jid.value] = (f_out, f2_out)
        return jid.value

    def wait(self, job_id: int, timeout_s: Optional[float] = None):
        t = -1 if timeout_s is None else int(timeout_s * 1e6)
        rc = self.ctx.lib.scff_wait(self.h, int(job_id), t)
        if rc == 0:
            self._keep.pop(job_id, None)
        _check(rc)

    def cancel(self, job_id: int):
        _check(self.ctx.lib.scff_cancel(self.h, int(job_id)))

    def times(self, job_id: int):
        """Host clock (ms) at submission, admission and completion."""
        out = np.zeros(3, dtype=np.float64)
        _check(self.ctx.lib.scff_job_times(self.h, int(job_id), _p(out)))
        return tuple(float(x) for x in out)

    def stats(self) -> dict:
        out = np.zeros(7, dtype=np.int64)
        _check(self.ctx.lib.scff_server_stats(self.h, _p(out)))
        keys = ("submitted", "completed", "cancelled", "failed", "batches", "max_inflight", "arena_bytes")
        return {k: int(v) for k, v in zip(keys, out)}

    def close(self):
        if self.h:
            self.ctx.lib.scff_server_destroy(self.h)
            self.h = None
            self._keep.clear()


class Context:
    """One library context on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.lib = load()
        h = ctypes.c_void_p()
        _check(self.lib.scff_create(ctypes.byref(h), int(device), int(hbm_budget_bytes)))
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            self.lib.scff_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- inputs ------------------------------------------------------------
    def basis(self, mol, renorm: bool = True) -> Basis:
        xyz = _np(mol.xyz, np.float64)
        sa, sl, sn = _np(mol.shell_atom, np.int32), _np(mol.shell_l, np.int32), _np(mol.shell_nprim, np.int32)
        ex, co = _np(mol.exponents, np.float64), _np(mol.coefficients, np.float64)
        h = ctypes.c_void_p()
        nbf = ctypes.c_int32()
        _check(self.lib.scff_basis(self.h, int(xyz.shape[0]), _p(xyz), int(sl.shape[0]), _p(sa), _p(sl), _p(sn),
                                   _p(ex), _p(co), _basis_flags(mol, renorm), ctypes.byref(h),
                                   ctypes.byref(nbf)))
        return Basis(self, h, nbf.value)

    def transitions(self, basis: Basis, T) -> Transitions:
        h = ctypes.c_void_p()
        if _is_torch_cuda(T):
            import torch
            T = T.to(torch.float64).contiguous()
            if T.dim() == 2:
                T = T.unsqueeze(0)
            S = int(T.shape[0])
            if tuple(T.shape[1:]) != (basis.nbf, basis.nbf):
                raise ValueError(f"T has shape {tuple(T.shape)}, basis has {basis.nbf} functions")
            _check(self.lib.scff_transitions(self.h, basis.handle, S, ctypes.c_void_p(T.data_ptr()), 1,
                                             ctypes.byref(h)))
        else:
            T = _np(T, np.float64)
            if T.ndim == 2:
                T = T[None]
            S = int(T.shape[0])
            if T.shape[1:] != (basis.nbf, basis.nbf):
                raise ValueError(f"T has shape {T.shape}, basis has {basis.nbf} functions")
            _check(self.lib.scff_transitions(self.h, basis.handle, S, _p(T), 0, ctypes.byref(h)))
        return Transitions(self, h, S, basis)

    def qgrid_product(self, qx, qy, qz) -> QGrid:
        qx, qy, qz = _np(qx, np.float64), _np(qy, np.float64), _np(qz, np.float64)
        h = ctypes.c_void_p()
        _check(self.lib.scff_qgrid_product(self.h, _p(qx), len(qx), _p(qy), len(qy), _p(qz), len(qz),
                                           ctypes.byref(h)))
        return QGrid(self, h, len(qx) * len(qy) * len(qz), (len(qx), len(qy), len(qz)))

    def qgrid_list(self, q) -> QGrid:
        q = _np(q, np.float64).reshape(-1, 3)
        h = ctypes.c_void_p()
        _check(self.lib.scff_qgrid_list(self.h, _p(q), int(q.shape[0]), ctypes.byref(h)))
        return QGrid(self, h, int(q.shape[0]), None)

    def release(self, obj):
        if isinstance(obj, Basis):
            self.lib.scff_release_basis(self.h, obj.handle)
        elif isinstance(obj, Transitions):
            self.lib.scff_release_transitions(self.h, obj.handle)
        elif isinstance(obj, QGrid):
            self.lib.scff_release_qgrid(self.h, obj.handle)

    # -- evaluation --------------------------------------------------------
    def form_factor(self, basis: Basis, trans: Transitions, grid: QGrid, precision=FP32, scale: float = 1.0,
                    f_out=None, f2_out=None, with_f2: bool = True, stream=None):
        """Evaluates f_s(q) (and |f_s(q)|^2).

        With torch CUDA tensors as outputs (or ``f_out="cuda"``) the call is
        asynchronous on ``stream`` (default: torch's current stream) and
        returns the tensors; otherwise it returns numpy arrays
        f[S, nq] (complex) and f2[S, nq].
        """
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        S, nq = trans.n_states, grid.n
        rdt = np.float64 if precision == FP64 else np.float32
        if isinstance(f_out, str) and f_out == "cuda":
            import torch
            tdt = torch.float64 if precision == FP64 else torch.float32
            dev = torch.device("cuda", self.device)
            f_out = torch.empty((S, nq, 2), dtype=tdt, device=dev)
            f2_out = torch.empty((S, nq), dtype=tdt, device=dev) if with_f2 else None
        if f_out is not None and _is_torch_cuda(f_out):
            import torch
            if stream is None:
                stream = torch.cuda.current_stream(f_out.device)
            sp = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
            _check(self.lib.scff_form_factor(self.h, basis.handle, trans.handle, grid.handle, int(precision),
                                             float(scale), ctypes.c_void_p(f_out.data_ptr()),
                                             ctypes.c_void_p(f2_out.data_ptr()) if f2_out is not None else None,
                                             1, sp))
            return f_out, f2_out
        caller_buffers = f_out is not None
        f = np.empty((S, nq, 2), dtype=rdt) if f_out is None else f_out
        f2 = (np.empty((S, nq), dtype=rdt) if with_f2 else None) if f2_out is None else f2_out
        if f.dtype != rdt or f.shape != (S, nq, 2) or not f.flags.c_contiguous:
            raise ValueError(f"f_out must be a C-contiguous {np.dtype(rdt).name} array of shape {(S, nq, 2)}")
        if f2 is not None and (f2.dtype != rdt or f2.shape != (S, nq) or not f2.flags.c_contiguous):
            raise ValueError(f"f2_out must be a C-contiguous {np.dtype(rdt).name} array of shape {(S, nq)}")
        sp = ctypes.c_void_p(0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream")
                                                       else int(stream)))
        _check(self.lib.scff_form_factor(self.h, basis.handle, trans.handle, grid.handle, int(precision),
                                         float(scale), _p(f), _p(f2) if f2 is not None else None, 0, sp))
        if caller_buffers:
            return f, f2
        return f[..., 0] + 1j * f[..., 1], f2

    def plan(self, jobs, precision=TF32X3, workspace_bytes: int = 0) -> Plan:
        """jobs: list of (basis, transitions, grid, f_out, f2_out_or_None, scale) with CUDA tensor outputs
        (f_out [S, nq, 2], f2_out [S, nq]; float64 for FP64, float32 otherwise)."""
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        arr = (_Job * len(jobs))()
        for i, (b, t, g, f, f2, sc) in enumerate(jobs):
            if not _is_torch_cuda(f) or not f.is_contiguous() or tuple(f.shape) != (t.n_states, g.n, 2):
                raise ValueError(f"job {i}: f_out must be a contiguous CUDA tensor of shape {(t.n_states, g.n, 2)}")
            arr[i] = _Job(b.handle.value, t.handle.value, g.handle.value, float(sc), f.data_ptr(),
                          f2.data_ptr() if f2 is not None else None)
        h = ctypes.c_void_p()
        _check(self.lib.scff_plan_create(self.h, len(jobs), ctypes.cast(arr, ctypes.c_void_p), int(precision),
                                         int(workspace_bytes), ctypes.byref(h)))
        return Plan(self, h, [(j[3], j[4]) for j in jobs])

    def sync(self, stream=None):
        sp = ctypes.c_void_p(0 if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream")
                                                       else int(stream)))
        _check(self.lib.scff_sync(self.h, sp))

    def set_tc_drain(self, drain_every: int):
        """k-chunks per tensor-core TMEM accumulation (0 = whole K, -1 = default)."""
        _check(self.lib.scff_set_tc_drain(self.h, int(drain_every)))

    def last_path(self) -> dict:
        """The path the last form-factor call ran: direct FP64/FP32 or tensor cores, the precision of its
        arithmetic, and the tensor-core W generator variant that ran (a GEN_VARIANTS name; None
        off the tensor cores)."""
        out = np.zeros(3, dtype=np.int32)
        _check(self.lib.scff_last_path(self.h, _p(out)))
        names = {v: k for k, v in PRECISIONS.items()}
        path = {0: "direct_fp64", 1: "direct_fp32", 2: "tensor_cores"}.get(int(out[0]))
        return {"path": path, "precision": names.get(int(out[1])),
                "variant": GEN_VARIANTS.get(int(out[2])) if path == "tensor_cores" else None}

    def set_tc_variant(self, mode: int):
        """Tensor-core launch shape and W generator variant: -1 automatic, 0 gather from global memory,
        1 stage Z and Y in shared memory where the grid allows it, 2 prefetch the next chunk's table
        entries with the running sums in TMEM, 3 CTA pairs (two SMs share each 256-row MMA and each
        generates half of W), 4 the octant form on antisymmetric grids (real W, half the tensor work:
        CTA pairs for FP16 hi/lo and BF16 hi/lo, single CTAs for BF16 hi/mid/lo; elsewhere 3 or 0);
        2 and 3 where the split allows them (FP16 hi/lo, BF16 hi/lo).  0 to 3 give bitwise the same
        results; 4 rounds differently within the same bar (GEN_VARIANTS names them)."""
        _check(self.lib.scff_set_tc_variant(self.h, int(mode)))

    def set_tc_zstage(self, mode: int):
        """The same as set_tc_variant (its earlier name)."""
        _check(self.lib.scff_set_tc_zstage(self.h, int(mode)))

    def separable_integral(self, basis: Basis, trans: Transitions, qx, wx, qy, wy, qz, wz,
                           scale: float = 1.0) -> np.ndarray:
        """I_s = scale * sum wx(qx) wy(qy) wz(qz) f_s(q) over the product grid, as complex [S]."""
        arrs = [_np(a, np.float64) for a in (qx, wx, qy, wy, qz, wz)]
        if len(arrs[0]) != len(arrs[1]) or len(arrs[2]) != len(arrs[3]) or len(arrs[4]) != len(arrs[5]):
            raise ValueError("each axis needs as many weights as points")
        out = np.zeros((trans.n_states, 2), dtype=np.float64)
        _check(self.lib.scff_separable_integral(self.h, basis.handle, trans.handle, _p(arrs[0]), _p(arrs[1]),
                                                len(arrs[0]), _p(arrs[2]), _p(arrs[3]), len(arrs[2]), _p(arrs[4]),
                                                _p(arrs[5]), len(arrs[4]), float(scale), _p(out)))
        return out[:, 0] + 1j * out[:, 1]

    def spherical(self, basis: Basis, trans: Transitions, q, lmax: int, theta=None, phi=None,
                  precision=FP64, scale: float = 1.0, want=("R", "f", "f2", "iso"), out: str = "host",
                  stream=None) -> dict:
        """Spherical method: R_lm(q), and on an angular grid f and |f|^2, and the isotropic average.

        Returns "R" complex [S, n_q, (lmax+1)^2], "f" complex [S, n_q, n_theta,
        n_phi], "f2" [S, n_q, n_theta, n_phi], "iso" [S, n_q] (those in
        `want`; f and f2 only with an angular grid): numpy arrays, or with
        out="cuda" the raw torch tensors written on the device (complex
        values as a trailing axis of 2).
        """
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        q = _np(q, np.float64)
        th = _np(theta if theta is not None else np.zeros(0), np.float64)
        ph = _np(phi if phi is not None else np.zeros(0), np.float64)
        S, nq, nt, npf = trans.n_states, len(q), len(th), len(ph)
        NR = (lmax + 1) ** 2
        angular = nt > 0 and npf > 0
        shapes = {"R": (S, nq, NR, 2), "f": (S, nq, nt, npf, 2), "f2": (S, nq, nt, npf), "iso": (S, nq)}
        keys = [k for k in ("R", "f", "f2", "iso") if k in want and (angular or k in ("R", "iso"))]
        g = _SphGrid(int(lmax), nq, _p(q), nt, _p(th) if nt else None, npf, _p(ph) if npf else None)
        if out == "cuda":
            import torch
            tdt = torch.float64 if precision == FP64 else torch.float32
            bufs = {k: torch.empty(shapes[k], dtype=tdt, device="cuda") for k in keys}
            ptr = lambda k: ctypes.c_void_p(bufs[k].data_ptr()) if k in bufs else None  # noqa: E731
            if stream is None:
                stream = torch.cuda.current_stream()
            sp = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
            _check(self.lib.scff_spherical(self.h, basis.handle, trans.handle, ctypes.byref(g), int(precision),
                                           float(scale), ptr("R"), ptr("f"), ptr("f2"), ptr("iso"), 1, sp))
            return bufs
        rdt = np.float64 if precision == FP64 else np.float32
        arrs = {k: np.zeros(shapes[k], rdt) for k in keys}
        ptr = lambda k: _p(arrs[k]) if k in arrs else None  # noqa: E731
        _check(self.lib.scff_spherical(self.h, basis.handle, trans.handle, ctypes.byref(g), int(precision),
                                       float(scale), ptr("R"), ptr("f"), ptr("f2"), ptr("iso"), 0, None))
        R, f, f2, iso = (arrs.get(k) for k in ("R", "f", "f2", "iso"))
        out = {}
        if R is not None:
            out["R"] = R[..., 0] + 1j * R[..., 1]
        if f is not None:
            out["f"] = f[..., 0] + 1j * f[..., 1]
        if f2 is not None:
            out["f2"] = f2
        if iso is not None:
            out["iso"] = iso
        return out

    def fft_form_factor(self, basis: Basis, trans: Transitions, n, dq, centre=(0.0, 0.0, 0.0),
                        threshold: float = 0.0, precision=FP32, scale: float = 1.0, want=("f", "f2"),
                        out: str = "host", stream=None) -> dict:
        """FFT method on a box of n[i] points, side 2 pi / dq[i], centred at `centre`.

        Returns "f" complex [S, n0, n1, n2] at q = dq (index - n/2), "f2", and
        "parseval" [S, 2] = (sum |Phi|^2 V_pix, sum |f|^2 dq^3 / (2 pi)^3); with
        out="cuda", f and f2 are torch tensors on the device (complex as a
        trailing axis of 2).
        """
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        if np.isscalar(n):
            n = (n, n, n)
        if np.isscalar(dq):
            dq = (dq, dq, dq)
        g = _FftGrid((ctypes.c_int * 3)(*[int(v) for v in n]), (ctypes.c_double * 3)(*[float(v) for v in dq]),
                     (ctypes.c_double * 3)(*[float(v) for v in centre]), float(threshold))
        S = trans.n_states
        shp = (S, int(n[0]), int(n[1]), int(n[2]))
        par = np.zeros((S, 2), np.float64)
        if out == "cuda":
            import torch
            tdt = torch.float64 if precision == FP64 else torch.float32
            bufs = {}
            if "f" in want:
                bufs["f"] = torch.empty(shp + (2,), dtype=tdt, device="cuda")
            if "f2" in want:
                bufs["f2"] = torch.empty(shp, dtype=tdt, device="cuda")
            if stream is None:
                stream = torch.cuda.current_stream()
            sp = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
            ptr = lambda k: ctypes.c_void_p(bufs[k].data_ptr()) if k in bufs else None  # noqa: E731
            _check(self.lib.scff_fft_form_factor(self.h, basis.handle, trans.handle, ctypes.byref(g), int(precision),
                                                 float(scale), ptr("f"), ptr("f2"), _p(par), 1, sp))
            bufs["parseval"] = par
            return bufs
        rdt = np.float64 if precision == FP64 else np.float32
        f = np.zeros(shp + (2,), rdt) if "f" in want else None
        f2 = np.zeros(shp, rdt) if "f2" in want else None
        _check(self.lib.scff_fft_form_factor(self.h, basis.handle, trans.handle, ctypes.byref(g), int(precision),
                                             float(scale), None if f is None else _p(f),
                                             None if f2 is None else _p(f2), _p(par), 0, None))
        res = {"parseval": par}
        if f is not None:
            res["f"] = f[..., 0] + 1j * f[..., 1]
        if f2 is not None:
            res["f2"] = f2
        return res

    def set_hermitian(self, enable: bool = True):
        """Evaluate half of an antisymmetric product grid and mirror f(-q) = conj(f(q)) (default on)."""
        _check(self.lib.scff_set_hermitian(self.h, 1 if enable else 0))

    def set_download_bands(self, n_bands: int = 0):
        """Host-output calls on the tensor cores: launches over column bands whose
        downloads overlap the next band's compute (0 = automatic, 1 = off, 2..8)."""
        _check(self.lib.scff_set_download_bands(self.h, int(n_bands)))

    def alu_peak(self, fp64: bool = False, iters: int = 65536, packed: bool = False):
        """Measured FMA-chain rate of this device: (TFLOP/s, ms of the timed launch).  FP64, FP32, or with
        packed=True FP32 on packed f32x2 pairs."""
        t = np.zeros(1, dtype=np.float64)
        m = np.zeros(1, dtype=np.float64)
        mode = 1 if fp64 else (2 if packed else 0)
        _check(self.lib.scff_alu_peak(self.h, mode, int(iters), _p(t), _p(m)))
        return float(t[0]), float(m[0])

    def wait_selftest(self, tries: int = 4096):
        """Runs the bounded-wait failure path once; raises ScffError(TIMEOUT) as intended."""
        _check(self.lib.scff_wait_selftest(self.h, int(tries)))

    def set_screening(self, eps: float):
        """Error-bounded pair screening: results within eps * max|f| of the exact ones (0 = off)."""
        _check(self.lib.scff_set_screening(self.h, float(eps)))

    def screening_info(self, trans: Transitions, grid: QGrid) -> dict:
        out = np.zeros(4, dtype=np.int64)
        _check(self.lib.scff_screening_info(self.h, trans.handle, grid.handle, _p(out)))
        return {"kept_pairs": int(out[0]), "pairs": int(out[1]), "kept_rows": int(out[2]), "rows": int(out[3])}

    def set_autotune(self, enable: bool = True):
        _check(self.lib.scff_set_autotune(self.h, 1 if enable else 0))

    def autotune_choice(self, basis: Basis, trans: Transitions, grid: QGrid, precision=TF32X3) -> dict:
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        out = np.zeros(5, dtype=np.int32)
        _check(self.lib.scff_autotune_choice(self.h, basis.handle, trans.handle, grid.handle, int(precision),
                                             _p(out)))
        return {"tensor_cores": bool(out[0]), "drain": int(out[1]), "state_block": int(out[2]),
                "best_us": int(out[3]), "zstage": int(out[4]), "variant": GEN_VARIANTS.get(int(out[4]))}

    def set_timing(self, enable: bool = True):
        _check(self.lib.scff_set_timing(self.h, 1 if enable else 0))

    def last_timing(self):
        """(q-evaluation ms, pair-prep + tables ms, total device ms) of the last call."""
        out = np.zeros(3, dtype=np.float64)
        _check(self.lib.scff_last_timing(self.h, _p(out)))
        return float(out[0]), float(out[1]), float(out[2])

    def kernel_launches(self) -> int:
        return int(self.lib.scff_kernel_launches(self.h))


def form_factor_static(mol, T_dev, q_dev, f_dev, f2_dev=None, scale: float = 1.0, renorm: bool = True,
                       stream=None):
    """FP64 form factor on an explicit q list without any device allocation.

    For callers that cannot allocate device memory themselves at run time
    (for example inside a framework whose caching allocator owns the device
    memory, or a serving loop that must not synchronise on cudaMalloc): T_dev
    [S, nbf, nbf], q_dev [n, 3], f_dev [S, n, 2] and f2_dev [S, n] are the
    caller's float64 CUDA tensors; the library's intermediates live in a fixed
    device array of its own.  Limits and sharing rules are in include/scff.h
    (scff_form_factor_static).  Blocks until the work on `stream` is done.
    """
    lib = load()
    import torch
    for name, t in (("T_dev", T_dev), ("q_dev", q_dev), ("f_dev", f_dev)):
        if not _is_torch_cuda(t) or t.dtype != torch.float64 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    S = int(T_dev.shape[0])
    n = int(q_dev.shape[0])
    if tuple(f_dev.shape) != (S, n, 2) or (f2_dev is not None and tuple(f2_dev.shape) != (S, n)):
        raise ValueError("output shapes must be [S, n, 2] and [S, n]")
    xyz = _np(mol.xyz, np.float64)
    sa, sl, sn = _np(mol.shell_atom, np.int32), _np(mol.shell_l, np.int32), _np(mol.shell_nprim, np.int32)
    ex, co = _np(mol.exponents, np.float64), _np(mol.coefficients, np.float64)
    if stream is None:
        stream = torch.cuda.current_stream(f_dev.device)
    sp = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    rc = lib.scff_form_factor_static(int(xyz.shape[0]), _p(xyz), int(sl.shape[0]), _p(sa), _p(sl), _p(sn), _p(ex),
                                     _p(co), _basis_flags(mol, renorm), S,
                                     ctypes.c_void_p(T_dev.data_ptr()), n, ctypes.c_void_p(q_dev.data_ptr()),
                                     float(scale), ctypes.c_void_p(f_dev.data_ptr()),
                                     ctypes.c_void_p(f2_dev.data_ptr()) if f2_dev is not None else None, sp)
    _check(rc)
    return f_dev, f2_dev


def evaluate_job(ctx: Context, job, precision=FP32, scale: float = 1.0, q_list=None):
    """Convenience: basis + transitions + grid of a workload job -> host f, f2."""
    b = ctx.basis(job.mol)
    t = ctx.transitions(b, job.T)
    g = ctx.qgrid_list(q_list) if q_list is not None else ctx.qgrid_product(job.qx, job.qy, job.qz)
    try:
        return ctx.form_factor(b, t, g, precision=precision, scale=scale)
    finally:
        ctx.release(g)
        ctx.release(b)
