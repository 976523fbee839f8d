"""Dual-select FMA radix-2 FFT for B300 — Python binding of ``libdsfft.so``.

Argument marshalling only: every step of a transform (table build, passes)
runs in the library's CUDA kernels.  PyTorch supplies device memory and the
current stream.  If the shared library is missing the import of the library
handle fails loudly — there is no CPU fallback.

    import paper_2604_00567_b300 as dsfft
    plan = dsfft.Plan(1024, "fp16", "dual_select")
    y = plan.exec(x)                  # x: (batch, 1024, 2) float16 on cuda

Storage layouts (interleaved re/im):
    fp32 : complex64 tensor (..., N)
    fp16 : float16 tensor  (..., N, 2)
    bf16 : bfloat16 tensor (..., N, 2)
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = ["Plan", "Batch", "lib", "twiddle_fp64", "DsfftError", "PRECISIONS", "FACTORIZATIONS",
           "FORWARD", "INVERSE"]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdsfft.so")

PRECISIONS = {"fp32": 0, "fp16": 1, "bf16": 2}
FACTORIZATIONS = {"linzer_feig_clamped": 0, "cosine": 1, "dual_select": 2}
FORWARD, INVERSE = -1, 1
STATUS = {0: "FFT_OK", 1: "FFT_ERR_INVALID_ARG", 2: "FFT_ERR_INVALID_SIZE", 3: "FFT_ERR_UNSUPPORTED",
          4: "FFT_ERR_OOM", 5: "FFT_ERR_CUDA", 6: "FFT_ERR_TIMEOUT"}


class DsfftError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


VARIANTS = {"auto": 0, "fused_wide": 1, "fused_narrow": 2, "cluster": 3, "sweeps": 4, "fused_tma": 5}
VARIANT_NAMES = {v: k for k, v in VARIANTS.items()}


class PlanOpts(ctypes.Structure):
    _fields_ = [("lf_eps", ctypes.c_double), ("scale_forward", ctypes.c_int32),
                ("scale_inverse", ctypes.c_int32), ("device", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("radix", ctypes.c_int32), ("sweep_passes", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("log2n", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("factorization", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("launches", ctypes.c_int32), ("points_per_thread", ctypes.c_int32),
                ("threads_per_transform", ctypes.c_int32), ("transforms_per_block", ctypes.c_int32),
                ("table_bytes", ctypes.c_int64), ("element_bytes", ctypes.c_int64),
                ("scale_forward", ctypes.c_int32), ("scale_inverse", ctypes.c_int32),
                ("cos_count", ctypes.c_int32), ("sin_count", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("autotuned", ctypes.c_int32), ("radix", ctypes.c_int32),
                ("sweep_passes", ctypes.c_int32)]


class BatchItemC(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("precision", ctypes.c_int32), ("factorization", ctypes.c_int32),
                ("direction", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class NoAllocItemC(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("direction", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p)]


NOALLOC_MAX_ITEMS = 4096


class BatchInfo(ctypes.Structure):
    _fields_ = [("items", ctypes.c_int64), ("plans", ctypes.c_int32), ("tiles", ctypes.c_int32),
                ("persistent_blocks", ctypes.c_int32), ("large_groups", ctypes.c_int32),
                ("launches", ctypes.c_int32), ("graph_ready", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64)]


class ServerOptsC(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_ticks_in_flight", ctypes.c_int32),
                ("memory_budget", ctypes.c_uint64), ("max_tick_transforms", ctypes.c_int64),
                ("autotune", ctypes.c_int32), ("release_on_complete", ctypes.c_int32),
                ("max_tick_bytes", ctypes.c_int64), ("reserved", ctypes.c_int32 * 2)]


class RequestC(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("precision", ctypes.c_int32), ("factorization", ctypes.c_int32),
                ("direction", ctypes.c_int32), ("reserved", ctypes.c_int32), ("count", ctypes.c_int64),
                ("in_", ctypes.c_void_p), ("tag", ctypes.c_uint64)]


class CompletionC(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("tag", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("out", ctypes.c_void_p), ("bytes", ctypes.c_int64),
                ("t_submit_ns", ctypes.c_int64), ("t_admit_ns", ctypes.c_int64),
                ("t_launch_ns", ctypes.c_int64), ("t_done_ns", ctypes.c_int64), ("tick", ctypes.c_int64)]


class ServerStatsC(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("released", ctypes.c_int64), ("queued", ctypes.c_int64), ("in_flight", ctypes.c_int64),
                ("ticks", ctypes.c_int64), ("transforms", ctypes.c_int64), ("plans", ctypes.c_int64),
                ("arena_bytes", ctypes.c_uint64), ("arena_used", ctypes.c_uint64),
                ("arena_peak", ctypes.c_uint64), ("reserved", ctypes.c_int64 * 4)]


_lib = None
_lock = threading.Lock()


def lib():
    """Load ``libdsfft.so`` (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libdsfft.so not found at {LIB_PATH}; build it with "
                                   "`python -m paper_2604_00567_b300.build`")
            L = ctypes.CDLL(LIB_PATH)
            P, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            L.fft_plan_opts_init.argtypes = [i32, ctypes.POINTER(PlanOpts)]
            L.fft_plan_create.argtypes = [ctypes.POINTER(P), i64, i32, i32, ctypes.POINTER(PlanOpts)]
            L.fft_plan_destroy.argtypes = [P]
            L.fft_exec.argtypes = [P, P, P, i64, i32, P]
            L.fft_plan_get_table.argtypes = [P, i32, P, ctypes.c_size_t]
            L.fft_plan_get_table4.argtypes = [P, i32, P, ctypes.c_size_t]
            L.fft_plan_get_info.argtypes = [P, ctypes.POINTER(PlanInfo)]
            L.fft_plan_device_status.argtypes = [P]
            L.fft_twiddle_fp64.argtypes = [i64, i32, d, P, P, P]
            L.fft_status_string.restype = ctypes.c_char_p
            L.fft_status_string.argtypes = [i32]
            L.fft_last_error_string.restype = ctypes.c_char_p
            L.fft_last_error_string.argtypes = []
            L.fft_batch_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(BatchItemC), i64,
                                           ctypes.POINTER(PlanOpts)]
            L.fft_batch_exec.argtypes = [P, P]
            L.fft_batch_exec_graph.argtypes = [P, P]
            L.fft_batch_get_info.argtypes = [P, ctypes.POINTER(BatchInfo)]
            L.fft_batch_destroy.argtypes = [P]
            L.fft_exec_batch_noalloc.argtypes = [ctypes.POINTER(NoAllocItemC), i64, P]
            L.fft_pipeline_create.argtypes = [ctypes.POINTER(P), P, i64, i32]
            L.fft_pipeline_exec.argtypes = [P, P, P, i64, i32, P]
            L.fft_pipeline_destroy.argtypes = [P]
            u64 = ctypes.c_uint64
            L.fft_server_opts_init.argtypes = [ctypes.POINTER(ServerOptsC)]
            L.fft_server_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(ServerOptsC)]
            L.fft_server_prepare.argtypes = [P, i64, i32, i32]
            L.fft_server_submit.argtypes = [P, ctypes.POINTER(RequestC), ctypes.POINTER(u64)]
            L.fft_server_replay.argtypes = [P, ctypes.POINTER(RequestC), ctypes.POINTER(i64), i64,
                                            ctypes.POINTER(u64)]
            L.fft_server_poll.argtypes = [P, ctypes.POINTER(CompletionC), i64, ctypes.POINTER(i64)]
            L.fft_server_wait.argtypes = [P, u64, d, ctypes.POINTER(CompletionC)]
            L.fft_server_copy_out.argtypes = [P, u64, P, i64, P]
            L.fft_server_release.argtypes = [P, u64]
            L.fft_server_drain.argtypes = [P, d]
            L.fft_server_get_stats.argtypes = [P, ctypes.POINTER(ServerStatsC)]
            L.fft_server_destroy.argtypes = [P]
            for name in ("fft_plan_opts_init", "fft_plan_create", "fft_plan_destroy", "fft_exec",
                         "fft_plan_get_table", "fft_plan_get_table4", "fft_plan_get_info", "fft_plan_device_status",
                         "fft_twiddle_fp64", "fft_batch_create",
                         "fft_batch_exec", "fft_batch_exec_graph", "fft_batch_get_info", "fft_batch_destroy",
                         "fft_exec_batch_noalloc", "fft_pipeline_create", "fft_pipeline_exec",
                         "fft_pipeline_destroy", "fft_server_opts_init", "fft_server_create",
                         "fft_server_prepare", "fft_server_submit", "fft_server_replay", "fft_server_poll",
                         "fft_server_wait", "fft_server_copy_out", "fft_server_release", "fft_server_drain",
                         "fft_server_get_stats", "fft_server_destroy"):
                getattr(L, name).restype = i32
            _lib = L
    return _lib


def _check(status: int, where: str):
    if status != 0:
        raise DsfftError(status, where, lib().fft_last_error_string().decode())


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """A resident FFT plan: length ``n``, precision and factorization."""

    def __init__(self, n: int, precision: str = "fp32", factorization: str = "dual_select",
                 lf_eps: float = 1e-7, scale_forward: bool | None = None,
                 scale_inverse: bool | None = None, device: int | None = None,
                 variant: str = "auto", autotune: bool = False, radix: int = 2, sweep_passes: int = 0):
        L = lib()
        self.n = int(n)
        self.precision = precision
        self.factorization = factorization
        opts = PlanOpts()
        _check(L.fft_plan_opts_init(PRECISIONS[precision], ctypes.byref(opts)), "fft_plan_opts_init")
        opts.lf_eps = float(lf_eps)
        if scale_forward is not None:
            opts.scale_forward = 1 if scale_forward else 0
        if scale_inverse is not None:
            opts.scale_inverse = 1 if scale_inverse else 0
        if device is not None:
            opts.device = int(device)
        opts.variant = VARIANTS[variant]
        opts.autotune = 1 if autotune else 0
        opts.radix = int(radix)
        opts.sweep_passes = int(sweep_passes)
        self.radix = int(radix)
        self.scale_forward = bool(opts.scale_forward)
        self.scale_inverse = bool(opts.scale_inverse)
        h = ctypes.c_void_p()
        _check(L.fft_plan_create(ctypes.byref(h), self.n, PRECISIONS[precision],
                                 FACTORIZATIONS[factorization], ctypes.byref(opts)),
               f"fft_plan_create(N={n}, {precision}, {factorization})")
        self._h = h

    # ------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().fft_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def info(self) -> dict:
        inf = PlanInfo()
        _check(lib().fft_plan_get_info(self._h, ctypes.byref(inf)), "fft_plan_get_info")
        d = {k: getattr(inf, k) for k, _ in PlanInfo._fields_}
        d["variant_name"] = VARIANT_NAMES.get(d["variant"], "?")
        return d

    def device_status(self) -> None:
        """Raise DsfftError (FFT_ERR_TIMEOUT) if a bounded device-side wait
        of this plan's kernels gave up since the last call; clears the word."""
        _check(lib().fft_plan_device_status(self._h), "fft_plan_device_status")

    def element_bytes(self) -> int:
        return 8 if self.precision == "fp32" else 4

    def _check_tensor_shape(self, x):
        """Signals in a contiguous tensor of the plan's layout (any device)."""
        import torch
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if self.precision == "fp32":
            if x.dtype != torch.complex64 or x.shape[-1] != self.n:
                raise ValueError(f"expected complex64 (..., {self.n}), got {x.dtype} {tuple(x.shape)}")
            return x.numel() // self.n
        want = torch.float16 if self.precision == "fp16" else torch.bfloat16
        if x.dtype != want or x.shape[-2:] != (self.n, 2):
            raise ValueError(f"expected {want} (..., {self.n}, 2), got {x.dtype} {tuple(x.shape)}")
        return x.numel() // (2 * self.n)

    def _check_tensor(self, x, name):
        import torch
        if not x.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if self.precision == "fp32":
            if x.dtype != torch.complex64 or x.shape[-1] != self.n:
                raise ValueError(f"{name}: expected complex64 (..., {self.n}), got {x.dtype} {tuple(x.shape)}")
            return x.numel() // self.n
        want = torch.float16 if self.precision == "fp16" else torch.bfloat16
        if x.dtype != want or x.shape[-2:] != (self.n, 2):
            raise ValueError(f"{name}: expected {want} (..., {self.n}, 2), got {x.dtype} {tuple(x.shape)}")
        return x.numel() // (2 * self.n)

    def exec(self, x, direction: int = FORWARD, out=None, stream=None):
        """Transform every signal of ``x`` (see module docstring for layouts)
        on ``stream`` (default: torch's current stream).  Returns ``out``."""
        import torch
        batch = self._check_tensor(x, "x")
        if out is None:
            out = torch.empty_like(x)
        elif self._check_tensor(out, "out") != batch or out.shape != x.shape:
            raise ValueError("out must have the shape of x")
        _check(lib().fft_exec(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                              batch, int(direction), _stream_handle(stream)), "fft_exec")
        return out

    def exec_ptr(self, in_ptr: int, out_ptr: int, batch: int, direction: int = FORWARD,
                 stream_handle: int = 0):
        """Raw-pointer form of :meth:`exec` (device pointers, cudaStream_t)."""
        _check(lib().fft_exec(self._h, ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr), int(batch),
                              int(direction), ctypes.c_void_p(stream_handle)), "fft_exec")

    def raw_table(self, direction: int = FORWARD) -> np.ndarray:
        """The packed device table for ``direction`` as a (N/2, 4) uint32 array."""
        h = self.n // 2
        buf = np.empty((h, 4), dtype=np.uint32)
        _check(lib().fft_plan_get_table(self._h, int(direction), buf.ctypes.data_as(ctypes.c_void_p),
                                        buf.nbytes), "fft_plan_get_table")
        return buf

    def raw_table4(self, direction: int = FORWARD) -> np.ndarray:
        """Radix-4 plans: the packed radix-4 table (k < 3N/4) as (3N/4, 4) uint32."""
        h = 3 * self.n // 4
        buf = np.empty((max(h, 1), 4), dtype=np.uint32)
        _check(lib().fft_plan_get_table4(self._h, int(direction), buf.ctypes.data_as(ctypes.c_void_p),
                                         buf.nbytes), "fft_plan_get_table4")
        return buf[:h]

    def table4(self, direction: int = FORWARD):
        """Decode the radix-4 table like :meth:`table` (m includes the /4 of a
        scaled direction)."""
        return self._decode(self.raw_table4(direction))

    def table(self, direction: int = FORWARD):
        """Decode the packed table: ``(t, m, path)`` as float64/float64/int32
        arrays (m includes the x0.5 of a scaled direction)."""
        return self._decode(self.raw_table(direction))

    def _decode(self, raw):
        if self.precision == "fp32":
            path = raw[:, 3].astype(np.int32)
        else:
            path = (raw[:, 2] == 0x3210).astype(np.int32)
        if self.precision == "fp32":
            t = raw[:, 0].view(np.float32).astype(np.float64)
            m = raw[:, 1].view(np.float32).astype(np.float64)
        else:
            thi = (raw[:, 0] >> 16).astype(np.uint16)
            mhi = (raw[:, 1] >> 16).astype(np.uint16)
            if self.precision == "fp16":
                t = thi.view(np.float16).astype(np.float64)
                m = mhi.view(np.float16).astype(np.float64)
            else:
                t = (thi.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
                m = (mhi.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        return t, m, path


class Batch:
    """A mixed batch: transforms of different sizes, precisions,
    factorizations and directions, each with its own tensors, run as one
    persistent launch (plus one launch per group of sizes above 2^14).

    ``items``: iterable of ``(n, precision, factorization, direction, x, out)``
    with ``x``/``out`` CUDA tensors in the layouts of :class:`Plan`."""

    def __init__(self, items, lf_eps: float | None = None):
        L = lib()
        items = list(items)
        arr = (BatchItemC * max(1, len(items)))()
        self._keep = []
        for i, (n, prec, fac, direction, x, out) in enumerate(items):
            for t in (x, out):
                if not t.is_cuda or not t.is_contiguous():
                    raise ValueError("batch tensors must be contiguous CUDA tensors")
            arr[i].n = int(n)
            arr[i].precision = PRECISIONS[prec]
            arr[i].factorization = FACTORIZATIONS[fac]
            arr[i].direction = int(direction)
            arr[i].reserved = 0
            arr[i].in_ = x.data_ptr()
            arr[i].out = out.data_ptr()
            self._keep.append((x, out))
        opts_p = None
        if lf_eps is not None:
            o = PlanOpts()
            L.fft_plan_opts_init(0, ctypes.byref(o))
            o.lf_eps = float(lf_eps)
            opts_p = ctypes.byref(o)
        h = ctypes.c_void_p()
        _check(L.fft_batch_create(ctypes.byref(h), arr, len(items), opts_p), "fft_batch_create")
        self._h = h

    def exec(self, stream=None):
        _check(lib().fft_batch_exec(self._h, _stream_handle(stream)), "fft_batch_exec")

    def exec_graph(self, stream=None):
        _check(lib().fft_batch_exec_graph(self._h, _stream_handle(stream)), "fft_batch_exec_graph")

    def info(self) -> dict:
        inf = BatchInfo()
        _check(lib().fft_batch_get_info(self._h, ctypes.byref(inf)), "fft_batch_get_info")
        return {k: getattr(inf, k) for k, _ in BatchInfo._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().fft_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pipeline:
    """Host-memory batches through a plan (``fft_pipeline_*``): chunks of
    ``chunk_transforms`` signals are copied in, transformed and copied back on
    ``depth`` streams so that copies and kernels overlap."""

    def __init__(self, plan: Plan, chunk_transforms: int, depth: int = 3):
        self.plan = plan
        h = ctypes.c_void_p()
        _check(lib().fft_pipeline_create(ctypes.byref(h), plan.handle, int(chunk_transforms), int(depth)),
               "fft_pipeline_create")
        self._h = h

    def exec(self, host_in, host_out, direction: int = FORWARD, stream=None):
        """``host_in``/``host_out``: CPU tensors (pinned for overlap) in the
        plan's layout."""
        if host_in.is_cuda or host_out.is_cuda:
            raise ValueError("pipeline buffers are host tensors")
        batch = self.plan._check_tensor_shape(host_in)
        if self.plan._check_tensor_shape(host_out) != batch:
            raise ValueError("host_out must match host_in")
        _check(lib().fft_pipeline_exec(self._h, ctypes.c_void_p(host_in.data_ptr()),
                                       ctypes.c_void_p(host_out.data_ptr()), batch, int(direction),
                                       _stream_handle(stream)), "fft_pipeline_exec")
        return host_out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().fft_pipeline_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _completion(c: CompletionC) -> dict:
    return {k: getattr(c, k) for k, _ in CompletionC._fields_ if k != "reserved"}


class Server:
    """The serving loop (``fft_server_*``): requests of any size, precision
    and direction are queued, admitted under the arena budget and launched
    together in ticks by the library's scheduler thread.  Inputs are CUDA
    tensors that must stay alive and unchanged until their request is done
    (the binding keeps a reference until then); outputs live in the server's
    arena until :meth:`release`."""

    def __init__(self, memory_budget: int = 40_000_000_000, max_ticks_in_flight: int = 2,
                 max_tick_transforms: int = 1 << 20, device: int | None = None, autotune: bool = False,
                 release_on_complete: bool = False, max_tick_bytes: int = 0):
        L = lib()
        o = ServerOptsC()
        _check(L.fft_server_opts_init(ctypes.byref(o)), "fft_server_opts_init")
        o.memory_budget = int(memory_budget)
        o.max_ticks_in_flight = int(max_ticks_in_flight)
        o.max_tick_transforms = int(max_tick_transforms)
        o.autotune = 1 if autotune else 0
        o.release_on_complete = 1 if release_on_complete else 0
        o.max_tick_bytes = int(max_tick_bytes)
        if device is not None:
            o.device = int(device)
        h = ctypes.c_void_p()
        _check(L.fft_server_create(ctypes.byref(h), ctypes.byref(o)), "fft_server_create")
        self._h = h
        self._inputs = {}

    @staticmethod
    def request(x, n: int, precision: str, factorization: str = "dual_select", direction: int = FORWARD,
                tag: int = 0) -> RequestC:
        """Request descriptor for the signals of CUDA tensor ``x``."""
        eb = 8 if precision == "fp32" else 4
        count = x.numel() * x.element_size() // (eb * int(n))
        r = RequestC()
        r.n, r.precision, r.factorization = int(n), PRECISIONS[precision], FACTORIZATIONS[factorization]
        r.direction, r.reserved, r.count, r.in_, r.tag = int(direction), 0, int(count), x.data_ptr(), int(tag)
        return r

    def prepare(self, n: int, precision: str, factorization: str = "dual_select"):
        _check(lib().fft_server_prepare(self._h, int(n), PRECISIONS[precision], FACTORIZATIONS[factorization]),
               "fft_server_prepare")

    def submit(self, x, n: int, precision: str, factorization: str = "dual_select", direction: int = FORWARD,
               tag: int = 0) -> int:
        if not x.is_cuda or not x.is_contiguous():
            raise ValueError("x must be a contiguous CUDA tensor")
        r = self.request(x, n, precision, factorization, direction, tag)
        t = ctypes.c_uint64()
        _check(lib().fft_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)), "fft_server_submit")
        self._inputs[t.value] = x
        return t.value

    def replay(self, requests, arrival_ns, keep=None):
        """Open-loop replay: ``requests`` (list of RequestC) submitted at
        ``arrival_ns`` offsets from now; returns the tickets.  ``keep``:
        tensors the requests read (kept alive by the caller)."""
        n = len(requests)
        arr = (RequestC * max(1, n))(*requests)
        t = (ctypes.c_int64 * max(1, n))(*[int(a) for a in arrival_ns])
        tickets = (ctypes.c_uint64 * max(1, n))()
        _check(lib().fft_server_replay(self._h, arr, t, n, tickets), "fft_server_replay")
        return list(tickets)[:n]

    def poll(self, max_items: int = 4096) -> list:
        buf = (CompletionC * max(1, max_items))()
        got = ctypes.c_int64()
        _check(lib().fft_server_poll(self._h, buf, int(max_items), ctypes.byref(got)), "fft_server_poll")
        out = [_completion(buf[i]) for i in range(got.value)]
        for c in out:
            self._inputs.pop(c["ticket"], None)
        return out

    def wait(self, ticket: int, timeout_s: float = 30.0) -> dict:
        c = CompletionC()
        _check(lib().fft_server_wait(self._h, int(ticket), float(timeout_s), ctypes.byref(c)), "fft_server_wait")
        self._inputs.pop(int(ticket), None)
        return _completion(c)

    def copy_out(self, ticket: int, dst, stream=None):
        """Copy a done request's output into tensor ``dst`` (CUDA or CPU)."""
        nbytes = dst.numel() * dst.element_size()
        _check(lib().fft_server_copy_out(self._h, int(ticket), ctypes.c_void_p(dst.data_ptr()), nbytes,
                                         _stream_handle(stream)), "fft_server_copy_out")
        return dst

    def release(self, ticket: int):
        _check(lib().fft_server_release(self._h, int(ticket)), "fft_server_release")

    def drain(self, timeout_s: float = 60.0):
        _check(lib().fft_server_drain(self._h, float(timeout_s)), "fft_server_drain")

    def stats(self) -> dict:
        st = ServerStatsC()
        _check(lib().fft_server_get_stats(self._h, ctypes.byref(st)), "fft_server_get_stats")
        return {k: getattr(st, k) for k, _ in ServerStatsC._fields_ if k != "reserved"}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().fft_server_destroy(self._h)
            self._h = None
            self._inputs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def exec_batch_noalloc(items, stream=None):
    """Mixed batch through ``fft_exec_batch_noalloc``, the entry point that
    allocates no device memory (for callers that cannot call cudaMalloc
    where they transform: programs that own all device memory through
    their own pool, or latency-bound loops that must not stall on the
    allocator).  ``items``: ``(plan, direction, x, out)`` with plans created
    beforehand and at most ``NOALLOC_MAX_ITEMS`` entries.  The library's
    fixed descriptor array is shared by all calls: keep calls that could
    overlap on the GPU on one stream."""
    items = list(items)
    arr = (NoAllocItemC * max(1, len(items)))()
    for i, (plan, direction, x, out) in enumerate(items):
        arr[i].plan = plan.handle.value
        arr[i].direction = int(direction)
        arr[i].reserved = 0
        arr[i].in_ = x.data_ptr()
        arr[i].out = out.data_ptr()
    _check(lib().fft_exec_batch_noalloc(arr, len(items), _stream_handle(stream)), "fft_exec_batch_noalloc")


def twiddle_fp64(n: int, factorization: str = "dual_select", lf_eps: float = 1e-7):
    """The GPU's FP64 table stage (before rounding), forward direction:
    ``(t, m, path)`` for k in [0, n/2)."""
    h = int(n) // 2
    t = np.empty(h, dtype=np.float64)
    m = np.empty(h, dtype=np.float64)
    p = np.empty(h, dtype=np.int32)
    _check(lib().fft_twiddle_fp64(int(n), FACTORIZATIONS[factorization], float(lf_eps),
                                  t.ctypes.data_as(ctypes.c_void_p), m.ctypes.data_as(ctypes.c_void_p),
                                  p.ctypes.data_as(ctypes.c_void_p)), "fft_twiddle_fp64")
    return t, m, p
