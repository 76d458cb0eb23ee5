"""GB300 layered BP syndrome decoder for QC-MET-LDPC codes (arXiv 2004.09084).

Python binding of ``libqcmet.so`` (C ABI in ``include/qcmet.h``).  This module
only marshals arguments: every step of decoding runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.  Importing the package
compiles the library with nvcc when it is missing or stale; without nvcc the
import raises.  There is no CPU fallback.

Typical use::

    import torch, paper_2004_09084_gb300 as q
    code = q.Code(base, shifts, Z)                   # host-only
    hard, post, ok = q.decode(code, llr, syn, iterations=100)   # CUDA tensors
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

# QCMET_DEBUG_BUILD=1 loads the debug build (every kernel index checked,
# qcmet_debug_checks); the default is the release build
_DEBUG = os.environ.get("QCMET_DEBUG_BUILD", "") == "1"
_LIB_PATH = _build.LIB_DEBUG if _DEBUG else _build.LIB

# status codes (include/qcmet.h)
OK = 0
ERR_INVALID_ARG = -1
ERR_SHIFT_RANGE = -2
ERR_DEGREE_LIMIT = -3
ERR_ALIGNMENT = -4
ERR_OOM = -5
ERR_CUDA = -6
ERR_TIMEOUT = -7
ERR_UNSUPPORTED = -8

MAX_ROW_DEGREE = 16

MERGE = {"none": 0, "exact": 1, "greedy": 2}
MSG = {"fp32": 0, "fp16": 1, "bf16": 2}
KERNEL = {"auto": 0, "frame": 1, "group": 2}

# every symbol the header declares
EXPORTS = (
    "qcmet_code_create", "qcmet_code_create_ex", "qcmet_code_destroy", "qcmet_code_get_info",
    "qcmet_code_get_schedule", "qcmet_decode", "qcmet_decode_ex", "qcmet_decode_host",
    "qcmet_last_error", "qcmet_status_string", "qcmet_version", "qcmet_decode_noalloc",
    "qcmet_decode_early_stop", "qcmet_minsum_decode", "qcmet_minsum_forward",
    "qcmet_minsum_backward", "qcmet_batch_create", "qcmet_batch_run", "qcmet_batch_get_config",
    "qcmet_batch_destroy", "qcmet_debug_checks", "qcmet_group_plan",
)


class QcmetError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"qcmet status {status}: {message}")
        self.status = status


class CodeInfo(ctypes.Structure):
    _fields_ = [("mb", ctypes.c_int32), ("nb", ctypes.c_int32), ("Z", ctypes.c_int32),
                ("n", ctypes.c_int32), ("m", ctypes.c_int32), ("edges", ctypes.c_int64),
                ("circulants", ctypes.c_int32), ("msg_slots", ctypes.c_int32),
                ("degree1_columns", ctypes.c_int32), ("layers", ctypes.c_int32),
                ("max_row_degree", ctypes.c_int32), ("merge_mode", ctypes.c_int32)]


class GroupPlan(ctypes.Structure):
    _fields_ = [("cluster_size", ctypes.c_int32), ("groups_per_cluster", ctypes.c_int32),
                ("threads_per_block", ctypes.c_int32), ("clusters", ctypes.c_int32),
                ("blocks", ctypes.c_int32), ("active_clusters", ctypes.c_int32),
                ("shared_bytes", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Frame(ctypes.Structure):
    _fields_ = [("code", ctypes.c_void_p), ("llr_ch", ctypes.c_void_p),
                ("syndrome", ctypes.c_void_p), ("hard", ctypes.c_void_p),
                ("llr_post", ctypes.c_void_p), ("ok", ctypes.c_void_p)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("threads_per_block", ctypes.c_int32), ("alternate_schedule", ctypes.c_int32),
                ("largest_first", ctypes.c_int32), ("candidates", ctypes.c_int32),
                ("trial_ms", ctypes.c_float), ("kernel", ctypes.c_int32),
                ("cluster_size", ctypes.c_int32), ("per_code_launches", ctypes.c_int32)]


class DecodeOptions(ctypes.Structure):
    _fields_ = [("msg_format", ctypes.c_int32), ("threads_per_block", ctypes.c_int32),
                ("l2_persist", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("cluster_size", ctypes.c_int32), ("groups_per_cluster", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


def _load():
    # Compile the CUDA library when it is missing or older than its sources
    # (raises without nvcc: there is no CPU fallback).
    _build.build(debug=_DEBUG)
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} was not built; there is no CPU fallback")
    lib = ctypes.CDLL(_LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.qcmet_code_create.argtypes = [vp, vp, i32, i32, i32, ctypes.POINTER(vp)]
    lib.qcmet_code_create_ex.argtypes = [vp, vp, i32, i32, i32, i32, ctypes.POINTER(vp)]
    lib.qcmet_code_destroy.argtypes = [vp]
    lib.qcmet_code_destroy.restype = None
    lib.qcmet_batch_destroy.restype = None
    lib.qcmet_code_get_info.argtypes = [vp, ctypes.POINTER(CodeInfo)]
    lib.qcmet_code_get_schedule.argtypes = [vp, vp, vp]
    dec = [vp, vp, vp, i32, i32, vp, vp, vp]
    lib.qcmet_decode.argtypes = dec + [vp]
    lib.qcmet_decode_ex.argtypes = dec + [ctypes.POINTER(DecodeOptions), vp]
    lib.qcmet_decode_host.argtypes = dec + [ctypes.POINTER(DecodeOptions), vp]
    lib.qcmet_decode_noalloc.argtypes = dec + [vp]
    lib.qcmet_decode_early_stop.argtypes = [vp, vp, vp, i32, i32, i32, vp, vp, vp, vp,
                                            ctypes.POINTER(DecodeOptions), vp]
    lib.qcmet_minsum_decode.argtypes = [vp, vp, vp, i32, i32, vp, vp, vp, vp, vp, vp]
    lib.qcmet_minsum_forward.argtypes = [vp, vp, vp, vp, i32, i32, vp, vp, vp, vp]
    lib.qcmet_minsum_backward.argtypes = [vp, vp, vp, vp]
    lib.qcmet_batch_create.argtypes = [ctypes.POINTER(Frame), i32, i32, i32, i32, vp,
                                       ctypes.POINTER(vp)]
    lib.qcmet_batch_run.argtypes = [vp, vp]
    lib.qcmet_batch_get_config.argtypes = [vp, ctypes.POINTER(BatchConfig)]
    lib.qcmet_batch_destroy.argtypes = [vp]
    lib.qcmet_last_error.argtypes = []
    lib.qcmet_last_error.restype = ctypes.c_char_p
    lib.qcmet_status_string.argtypes = [ctypes.c_int]
    lib.qcmet_status_string.restype = ctypes.c_char_p
    lib.qcmet_version.argtypes = []
    lib.qcmet_debug_checks.argtypes = [vp]
    lib.qcmet_group_plan.argtypes = [vp, i32, ctypes.POINTER(DecodeOptions), ctypes.POINTER(GroupPlan)]
    for name in EXPORTS:
        if name not in ("qcmet_code_destroy", "qcmet_last_error", "qcmet_status_string",
                        "qcmet_batch_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    del i64
    return lib


lib = _load()


def _check(status: int):
    if status != OK:
        raise QcmetError(status, lib.qcmet_last_error().decode(errors="replace"))


def library_path() -> str:
    return _LIB_PATH


def debug_checks() -> int:
    """Index-check bits recorded by the debug build since the last call (waits
    for the device; raises QcmetError(UNSUPPORTED) in the release build)."""
    bits = ctypes.c_uint32(0)
    _check(lib.qcmet_debug_checks(ctypes.byref(bits)))
    return int(bits.value)



def group_plan(code: "Code", K: int, msg: str = "fp32", cluster: int = 0, groups: int = 0) -> dict:
    """The launch shape of a grouped-kernel decode of K frames on the current
    device (``qcmet_group_plan``): cluster size, groups per cluster, threads,
    clusters, blocks, clusters the device holds at once, shared memory."""
    plan = GroupPlan()
    opts = _options(msg, 0, False, "group", cluster, groups)
    _check(lib.qcmet_group_plan(code._h, int(K), ctypes.byref(opts), ctypes.byref(plan)))
    return {name: int(getattr(plan, name)) for name, _ in GroupPlan._fields_ if name != "reserved"}


class Code:
    """A QC-MET-LDPC code: base matrix (1 = circulant), shifts and Z."""

    def __init__(self, base, shifts, Z: int, merge: str = "exact"):
        base = np.ascontiguousarray(base, dtype=np.int8)
        shifts = np.ascontiguousarray(shifts, dtype=np.int32)
        if base.ndim != 2 or shifts.shape != base.shape:
            raise ValueError("base and shifts must be 2-D arrays of the same shape")
        if merge not in MERGE:
            raise ValueError(f"merge must be one of {sorted(MERGE)}")
        self._h = ctypes.c_void_p()
        mb, nb = base.shape
        _check(lib.qcmet_code_create_ex(base.ctypes.data, shifts.ctypes.data, mb, nb, int(Z),
                                        MERGE[merge], ctypes.byref(self._h)))
        self.base = base
        self.shifts = shifts
        self.Z = int(Z)

    @classmethod
    def from_shift_matrix(cls, M, Z: int, merge: str = "exact") -> "Code":
        """Build from the paper's notation: entry a >= 0 is a shift, -1 a zero block."""
        M = np.asarray(M)
        return cls((M >= 0).astype(np.int8), np.where(M >= 0, M, 0).astype(np.int32), Z, merge)

    @property
    def handle(self):
        if not self._h:
            raise ValueError("code handle is closed")
        return self._h

    def info(self) -> dict:
        ci = CodeInfo()
        _check(lib.qcmet_code_get_info(self.handle, ctypes.byref(ci)))
        return {name: getattr(ci, name) for name, _ in CodeInfo._fields_}

    def schedule(self):
        """(rows in visiting order, list of layers as lists of base rows)."""
        inf = self.info()
        rows = np.full(inf["mb"], -1, dtype=np.int32)
        first = np.zeros(inf["layers"] + 1, dtype=np.int32)
        _check(lib.qcmet_code_get_schedule(self.handle, rows.ctypes.data, first.ctypes.data))
        layers = [rows[first[k]:first[k + 1]].tolist() for k in range(inf["layers"])]
        return rows[:first[-1]], layers

    def close(self):
        if self._h:
            lib.qcmet_code_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _options(msg: str, threads: int, l2_persist: bool = False, kernel: str = "auto",
             cluster: int = 0, groups: int = 0) -> DecodeOptions:
    if msg not in MSG:
        raise ValueError(f"msg must be one of {sorted(MSG)}")
    if kernel not in KERNEL:
        raise ValueError(f"kernel must be one of {sorted(KERNEL)}")
    o = DecodeOptions()
    o.msg_format = MSG[msg]
    o.threads_per_block = int(threads)
    o.l2_persist = 1 if l2_persist else 0
    o.kernel = KERNEL[kernel]
    o.cluster_size = int(cluster)
    o.groups_per_cluster = int(groups)
    return o


def decode(code: Code, llr, syn, iterations: int, hard=None, llr_post=None, ok=None,
           msg: str = "fp32", threads: int = 0, stream=None, want_post: bool = True,
           l2_persist: bool = False, kernel: str = "auto", cluster: int = 0, groups: int = 0):
    """Decode K frames on the GPU (``qcmet_decode_ex``).

    ``llr``: float32 CUDA tensor [K, n]; ``syn``: uint8 CUDA tensor [K, m].
    Outputs are allocated when not given.  Returns ``(hard, llr_post, ok)``
    (``llr_post`` is None when ``want_post`` is false and none was passed).
    The call is asynchronous on ``stream`` (default: torch's current stream).
    ``l2_persist`` keeps the core posteriors in a persisting L2 window (frame
    kernel only); the persisting-L2 limit it raises is put back before the
    library's next decode without a window on that device.
    ``kernel`` is "auto", "frame" or "group" (``QCMET_KERNEL_*``); ``cluster``
    the grouped kernel's cluster size and ``groups`` its groups of four frames
    per cluster (0 = automatic).
    """
    import torch

    inf_n = code.base.shape[1] * code.Z
    inf_m = code.base.shape[0] * code.Z
    if llr.dtype != torch.float32 or syn.dtype != torch.uint8:
        raise TypeError("llr must be float32 and syn uint8")
    if not (llr.is_cuda and syn.is_cuda):
        raise ValueError("llr and syn must be CUDA tensors (use decode_host for host arrays)")
    if llr.dim() != 2 or llr.shape[1] != inf_n or syn.shape != (llr.shape[0], inf_m):
        raise ValueError(f"expected llr [K, {inf_n}] and syn [K, {inf_m}]")
    if not (llr.is_contiguous() and syn.is_contiguous()):
        raise ValueError("llr and syn must be contiguous")
    K = llr.shape[0]
    dev = llr.device
    if hard is None:
        hard = torch.empty((K, inf_n), dtype=torch.uint8, device=dev)
    if ok is None:
        ok = torch.empty((K,), dtype=torch.uint8, device=dev)
    if llr_post is None and want_post:
        llr_post = torch.empty((K, inf_n), dtype=torch.float32, device=dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    opts = _options(msg, threads, l2_persist, kernel, cluster, groups)
    _check(lib.qcmet_decode_ex(code.handle, llr.data_ptr(), syn.data_ptr(), K, int(iterations),
                               hard.data_ptr(), llr_post.data_ptr() if llr_post is not None else None,
                               ok.data_ptr(), ctypes.byref(opts), sptr))
    return hard, llr_post, ok


def decode_early_stop(code: Code, llr, syn, max_iterations: int, check_every: int = 1,
                      msg: str = "fp32", threads: int = 0, stream=None, l2_persist: bool = False,
                      kernel: str = "auto"):
    """Decode with early termination (``qcmet_decode_early_stop``).

    Returns ``(hard, llr_post, ok, iterations_used)`` as CUDA tensors; the call
    is asynchronous on ``stream``.
    """
    import torch

    n = code.base.shape[1] * code.Z
    m = code.base.shape[0] * code.Z
    if llr.dtype != torch.float32 or syn.dtype != torch.uint8 or not (llr.is_cuda and syn.is_cuda):
        raise TypeError("llr must be a float32 CUDA tensor and syn a uint8 CUDA tensor")
    if llr.dim() != 2 or llr.shape[1] != n or syn.shape != (llr.shape[0], m):
        raise ValueError(f"expected llr [K, {n}] and syn [K, {m}]")
    K = llr.shape[0]
    dev = llr.device
    hard = torch.empty((K, n), dtype=torch.uint8, device=dev)
    post = torch.empty((K, n), dtype=torch.float32, device=dev)
    ok = torch.empty((K,), dtype=torch.uint8, device=dev)
    iters = torch.empty((K,), dtype=torch.int32, device=dev)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    opts = _options(msg, threads, l2_persist, kernel)
    _check(lib.qcmet_decode_early_stop(code.handle, llr.data_ptr(), syn.data_ptr(), K,
                                       int(max_iterations), int(check_every), hard.data_ptr(),
                                       post.data_ptr(), ok.data_ptr(), iters.data_ptr(),
                                       ctypes.byref(opts), sptr))
    return hard, post, ok, iters


def decode_host(code: Code, llr: np.ndarray, syn: np.ndarray, iterations: int,
                want_post: bool = True, msg: str = "fp32", threads: int = 0, stream=None,
                out=None, l2_persist: bool = False, kernel: str = "auto", cluster: int = 0,
                groups: int = 0):
    """Decode frames held in host memory (``qcmet_decode_host``); synchronous.

    ``out`` may supply preallocated (hard, llr_post, ok) host arrays, e.g. pinned.
    """
    K = llr.shape[0]
    n = code.base.shape[1] * code.Z
    if out is None:
        hard = np.empty((K, n), dtype=np.uint8)
        post = np.empty((K, n), dtype=np.float32) if want_post else None
        ok = np.empty((K,), dtype=np.uint8)
    else:
        hard, post, ok = out
    for a, dt in ((llr, np.float32), (syn, np.uint8), (hard, np.uint8), (ok, np.uint8)):
        if a.dtype != dt or not a.flags.c_contiguous:
            raise ValueError("host arrays must be C-contiguous with the documented dtypes")
    opts = _options(msg, threads, l2_persist, kernel, cluster, groups)
    sptr = 0
    if stream is not None:
        sptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _check(lib.qcmet_decode_host(code.handle, llr.ctypes.data, syn.ctypes.data, K,
                                 int(iterations), hard.ctypes.data,
                                 post.ctypes.data if post is not None else None, ok.ctypes.data,
                                 ctypes.byref(opts), sptr))
    return hard, post, ok


class Batch:
    """A mixed batch plan (``qcmet_batch_*``): frames of several codes in one
    captured graph (one launch, or one concurrent launch per code).

    ``frames`` is a list of ``(code, llr, syn)`` with CUDA tensors of that
    code's sizes.  Outputs are allocated here (``self.hard``, ``self.post``,
    ``self.ok``); :meth:`run` replays the captured graph.  Keep the input
    tensors alive and write new data into them to decode again.  ``autotune``:
    True (1) times every configuration, False (0) takes the grouped kernel with
    clusters of 4, 2 takes one concurrent launch per code without timing.
    """

    def __init__(self, frames, iterations: int, msg: str = "fp32", autotune=True,
                 stream=None, want_post: bool = True):
        import torch
        self._keep = []
        arr = (Frame * len(frames))()
        self.hard, self.post, self.ok = [], [], []
        for k, (code, llr, syn) in enumerate(frames):
            n = code.base.shape[1] * code.Z
            m = code.base.shape[0] * code.Z
            if llr.numel() != n or syn.numel() != m or llr.dtype != torch.float32 \
                    or syn.dtype != torch.uint8 or not (llr.is_cuda and syn.is_cuda):
                raise ValueError(f"frame {k}: expected float32 llr [{n}] and uint8 syn [{m}] on CUDA")
            h = torch.empty((n,), dtype=torch.uint8, device=llr.device)
            o = torch.empty((16,), dtype=torch.uint8, device=llr.device)
            p = torch.empty((n,), dtype=torch.float32, device=llr.device) if want_post else None
            self.hard.append(h)
            self.ok.append(o)
            self.post.append(p)
            self._keep += [code, llr, syn]
            arr[k] = Frame(code.handle.value, llr.data_ptr(), syn.data_ptr(), h.data_ptr(),
                           p.data_ptr() if p is not None else None, o.data_ptr())
        self._h = ctypes.c_void_p()
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        _check(lib.qcmet_batch_create(arr, len(frames), int(iterations), MSG[msg],
                                      int(autotune), self._stream, ctypes.byref(self._h)))

    def run(self, stream=None):
        s = self._stream if stream is None else (
            stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        _check(lib.qcmet_batch_run(self._h, s))

    def config(self) -> dict:
        c = BatchConfig()
        _check(lib.qcmet_batch_get_config(self._h, ctypes.byref(c)))
        return {name: getattr(c, name) for name, _ in BatchConfig._fields_ if name != "reserved"}

    def close(self):
        if self._h:
            lib.qcmet_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
