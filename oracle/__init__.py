"""FP64 CPU oracle for layered sum-product syndrome decoding (arXiv 2004.09084).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The CUDA decoder never imports it
and shares no code with it.  The arithmetic lives in ``qcmet_oracle.c`` (plain
C, double precision); this module compiles it with gcc when needed and wraps it
with ctypes.

Functions mirror the paper's Methods section:

* :func:`phi` -- ``Phi(x) = -ln tanh(x/2)`` with the clipping reading.
* :func:`check_update` -- step 2 for one check node.
* :func:`decode` -- steps 1-4 over a layered schedule (base rows in order, or
  a caller-given row order).

Parity status: every function is pinned by ``tests/test_oracle_pins.py``
(brute-force marginals, exact APP on cycle-free codes, closed forms and
invariants).  The min-sum rule is pinned by brute force on single checks and
by the finite-difference check of its backward pass.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qcmet_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

RULE_PHI = 0
RULE_TANH = 1
RULE_MINSUM = 2

MSG_EXACT = 0
MSG_FP16 = 1
MSG_BF16 = 2

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``qcmet_oracle.c`` into ``liboracle.so`` (gcc, -O2, no fast-math)."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                   "-ffp-contract=off", "-D_GNU_SOURCE", "-o", tmp, _SRC, "-lm", "-lpthread"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    d = ctypes.c_double
    i = ctypes.c_int
    p = ctypes.c_void_p
    lib.oracle_phi.argtypes = [d]
    lib.oracle_phi.restype = d
    lib.oracle_clip_min.argtypes = []
    lib.oracle_clip_min.restype = d
    lib.oracle_clip_max.argtypes = []
    lib.oracle_clip_max.restype = d
    lib.oracle_round_msg.argtypes = [d, i]
    lib.oracle_round_msg.restype = d
    lib.oracle_check_update.argtypes = [i, p, i, i, p]
    lib.oracle_check_update.restype = None
    lib.oracle_decode.argtypes = [i, i, i, p, p, p, i, i, i, p, p, p, p, p, i, i, p, p, i, i, p]
    lib.oracle_decode.restype = i
    lib.oracle_minsum_train.argtypes = [i, i, i, p, p, i, i, p, p, p, p, p, p, p, p]
    lib.oracle_minsum_train.restype = i
    _lib = lib
    return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def clip_min() -> float:
    return _load().oracle_clip_min()


def clip_max() -> float:
    return _load().oracle_clip_max()


def phi(x: float) -> float:
    """Clipped ``Phi(x) = -ln tanh(x/2)`` (Methods, step 2)."""
    return _load().oracle_phi(float(x))


def round_msg(r: float, fmt: int) -> float:
    """Round a message to the storage format ``fmt`` (MSG_EXACT/FP16/BF16)."""
    return _load().oracle_round_msg(float(r), int(fmt))


def check_update(q, s: int = 0, rule: int = RULE_PHI) -> np.ndarray:
    """Step 2 for one check node: V2C messages ``q`` -> C2V messages."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    r = np.empty_like(q)
    _load().oracle_check_update(int(q.size), _ptr(q), int(s) & 1, int(rule), _ptr(r))
    return r


def decode(base, shifts, Z: int, llr, syn, iterations: int, order=None,
           rule: int = RULE_PHI, msg_fmt: int = MSG_EXACT, w_scale=None, w_offset=None,
           nthreads: int = 1, early_every: int = 0, return_iters: bool = False):
    """Layered BP (Methods steps 1-4) on ``K`` frames.

    Returns ``(hard uint8 [K, n], llr_post float64 [K, n], ok uint8 [K])``, plus
    ``iters_used int32 [K]`` when ``return_iters``.  ``order`` is the sequence
    of base rows one iteration visits (default ``0..mb-1``).  ``w_scale``/
    ``w_offset`` are the min-sum weights with shape ``[iterations, mb, 2]``.
    ``early_every > 0`` stops a frame after the first multiple of
    ``early_every`` iterations at which ``H c = s`` (early termination).
    """
    base = np.ascontiguousarray(base, dtype=np.int8)
    shifts = np.ascontiguousarray(shifts, dtype=np.int32)
    mb, nb = base.shape
    n, m = nb * Z, mb * Z
    llr = np.ascontiguousarray(llr, dtype=np.float32).reshape(-1, n)
    syn = np.ascontiguousarray(syn, dtype=np.uint8).reshape(-1, m)
    K = llr.shape[0]
    if syn.shape[0] != K:
        raise ValueError("llr and syn disagree on the number of frames")
    hard = np.empty((K, n), dtype=np.uint8)
    post = np.empty((K, n), dtype=np.float64)
    ok = np.empty((K,), dtype=np.uint8)
    ordr = None
    n_order = 0
    if order is not None:
        ordr = np.ascontiguousarray(order, dtype=np.int32)
        n_order = int(ordr.size)
    ws = wo = None
    if rule == RULE_MINSUM:
        ws = np.ascontiguousarray(w_scale, dtype=np.float64).reshape(-1)
        wo = np.ascontiguousarray(w_offset, dtype=np.float64).reshape(-1)
        if ws.size < iterations * mb * 2 or wo.size < iterations * mb * 2:
            raise ValueError("min-sum weights must have shape [iterations, mb, 2]")
    iters = np.empty((K,), dtype=np.int32)
    rc = _load().oracle_decode(mb, nb, int(Z), _ptr(base), _ptr(shifts), _ptr(ordr), n_order,
                               K, int(iterations), _ptr(llr), _ptr(syn), _ptr(hard), _ptr(post),
                               _ptr(ok), int(rule), int(msg_fmt), _ptr(ws), _ptr(wo),
                               int(nthreads), int(early_every), _ptr(iters))
    if rc != 0:
        raise ValueError(f"oracle_decode failed with status {rc}")
    if return_iters:
        return hard, post, ok, iters
    return hard, post, ok


def minsum_train(base, shifts, Z: int, llr, syn, x, iterations: int, w_scale, w_offset):
    """Learned min-sum: per-frame loss and the gradient of the summed loss.

    The loss is the mean over iterations and variables of the cross-entropy
    of sigma(-L) against the transmitted bits.  Returns ``(loss [K],
    g_scale [T, mb, 2], g_offset [T, mb, 2])`` in float64.
    """
    base = np.ascontiguousarray(base, dtype=np.int8)
    shifts = np.ascontiguousarray(shifts, dtype=np.int32)
    mb, nb = base.shape
    n, m = nb * Z, mb * Z
    llr = np.ascontiguousarray(llr, dtype=np.float32).reshape(-1, n)
    syn = np.ascontiguousarray(syn, dtype=np.uint8).reshape(-1, m)
    x = np.ascontiguousarray(x, dtype=np.uint8).reshape(-1, n)
    K = llr.shape[0]
    ws = np.ascontiguousarray(w_scale, dtype=np.float64).reshape(iterations, mb, 2)
    wo = np.ascontiguousarray(w_offset, dtype=np.float64).reshape(iterations, mb, 2)
    loss = np.empty((K,), dtype=np.float64)
    gs = np.empty_like(ws)
    go = np.empty_like(wo)
    rc = _load().oracle_minsum_train(mb, nb, int(Z), _ptr(base), _ptr(shifts), K, int(iterations),
                                     _ptr(llr), _ptr(syn), _ptr(x), _ptr(ws), _ptr(wo),
                                     _ptr(loss), _ptr(gs), _ptr(go))
    if rc != 0:
        raise ValueError(f"oracle_minsum_train failed with status {rc}")
    return loss, gs, go
