"""Learned offset/scaled min-sum on top of the layered decoder.

Not part of arXiv 2004.09084's method: its layered decoder (Methods, steps
1-4) with the check rule of step 2 replaced by a min-sum rule with one scale
and one offset per (iteration, base row, edge type).  Forward and backward run
in the library's CUDA kernels (``qcmet_minsum_forward`` /
``qcmet_minsum_backward``); this module wraps them in a
``torch.autograd.Function`` and provides weight initialisation, decoding and a
training step.  Plain tanh-rule BP (``paper_2004_09084_gb300.decode``) remains
the reference decoder.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import Code, _check, lib

WEIGHTS_FORMAT = "qcmet-minsum-weights"
WEIGHTS_VERSION = 1


def _ptr(t):
    return t.data_ptr() if t is not None else None


def _stream(torch, dev, stream=None):
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    return s.cuda_stream if hasattr(s, "cuda_stream") else int(s)


def init_weights(code: Code, iterations: int, scale: float = 1.0, offset: float = 0.0,
                 device="cuda"):
    """Weights [iterations, mb, 2] (FP32, on `device`); (1, 0) is plain min-sum."""
    import torch
    mb = code.base.shape[0]
    ws = torch.full((iterations, mb, 2), float(scale), dtype=torch.float32, device=device)
    wo = torch.full((iterations, mb, 2), float(offset), dtype=torch.float32, device=device)
    return ws, wo


def decode(code: Code, llr, syn, w_scale, w_offset, stream=None):
    """Decode with learned weights; returns (hard, llr_post, ok) CUDA tensors."""
    import torch
    T = int(w_scale.shape[0])
    K, n = llr.shape
    dev = llr.device
    hard = torch.empty((K, n), dtype=torch.uint8, device=dev)
    post = torch.empty((K, n), dtype=torch.float32, device=dev)
    ok = torch.empty((K,), dtype=torch.uint8, device=dev)
    ws = w_scale.detach().contiguous()
    wo = w_offset.detach().contiguous()
    _check(lib.qcmet_minsum_decode(code.handle, llr.data_ptr(), syn.data_ptr(), K, T,
                                   ws.data_ptr(), wo.data_ptr(), hard.data_ptr(), post.data_ptr(),
                                   ok.data_ptr(), _stream(torch, dev, stream)))
    return hard, post, ok


def _function():
    import torch

    class MinSumLoss(torch.autograd.Function):
        """loss[k] of the unrolled learned decoder; backward by the hand-written kernel."""

        @staticmethod
        def forward(ctx, w_scale, w_offset, code, llr, syn, bits):
            ws = w_scale.detach().contiguous()
            wo = w_offset.detach().contiguous()
            K = llr.shape[0]
            T = int(ws.shape[0])
            loss = torch.empty((K,), dtype=torch.float32, device=llr.device)
            _check(lib.qcmet_minsum_forward(code.handle, llr.data_ptr(), syn.data_ptr(),
                                            bits.data_ptr(), K, T, ws.data_ptr(), wo.data_ptr(),
                                            loss.data_ptr(), _stream(torch, llr.device)))
            ctx.code = code
            ctx.keep = (ws, wo, llr, syn, bits)   # the kernels read them in backward
            return loss

        @staticmethod
        def backward(ctx, g_loss):
            ws = ctx.keep[0]
            gs = torch.empty_like(ws)
            go = torch.empty_like(ws)
            _check(lib.qcmet_minsum_backward(ctx.code.handle, gs.data_ptr(), go.data_ptr(),
                                             _stream(torch, ws.device)))
            # the kernel returns the gradient of sum_k loss[k]; the chain rule through
            # a per-frame upstream gradient needs it frame by frame, which the kernel
            # does not keep, so only a uniform upstream gradient is supported
            g = g_loss.detach()
            if not torch.allclose(g, g[:1].expand_as(g)):
                raise NotImplementedError("MinSumLoss supports loss.sum() / loss.mean() only")
            scale = g[0]
            return gs * scale, go * scale, None, None, None, None

    return MinSumLoss


_FN = None


def minsum_loss(w_scale, w_offset, code: Code, llr, syn, bits):
    """Per-frame training loss (differentiable in the weights)."""
    global _FN
    if _FN is None:
        _FN = _function()
    return _FN.apply(w_scale, w_offset, code, llr, syn, bits)


def make_batch(code: Code, K: int, snr_lo: float, snr_hi: float, generator):
    """Decoder-generated training frames on the GPU: random bits, their syndromes
    s = Hx and BIAWGN LLRs, each frame at an SNR drawn uniformly in [snr_lo, snr_hi]."""
    import torch
    dev = generator.device
    Z = code.Z
    mb, nb = code.base.shape
    x = torch.randint(0, 2, (K, nb * Z), generator=generator, device=dev, dtype=torch.uint8)
    xb = x.view(K, nb, Z)
    syn = torch.zeros((K, mb, Z), dtype=torch.uint8, device=dev)
    for l in range(mb):
        for c in np.flatnonzero(code.base[l]):
            a = int(code.shifts[l, c])
            syn[:, l, :] ^= torch.roll(xb[:, c, :], shifts=-a, dims=1)   # row i takes x[c, (i + a) mod Z]
    snr = snr_lo + (snr_hi - snr_lo) * torch.rand((K, 1), generator=generator, device=dev)
    noise = torch.randn((K, nb * Z), generator=generator, device=dev)
    y = (1.0 - 2.0 * x.float()) + noise / torch.sqrt(snr)
    llr = (2.0 * y * snr).float().contiguous()
    return llr, syn.view(K, mb * Z).contiguous(), x.contiguous()


def code_digest(base, shifts, Z: int) -> str:
    """sha256 of a code's description (shape, base matrix, shifts, Z): weights
    belong to one code, so a file records which."""
    base = np.ascontiguousarray(base, dtype=np.int8)
    shifts = np.ascontiguousarray(np.where(base == 1, shifts, 0), dtype=np.int32)
    h = hashlib.sha256()
    h.update(np.asarray(base.shape, dtype=np.int64).tobytes())
    h.update(base.tobytes())
    h.update(shifts.astype("<i4").tobytes())
    h.update(np.int64(Z).tobytes())
    return h.hexdigest()


def save_weights(path: str, w_scale, w_offset, base, shifts, Z: int, info: dict | None = None):
    """Write learned weights as a flat FP32 file plus a JSON header.

    ``path`` receives the raw little-endian float32 values of ``w_scale``
    followed by those of ``w_offset``, each ``[iterations][mb][2]`` row-major
    (edge type 0: edges to variables of degree > 1, 1: edges to degree-1
    variables); ``path + ".json"`` receives the header: format, version,
    shape, layout, byte counts, the sha256 of the data, the code it belongs to
    (mb, nb, Z, digest of base and shifts) and ``info`` (free-form, e.g. the
    training SNR range).  Accepts numpy arrays or tensors (any device).
    """
    ws = _as_numpy(w_scale)
    wo = _as_numpy(w_offset)
    base = np.asarray(base)
    mb, nb = base.shape
    if ws.shape != wo.shape or ws.ndim != 3 or ws.shape[1] != mb or ws.shape[2] != 2:
        raise ValueError(f"weights must both have shape [iterations, {mb}, 2]")
    data = ws.astype("<f4").tobytes() + wo.astype("<f4").tobytes()
    header = {
        "format": WEIGHTS_FORMAT, "version": WEIGHTS_VERSION, "dtype": "float32-le",
        "shape": [int(ws.shape[0]), int(mb), 2],
        "layout": "w_scale then w_offset, each [iteration][base row][edge type] row-major; "
                  "edge type 0: to a variable of degree > 1, 1: to a degree-1 variable",
        "bytes": len(data), "sha256": hashlib.sha256(data).hexdigest(),
        "code": {"mb": int(mb), "nb": int(nb), "Z": int(Z), "digest": code_digest(base, shifts, Z)},
        "info": info or {},
    }
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        f.write(data)
    os.replace(tmp, path)
    with open(path + ".json", "w") as f:
        json.dump(header, f, indent=1, sort_keys=True)
    return header


def load_weights(path: str, base=None, shifts=None, Z: int | None = None):
    """Read weights written by :func:`save_weights`; returns ``(w_scale,
    w_offset, header)`` as float32 numpy arrays.  Checks the format, the byte
    count and the data digest, and, when the code is given, that the weights
    belong to it; raises ValueError otherwise."""
    with open(path + ".json") as f:
        header = json.load(f)
    if header.get("format") != WEIGHTS_FORMAT or header.get("version") != WEIGHTS_VERSION:
        raise ValueError(f"{path}: not a {WEIGHTS_FORMAT} v{WEIGHTS_VERSION} file")
    with open(path, "rb") as f:
        data = f.read()
    if len(data) != header["bytes"] or hashlib.sha256(data).hexdigest() != header["sha256"]:
        raise ValueError(f"{path}: data does not match its header (size or sha256)")
    T, mb, two = header["shape"]
    count = T * mb * two
    if header["bytes"] != 2 * 4 * count:
        raise ValueError(f"{path}: byte count disagrees with the shape")
    vals = np.frombuffer(data, dtype="<f4")
    ws = vals[:count].reshape(T, mb, two).astype(np.float32)
    wo = vals[count:].reshape(T, mb, two).astype(np.float32)
    if base is not None:
        if Z is None or shifts is None:
            raise ValueError("give base, shifts and Z together")
        if code_digest(base, shifts, Z) != header["code"]["digest"]:
            raise ValueError(f"{path}: the weights belong to another code")
    return ws, wo, header


def _as_numpy(x):
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(x, dtype=np.float32)
