"""Seeded synthetic workloads for QC-MET-LDPC syndrome decoding.

This module produces *inputs only*: a quasi-cyclic base matrix with circulant
shifts, random information bits, their syndromes and BIAWGN channel LLRs.  It
contains none of the decoder's arithmetic and is the one module that both the
CUDA path (tests, ``bench.py``) and the CPU oracle side (tests) draw inputs
from.

Conventions (arXiv 2004.09084):

* Circulant convention, Results section around Eq. (m): a non-negative base
  entry ``a`` is the Z x Z identity cyclically shifted to the right by ``a``,
  so row ``i`` of that block has its one in column ``(i + a) mod Z``.  Check
  ``l*Z + i`` therefore touches variable ``c*Z + (i + a) mod Z``.
* Channel, Methods step 1: ``L = 2R / sigma^2``.  BPSK maps bit 0 -> +1 and
  bit 1 -> -1, ``R = (1 - 2x) + N(0, sigma^2)`` and ``sigma^2 = 1/SNR`` (the
  reading that reproduces the efficiencies of Table tab1).
* Syndrome decoding, Methods step 2: ``s = H x mod 2``.

Code construction.  The paper's own codes (Z = 2500, n = 10^6) are not
published with it.  The stand-in is the multi-edge-type shape
``[[A, 0], [B, I]]``: ``A`` is 2 x core with every block a circulant, each row
of ``B`` holds 3 circulants on distinct core columns, and ``I`` is an identity
block (shift 0) per ``B`` row, which makes the last ``nb - core`` columns
degree-1 variables.  Shapes per named rate (nb = 80 throughout):

======  =====  ======  ==========================================
rate    mb     core    design rate 1 - mb/nb
======  =====  ======  ==========================================
0.1     72     10      0.1
0.05    76     6       0.05
0.02    78     4       0.025 (the 78 x 80 shape of the named code)
======  =====  ======  ==========================================

Random numbers come from NumPy's PCG64 (``numpy.random.default_rng``).  The
code uses seed 20040908; frame ``k`` uses seed ``9084 + k``.  The draw order is
fixed and documented in each function so that a stream can be replayed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

CODE_SEED = 20040908
FRAME_SEED0 = 9084

# named rate -> (mb, nb, core columns)
RATE_SHAPES = {
    "0.1": (72, 80, 10),
    "0.05": (76, 80, 6),
    "0.02": (78, 80, 4),
}

# SNR each named rate is decoded at (Table tab1 / the workload configurations)
RATE_SNR = {"0.1": 0.161, "0.05": 0.076, "0.02": 0.029}


@dataclass(frozen=True)
class Code:
    """A QC code: ``base[l, c] = 1`` marks a circulant with shift ``shifts[l, c]``."""

    base: np.ndarray    # int8  [mb, nb]
    shifts: np.ndarray  # int32 [mb, nb] (0 where base == 0)
    Z: int

    @property
    def mb(self) -> int:
        return int(self.base.shape[0])

    @property
    def nb(self) -> int:
        return int(self.base.shape[1])

    @property
    def n(self) -> int:
        return self.nb * self.Z

    @property
    def m(self) -> int:
        return self.mb * self.Z

    @property
    def edges(self) -> int:
        return int(self.base.sum()) * self.Z


def make_code(rate: str = "0.1", Z: int = 64, seed: int = CODE_SEED) -> Code:
    """Build the ``[[A, 0], [B, I]]`` stand-in code for a named rate.

    Draw order from ``default_rng(seed)``: the 2 x core shifts of ``A`` (row
    major, ``integers(0, Z)``); then for each ``B`` row in order, 3 distinct
    core columns (``choice(core, 3, replace=False)``) followed by their 3
    shifts (``integers(0, Z, 3)``).  Identity blocks have shift 0.
    """
    if rate not in RATE_SHAPES:
        raise ValueError(f"unknown rate {rate!r}; choose from {sorted(RATE_SHAPES)}")
    if Z < 1:
        raise ValueError("Z must be >= 1")
    mb, nb, core = RATE_SHAPES[rate]
    rng = np.random.default_rng(seed)
    base = np.zeros((mb, nb), dtype=np.int8)
    shifts = np.zeros((mb, nb), dtype=np.int32)
    base[0:2, :core] = 1
    shifts[0:2, :core] = rng.integers(0, Z, size=(2, core))
    for j in range(mb - 2):
        cols = rng.choice(core, 3, replace=False)
        base[2 + j, cols] = 1
        shifts[2 + j, cols] = rng.integers(0, Z, size=3)
        base[2 + j, core + j] = 1
        shifts[2 + j, core + j] = 0
    return Code(base=base, shifts=shifts, Z=int(Z))


def syndrome(code: Code, x: np.ndarray) -> np.ndarray:
    """``s = H x mod 2`` for bits ``x`` of shape ``[..., n]`` (uint8 result ``[..., m]``)."""
    Z = code.Z
    x = np.asarray(x, dtype=np.uint8)
    lead = x.shape[:-1]
    xb = x.reshape(lead + (code.nb, Z))
    s = np.zeros(lead + (code.mb, Z), dtype=np.uint8)
    for l in range(code.mb):
        for c in np.flatnonzero(code.base[l]):
            a = int(code.shifts[l, c])
            # row i of the block picks x[c*Z + (i + a) mod Z]
            s[..., l, :] ^= np.roll(xb[..., c, :], -a, axis=-1)
    return s.reshape(lead + (code.m,))


@dataclass
class Frames:
    x: np.ndarray    # uint8   [K, n] transmitted bits
    llr: np.ndarray  # float32 [K, n] channel LLRs 2R/sigma^2
    syn: np.ndarray  # uint8   [K, m] syndromes H x
    snr: float


def make_frames(code: Code, K: int, snr: float, seed0: int = FRAME_SEED0,
                first: int = 0, noiseless: bool = False) -> Frames:
    """Random frames over the BIAWGN channel.

    Frame ``k`` draws from ``default_rng(seed0 + first + k)``: ``n`` bits with
    ``integers(0, 2)`` then ``n`` standard normals.  ``noiseless`` keeps the
    same draws but drops the noise term (``R = 1 - 2x``).
    """
    if K < 0:
        raise ValueError("K must be >= 0")
    if snr <= 0:
        raise ValueError("snr must be > 0")
    n = code.n
    sigma2 = 1.0 / snr
    sigma = math.sqrt(sigma2)
    x = np.empty((K, n), dtype=np.uint8)
    llr = np.empty((K, n), dtype=np.float32)
    for k in range(K):
        rng = np.random.default_rng(seed0 + first + k)
        x[k] = rng.integers(0, 2, size=n, dtype=np.uint8)
        noise = rng.standard_normal(n)
        R = (1.0 - 2.0 * x[k].astype(np.float64))
        if not noiseless:
            R = R + sigma * noise
        llr[k] = (2.0 * R / sigma2).astype(np.float32)
    return Frames(x=x, llr=llr, syn=syndrome(code, x), snr=float(snr))


def capacity_biawgn_gaussian(snr: float) -> float:
    """Shannon capacity ``0.5 * log2(1 + SNR)`` in bits per channel use."""
    return 0.5 * math.log2(1.0 + snr)


def efficiency(rate: float, snr: float) -> float:
    """Reconciliation efficiency ``beta = R / C(SNR)`` (Table tab1, row beta)."""
    return rate / capacity_biawgn_gaussian(snr)
