"""Test-side helpers written independently of both decoders.

* :func:`expand_dense` builds H from (base, shifts, Z) with the circulant
  convention of arXiv 2004.09084 (Results, the sentence after Eq. (m)); it is
  itself pinned by ``golden/circulant_Z4_shift1.txt``.
* :func:`exact_app` computes exact a-posteriori LLRs by enumerating every word
  with ``H x = s`` (the definition of the bitwise MAP posterior).
* :func:`read_golden_*` parse the text fixtures under ``tests/golden``.
"""
from __future__ import annotations

import itertools
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def circulant(Z: int, a: int) -> np.ndarray:
    """Z x Z identity shifted right by a: entry (i, (i + a) mod Z) is one."""
    P = np.zeros((Z, Z), dtype=np.uint8)
    for i in range(Z):
        P[i, (i + a) % Z] = 1
    return P


def expand_dense(base, shifts, Z: int) -> np.ndarray:
    base = np.asarray(base)
    mb, nb = base.shape
    H = np.zeros((mb * Z, nb * Z), dtype=np.uint8)
    for l in range(mb):
        for c in range(nb):
            if base[l, c]:
                H[l * Z:(l + 1) * Z, c * Z:(c + 1) * Z] = circulant(Z, int(shifts[l, c]))
    return H


def syndrome_dense(H: np.ndarray, x: np.ndarray) -> np.ndarray:
    return ((H.astype(np.int64) @ x.astype(np.int64).T).T % 2).astype(np.uint8)


def exact_app(H: np.ndarray, llr: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Exact posterior LLRs log P(x_v = 0 | y, Hx = s) / P(x_v = 1 | y, Hx = s).

    The channel likelihood of a word x is proportional to exp(-sum_n x_n llr_n).
    Enumerates all 2^n words (n <= 20).
    """
    m, n = H.shape
    assert n <= 20
    words = np.array(list(itertools.product([0, 1], repeat=n)), dtype=np.uint8)
    synd = (words.astype(np.int64) @ H.T.astype(np.int64)) % 2
    keep = np.all(synd == s[None, :], axis=1)
    w = words[keep].astype(np.float64)
    logp = -(w @ llr.astype(np.float64))
    mx = logp.max()
    p = np.exp(logp - mx)
    p0 = ((1.0 - w) * p[:, None]).sum(axis=0)
    p1 = (w * p[:, None]).sum(axis=0)
    return np.log(p0) - np.log(p1)


def check_message_bruteforce(q, s: int) -> np.ndarray:
    """Extrinsic check message of a parity check with syndrome bit s.

    Each incoming message q_k = log P(x_k = 0) / P(x_k = 1).  For edge j the
    outgoing message is log P(xor_{k != j} x_k = s) / P(xor_{k != j} x_k = s ^ 1),
    summed over all configurations of the other bits.
    """
    q = np.asarray(q, dtype=np.float64)
    d = q.size
    p1 = 1.0 / (1.0 + np.exp(q))          # P(x_k = 1)
    p0 = 1.0 - p1
    out = np.empty(d)
    for j in range(d):
        others = [k for k in range(d) if k != j]
        num = 0.0
        den = 0.0
        for bits in itertools.product([0, 1], repeat=len(others)):
            pr = 1.0
            for k, b in zip(others, bits):
                pr *= p1[k] if b else p0[k]
            if (sum(bits) & 1) == s:
                num += pr
            else:
                den += pr
        out[j] = np.log(num) - np.log(den)
    return out


def read_matrix_file(name: str) -> np.ndarray:
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(t) for t in line.split()])
    return np.array(rows)


def read_merge_examples():
    """Returns a list of (name, base_with_minus_one, [[rows], ...])."""
    out = []
    name = None
    mat = []
    with open(os.path.join(GOLDEN, "merge_examples.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("eq "):
                name = line.split()[1]
                mat = []
            elif line.startswith("layers"):
                groups = [[int(t) for t in g.split()] for g in line[len("layers"):].split("|")]
                out.append((name, np.array(mat), groups))
            else:
                mat.append([int(t) for t in line.split()])
    return out


def read_table(name: str):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(t) for t in line.split()])
    return np.array(rows)


def tree_code(seed: int, Z: int = 1):
    """A small QC code whose base Tanner graph is a tree (so its lift is a forest).

    Returns (base, shifts).  Checks are attached one at a time; each new check
    joins exactly one existing variable and brings fresh ones, so no cycle can
    form.  Shifts are random in [0, Z).
    """
    rng = np.random.default_rng(seed)
    rows = []
    n_var = int(rng.integers(2, 4))
    rows.append(list(range(n_var)))
    for _ in range(int(rng.integers(2, 4))):
        attach = int(rng.integers(0, n_var))
        fresh = int(rng.integers(1, 3))
        rows.append([attach] + list(range(n_var, n_var + fresh)))
        n_var += fresh
    base = np.zeros((len(rows), n_var), dtype=np.int8)
    for l, cols in enumerate(rows):
        base[l, cols] = 1
    shifts = np.where(base == 1, rng.integers(0, Z, size=base.shape), 0).astype(np.int32)
    return base, shifts
