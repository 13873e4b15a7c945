"""Sparse-sign embedding Omega (d x n) from a counter-based hash.  Oracle side.

The paper's embedding (Sec. 5, experimental setup; Sec. 1.1 oblivious subspace
embeddings) is a sparse-sign matrix: every column of Omega holds zeta nonzeros
equal to +-c at random rows.  Readings taken here, where the paper is silent:

* scale c = 1/sqrt(zeta), so that E||Omega x||^2 = ||x||^2 (the paper prints
  1/sqrt(d); a global scale of Omega cancels in B, b, the Ritz values and the
  residual estimates, so only the stored sketches depend on it);
* the zeta rows of a column are distinct;
* rows and signs come from SplitMix64 (Steele, Lea & Flood 2014) as follows.

Hash specification (all arithmetic on unsigned 64-bit integers, wrapping):

    gamma      = 0x9E3779B97F4A7C15
    mix(z)     : z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
                 z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31
    base_i     = mix(seed * gamma + i)                    (column i, 0-based)
    draw_{i,r} = mix(base_i + (r + 1) * gamma)            (r = 0, 1, 2, ...)
    row        = ((draw >> 32) * d) >> 32                 (in [0, d))
    sign       = -1 if (draw & 1) else +1

Slots t = 0..zeta-1 of column i take the draws in order; a draw whose row
equals the row of an earlier slot of the same column is rejected.  At most
32*zeta draws are allowed per column (with d >= 2*zeta the chance of needing
more is below 1e-30); exceeding the cap is an error.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

GAMMA = 0x9E3779B97F4A7C15
MASK = (1 << 64) - 1
MAX_DRAWS_PER_SLOT = 32


def mix64_scalar(z: int) -> int:
    """SplitMix64 output function on one Python integer."""
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def column_rows_signs_scalar(i: int, d: int, zeta: int, seed: int):
    """Rows and signs of column i, one draw at a time (reference form of the spec)."""
    base = mix64_scalar((seed * GAMMA + i) & MASK)
    rows, signs = [], []
    r = 0
    while len(rows) < zeta:
        if r >= MAX_DRAWS_PER_SLOT * zeta:
            raise RuntimeError("sketch hash: draw cap exceeded")
        h = mix64_scalar((base + (r + 1) * GAMMA) & MASK)
        r += 1
        row = ((h >> 32) * d) >> 32
        if row in rows:
            continue
        rows.append(row)
        signs.append(-1 if (h & 1) else 1)
    return rows, signs


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def rows_signs(n: int, d: int, zeta: int, seed: int):
    """All (row, sign) pairs: arrays rows[n, zeta] (int64) and signs[n, zeta] (int8).

    Vectorised over columns; the per-column procedure is exactly that of
    ``column_rows_signs_scalar``.
    """
    if not (1 <= zeta and 2 * zeta <= d):
        raise ValueError("sketch needs 1 <= zeta and d >= 2*zeta")
    g = np.uint64(GAMMA)
    with np.errstate(over="ignore"):
        base = _mix64(np.uint64(seed & MASK) * g + np.arange(n, dtype=np.uint64))
    rows = np.full((n, zeta), -1, dtype=np.int64)
    signs = np.zeros((n, zeta), dtype=np.int8)
    count = np.zeros(n, dtype=np.int64)
    active = np.arange(n)
    r = 0
    while active.size:
        if r >= MAX_DRAWS_PER_SLOT * zeta:
            raise RuntimeError("sketch hash: draw cap exceeded")
        with np.errstate(over="ignore"):
            h = _mix64(base[active] + np.uint64(r + 1) * g)
        row = (((h >> np.uint64(32)) * np.uint64(d)) >> np.uint64(32)).astype(np.int64)
        dup = (rows[active] == row[:, None]).any(axis=1)
        acc = active[~dup]
        rows[acc, count[acc]] = row[~dup]
        signs[acc, count[acc]] = np.where((h[~dup] & np.uint64(1)) != 0, -1, 1)
        count[acc] += 1
        active = active[count[active] < zeta]
        r += 1
    return rows, signs


def omega_matrix(n: int, d: int, zeta: int, seed: int) -> sp.csr_matrix:
    """Omega as a scipy sparse d x n matrix with entries sign/sqrt(zeta)."""
    rows, signs = rows_signs(n, d, zeta, seed)
    cols = np.repeat(np.arange(n), zeta)
    vals = signs.ravel().astype(np.float64) / np.sqrt(zeta)
    return sp.csr_matrix((vals, (rows.ravel(), cols)), shape=(d, n))
