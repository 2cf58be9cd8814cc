"""Dense linear algebra over GF(2) on bit-packed rows.

Used only to *construct* decoding problems (logical operator bases, rank
checks of parity-check matrices); none of the decoder's arithmetic lives
here.  Rows are packed little-endian into uint64 words: bit ``c % 64`` of
word ``c // 64`` holds column ``c``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "pack_rows", "unpack_rows", "rref", "rank", "nullspace",
    "independent_extension", "in_rowspace", "matmul_mod2",
]


def pack_rows(a: np.ndarray) -> np.ndarray:
    """uint8/bool matrix [r, c] -> uint64 matrix [r, ceil(c/64)]."""
    a = np.asarray(a, dtype=np.uint8) & 1
    r, c = a.shape
    w = (c + 63) // 64
    padded = np.zeros((r, w * 64), dtype=np.uint8)
    padded[:, :c] = a
    bits = padded.reshape(r, w, 64).astype(np.uint64)
    shifts = np.arange(64, dtype=np.uint64)
    return np.bitwise_or.reduce(bits << shifts, axis=2) if r else np.zeros((0, w), np.uint64)


def unpack_rows(p: np.ndarray, ncols: int) -> np.ndarray:
    """Inverse of :func:`pack_rows`."""
    r, w = p.shape
    shifts = np.arange(64, dtype=np.uint64)
    bits = (p[:, :, None] >> shifts) & np.uint64(1)
    return bits.reshape(r, w * 64)[:, :ncols].astype(np.uint8)


def _bit(p: np.ndarray, col: int) -> np.ndarray:
    return (p[:, col // 64] >> np.uint64(col % 64)) & np.uint64(1)


def rref(a: np.ndarray, ncols: int | None = None):
    """Reduced row-echelon form.

    ``a`` is either a uint8 matrix or an already packed uint64 matrix (then
    ``ncols`` is required).  Returns ``(R, pivots)`` with ``R`` packed and
    holding exactly ``len(pivots)`` nonzero rows, pivot ``i`` in row ``i``.
    """
    if a.dtype != np.uint64:
        ncols = a.shape[1]
        p = pack_rows(a)
    else:
        assert ncols is not None
        p = a.copy()
    nrows = p.shape[0]
    pivots = []
    row = 0
    for col in range(ncols):
        if row >= nrows:
            break
        colbits = _bit(p[row:], col)
        hits = np.nonzero(colbits)[0]
        if hits.size == 0:
            continue
        piv = row + hits[0]
        if piv != row:
            p[[row, piv]] = p[[piv, row]]
        mask = _bit(p, col).astype(bool)
        mask[row] = False
        if mask.any():
            p[mask] ^= p[row]
        pivots.append(col)
        row += 1
    return p[:row], pivots


def rank(a: np.ndarray) -> int:
    return len(rref(a)[1])


def nullspace(a: np.ndarray) -> np.ndarray:
    """Basis (uint8 rows) of {x : a x^T = 0}."""
    a = np.asarray(a, dtype=np.uint8)
    ncols = a.shape[1]
    r, pivots = rref(a)
    dense = unpack_rows(r, ncols)
    free = [c for c in range(ncols) if c not in set(pivots)]
    basis = np.zeros((len(free), ncols), dtype=np.uint8)
    for k, f in enumerate(free):
        basis[k, f] = 1
        for i, pc in enumerate(pivots):
            if dense[i, f]:
                basis[k, pc] = 1
    return basis


def independent_extension(base: np.ndarray, cand: np.ndarray) -> np.ndarray:
    """Rows of ``cand`` that, added greedily, raise the rank of ``base``.

    Returns the selected candidate rows (uint8).  Used to pick logical
    operators: a basis of ker(H_X) that is independent of rowspace(H_Z).
    """
    ncols = base.shape[1]
    r, pivots = rref(base)
    r = list(r)
    piv = list(pivots)
    chosen = []
    for idx in range(cand.shape[0]):
        v = pack_rows(cand[idx:idx + 1])[0].copy()
        for row, pc in zip(r, piv):
            if (v[pc // 64] >> np.uint64(pc % 64)) & np.uint64(1):
                v ^= row
        nz = np.nonzero(v)[0]
        if nz.size == 0:
            continue
        w = nz[0]
        word = int(v[w])
        lead = w * 64 + (word & -word).bit_length() - 1
        # keep the reduced basis reduced
        for i, row in enumerate(r):
            if (row[lead // 64] >> np.uint64(lead % 64)) & np.uint64(1):
                r[i] = row ^ v
        r.append(v)
        piv.append(lead)
        chosen.append(idx)
    return cand[chosen]


def in_rowspace(base: np.ndarray, v: np.ndarray) -> bool:
    return rank(np.vstack([base, v[None, :]])) == rank(base)


def matmul_mod2(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """(a @ b) mod 2 for 0/1 matrices (dense or scipy sparse)."""
    prod = a @ b
    if hasattr(prod, "toarray"):
        prod = prod.toarray()
    return (np.asarray(prod) % 2).astype(np.uint8)
