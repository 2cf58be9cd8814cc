"""Seeded constructions of the decoding problems the paper studies.

A decoding problem is the tuple (H, D, L, priors):

* ``H`` — the matrix whose Tanner graph BP runs on: H_Z under code-capacity
  noise (Sec. II.C), the detector check matrix H_DCM otherwise (Sec. IV.A).
* ``D`` — the degeneracy matrix whose rows DC cuts along: H_X (Sec. III.A,
  Algorithm 1) or the detector degeneracy matrix H_DDM (Sec. IV.B).
* ``L`` — the logical operator matrix used for the failure test: O_Z
  (Sec. II.A/II.C) or O (Sec. IV.A).
* ``priors`` — error probabilities p_j (Eq. 8).

This module only *builds inputs*; it contains none of the decoder's
arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import gf2
from .sampler import splitmix64_hash

__all__ = [
    "Problem", "shift", "bb_matrices", "bb_code", "BB_TABLE", "gallager_regular",
    "hgp_matrices", "logical_basis", "code_capacity_problem",
    "phenomenological_matrices", "phenomenological_problem",
]


@dataclass
class Problem:
    """A decoding problem ``(H, D, L, priors)`` plus bookkeeping."""
    name: str
    H: sp.csr_matrix
    D: sp.csr_matrix
    L: sp.csr_matrix
    priors: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def M(self) -> int:
        return self.H.shape[0]

    @property
    def N(self) -> int:
        return self.H.shape[1]

    @property
    def K(self) -> int:
        return self.L.shape[0]

    @property
    def E(self) -> int:
        return int(self.H.nnz)

    def with_priors(self, priors, name: str | None = None) -> "Problem":
        pr = np.broadcast_to(np.asarray(priors, dtype=np.float64), (self.N,)).copy()
        return Problem(name or self.name, self.H, self.D, self.L, pr, dict(self.meta))


def _csr(a) -> sp.csr_matrix:
    m = sp.csr_matrix(a, dtype=np.uint8)
    m.sum_duplicates()
    m.data[:] = 1
    m.sort_indices()
    m.eliminate_zeros()
    return m


# ----------------------------------------------------------------------------
# Bivariate bicycle codes (Sec. II.B.2, Table I)
# ----------------------------------------------------------------------------

def shift(size: int) -> np.ndarray:
    """Cyclic shift S with (S)_{i,j} = 1 iff j = i + 1 mod size."""
    s = np.zeros((size, size), dtype=np.uint8)
    s[np.arange(size), (np.arange(size) + 1) % size] = 1
    return s


def _monomial(l: int, m: int, var: str, power: int) -> np.ndarray:
    x = np.kron(shift(l), np.eye(m, dtype=np.uint8))
    y = np.kron(np.eye(l, dtype=np.uint8), shift(m))
    base = x if var == "x" else y
    out = np.eye(l * m, dtype=np.uint8)
    for _ in range(power):
        out = (out @ base) % 2
    return out.astype(np.uint8)


def bb_matrices(l: int, m: int, a_terms, b_terms):
    """Return (H_X, H_Z, A_list, B_list) for the BB code defined by the terms.

    ``a_terms``/``b_terms`` are three (var, power) pairs, var in {"x", "y"};
    x = S_l (x) I_m and y = I_l (x) S_m.  H_X = [A|B], H_Z = [B^T|A^T].
    """
    A_list = [_monomial(l, m, v, p) for v, p in a_terms]
    B_list = [_monomial(l, m, v, p) for v, p in b_terms]
    A = sum(A_list) % 2
    B = sum(B_list) % 2
    hx = np.hstack([A, B]).astype(np.uint8)
    hz = np.hstack([B.T, A.T]).astype(np.uint8)
    return hx, hz, A_list, B_list


# Table I: (l, m), A = x^3 + y + y^2, B = y^3 + x + x^2.
BB_TABLE = {
    "bb72": dict(n=72, k=12, d=6, l=6, m=6),
    "bb108": dict(n=108, k=8, d=10, l=9, m=6),
    "bb144": dict(n=144, k=12, d=12, l=12, m=6),
}
BB_A = (("x", 3), ("y", 1), ("y", 2))
BB_B = (("y", 3), ("x", 1), ("x", 2))


def bb_code(name: str):
    """(H_X, H_Z) of a Table I code."""
    t = BB_TABLE[name]
    hx, hz, _, _ = bb_matrices(t["l"], t["m"], BB_A, BB_B)
    return hx, hz


# ----------------------------------------------------------------------------
# Rotated surface code (Sec. II.B.1)
# ----------------------------------------------------------------------------

def rotated_surface_code(d: int):
    """(H_X, H_Z) of the rotated surface code [[d^2, 1, d]], d odd.

    Data qubit (r, c), r, c in [0, d), has index r*d + c.  Plaquette (i, j),
    i, j in [-1, d-1], covers the qubits (i, j), (i+1, j), (i, j+1), (i+1, j+1)
    that exist; plaquettes with i + j even are Z-type, odd X-type.  Interior
    plaquettes (i, j in [0, d-2]) are all kept; on the boundary only weight-2
    X plaquettes on the top and bottom rows (i = -1, d-1) and weight-2 Z
    plaquettes on the left and right columns (j = -1, d-1) are kept.  Every
    stabilizer has weight <= 4 and every qubit is in <= 2 stabilizers of each
    type.
    """
    assert d % 2 == 1 and d >= 3
    hx, hz = [], []
    for i in range(-1, d):
        for j in range(-1, d):
            qs = [r * d + c for r in (i, i + 1) for c in (j, j + 1) if 0 <= r < d and 0 <= c < d]
            interior = 0 <= i <= d - 2 and 0 <= j <= d - 2
            ztype = (i + j) % 2 == 0
            if interior:
                (hz if ztype else hx).append(qs)
            elif len(qs) == 2:
                if not ztype and i in (-1, d - 1) and 0 <= j <= d - 2:
                    hx.append(qs)
                if ztype and j in (-1, d - 1) and 0 <= i <= d - 2:
                    hz.append(qs)
    def mat(rows):
        m = np.zeros((len(rows), d * d), dtype=np.uint8)
        for r, qs in enumerate(rows):
            m[r, qs] = 1
        return m
    return mat(hx), mat(hz)


# ----------------------------------------------------------------------------
# Hypergraph-product code of a seeded (3,4)-regular classical code
# ----------------------------------------------------------------------------

def _seeded_permutation(n: int, seed: int, stream: int) -> np.ndarray:
    """Fisher-Yates driven by the counter hash (platform independent)."""
    perm = np.arange(n)
    for i in range(n - 1, 0, -1):
        h = int(splitmix64_hash(seed, (stream << 32) | i))
        j = h % (i + 1)
        perm[i], perm[j] = perm[j], perm[i]
    return perm


def gallager_regular(n: int = 40, wc: int = 3, wr: int = 4, seed: int = 2510) -> np.ndarray:
    """Gallager (wc, wr)-regular parity-check matrix, (n*wc/wr) x n.

    wc stacked bands; each band is the n/wr x n matrix whose row i covers
    columns wr*i .. wr*i+wr-1, with the columns of the band permuted by a
    seeded permutation.  Draws are rejected until no two columns (and no two
    rows) coincide.
    """
    assert n % wr == 0
    mb = n // wr
    band = np.zeros((mb, n), dtype=np.uint8)
    for i in range(mb):
        band[i, wr * i: wr * (i + 1)] = 1
    attempt = 0
    while True:
        bands = [band[:, _seeded_permutation(n, seed, attempt * wc + b)] for b in range(wc)]
        h = np.vstack(bands)
        cols = {h[:, c].tobytes() for c in range(n)}
        rows = {h[r].tobytes() for r in range(h.shape[0])}
        if len(cols) == n and len(rows) == h.shape[0]:
            return h
        attempt += 1


def hgp_matrices(h1: np.ndarray, h2: np.ndarray):
    """Hypergraph product: H_X = [H1 (x) I_n2 | I_m1 (x) H2^T],
    H_Z = [I_n1 (x) H2 | H1^T (x) I_m2]."""
    m1, n1 = h1.shape
    m2, n2 = h2.shape
    hx = sp.hstack([sp.kron(h1, sp.eye(n2, dtype=np.uint8)),
                    sp.kron(sp.eye(m1, dtype=np.uint8), h2.T)])
    hz = sp.hstack([sp.kron(sp.eye(n1, dtype=np.uint8), h2),
                    sp.kron(h1.T, sp.eye(m2, dtype=np.uint8))])
    return _csr(hx), _csr(hz)


# ----------------------------------------------------------------------------
# Logical operators (Sec. II.A: O_Z H_X^T = 0)
# ----------------------------------------------------------------------------

def logical_basis(hx, hz) -> np.ndarray:
    """O_Z: rows spanning ker(H_X) that are independent of rowspace(H_Z).

    The paper states the defining property O_Z H_X^T = 0 but gives no
    construction; any such basis yields the same failure flag.
    """
    hx = hx.toarray() if sp.issparse(hx) else np.asarray(hx)
    hz = hz.toarray() if sp.issparse(hz) else np.asarray(hz)
    ker = gf2.nullspace(hx.astype(np.uint8))
    return gf2.independent_extension(hz.astype(np.uint8), ker)


def code_capacity_problem(hx, hz, p: float, name: str, oz=None) -> Problem:
    """Bit-flip decoding under code-capacity noise: H = H_Z, D = H_X, L = O_Z,
    p_i = p for every qubit (Sec. III.B)."""
    if oz is None:
        oz = logical_basis(hx, hz)
    n = hz.shape[1]
    return Problem(name, _csr(hz), _csr(hx), _csr(oz), np.full(n, float(p)),
                   meta=dict(kind="code_capacity", p=float(p)))


# ----------------------------------------------------------------------------
# Phenomenological noise (Sec. IV.C, Eq. 12-15)
# ----------------------------------------------------------------------------

def phenomenological_matrices(hx, hz, oz, T: int):
    """(H_DCM, H_DDM, O, is_meas) for T noisy rounds plus one perfect round.

    Column blocks, in order: D_1, M_1, D_2, M_2, ..., D_T, M_T, D_{T+1}
    (D_t = data errors before round t, M_t = measurement errors of round t).
    Row blocks of H_DCM: detectors of rounds 1..T+1 (Eq. 6).
    H_DCM stacks T staggered copies of [[H_Z, I], [0, I]] plus a final H_Z.
    H_DDM stacks T staggered copies of [[H_X, 0, 0], [I, H_Z^T, I]] over
    (D_t, M_t, D_{t+1}) plus a final H_X.  O puts O_Z on every data block.
    """
    hx = np.asarray(hx, dtype=np.uint8)
    hz = np.asarray(hz, dtype=np.uint8)
    oz = np.asarray(oz, dtype=np.uint8)
    mz, n = hz.shape
    mx = hx.shape[0]
    blk = n + mz
    N = T * blk + n
    Mdet = mz * (T + 1)

    def dcol(t):  # t = 1..T+1
        return (t - 1) * blk

    def mcol(t):  # t = 1..T
        return (t - 1) * blk + n

    dcm = sp.lil_matrix((Mdet, N), dtype=np.uint8)
    Imz = np.eye(mz, dtype=np.uint8)
    for t in range(1, T + 1):
        r0 = (t - 1) * mz
        dcm[r0:r0 + mz, dcol(t):dcol(t) + n] = hz
        dcm[r0:r0 + mz, mcol(t):mcol(t) + mz] = Imz
        dcm[r0 + mz:r0 + 2 * mz, mcol(t):mcol(t) + mz] = Imz
    r0 = T * mz
    dcm[r0:r0 + mz, dcol(T + 1):dcol(T + 1) + n] = hz

    rows_per = mx + n
    ddm = sp.lil_matrix((T * rows_per + mx, N), dtype=np.uint8)
    In = np.eye(n, dtype=np.uint8)
    for t in range(1, T + 1):
        r0 = (t - 1) * rows_per
        ddm[r0:r0 + mx, dcol(t):dcol(t) + n] = hx
        ddm[r0 + mx:r0 + rows_per, dcol(t):dcol(t) + n] = In
        ddm[r0 + mx:r0 + rows_per, mcol(t):mcol(t) + mz] = hz.T
        ddm[r0 + mx:r0 + rows_per, dcol(t + 1):dcol(t + 1) + n] = In
    r0 = T * rows_per
    ddm[r0:r0 + mx, dcol(T + 1):dcol(T + 1) + n] = hx

    k = oz.shape[0]
    obs = sp.lil_matrix((k, N), dtype=np.uint8)
    for t in range(1, T + 2):
        obs[:, dcol(t):dcol(t) + n] = oz

    is_meas = np.zeros(N, dtype=bool)
    for t in range(1, T + 1):
        is_meas[mcol(t):mcol(t) + mz] = True
    return _csr(dcm), _csr(ddm), _csr(obs), is_meas


def phenomenological_problem(hx, hz, T: int, p: float, q: float | None = None,
                             name: str = "phen", oz=None) -> Problem:
    """Phenomenological decoding problem: data errors with probability p
    before every round, measurement flips with probability q (= p by default)."""
    if q is None:
        q = p
    if oz is None:
        oz = logical_basis(hx, hz)
    dcm, ddm, obs, is_meas = phenomenological_matrices(hx, hz, oz, T)
    priors = np.where(is_meas, float(q), float(p))
    return Problem(name, dcm, ddm, obs, priors,
                   meta=dict(kind="phenomenological", T=T, p=float(p), q=float(q)))
