"""Circuit-level detector error model of a BB code memory experiment.

Appendix C.1 gives the syndrome-extraction circuit (one round = eight steps
of CNOTs, initialisations, idles and measurements on n data, n/2 X-ancilla
and n/2 Z-ancilla qubits, after a step 0 that prepares the Z ancillas) and
the noise: after every operation, idle -> X, Y or Z with p/3 each, CNOT ->
one of the 15 non-identity two-qubit Paulis with p/15 each, a wrong
preparation with p, a flipped measurement with p.  Appendix C.2 keeps only
the Z-type outcomes (X errors are decoded) and merges every set of fault
events with the same detector and logical effect into one mechanism whose
probability is that of an odd number of its events.

This module derives that model by Pauli-frame simulation: every fault
outcome with an X part is injected into its own frame, frames are pushed
through the remaining circuit (an X on a CNOT control spreads to the
target; a reset clears the qubit), and each Z measurement records the frame
of its ancilla.  Detectors are D_1 = m_1, D_t = m_t + m_(t-1) for the T noisy
rounds and D_(T+1) = H_Z e_data + m_T for the final noiseless data
measurement; the observable is O_Z e_data.  Outcomes of one channel are
mutually exclusive (their probabilities add); distinct channels are
independent (odd-parity combination).

It also writes out the block forms printed in the paper, H'_DCM (Eq. C1) and
H'_DDM for w = 3 (Eq. D2), stacked over T rounds; the tests check the
simulated model against them.  Nothing here is decoder arithmetic.
"""
from __future__ import annotations

import functools

import numpy as np
import scipy.sparse as sp

from . import codes

__all__ = ["bb_perms", "syndrome_circuit", "simulate_dem", "dcm_block_form", "ddm_block_form",
           "stabilizer_rows", "window_trivial_errors", "ddm_local_window", "circuit_level_problem"]


def bb_perms(name: str):
    """(n, A1..A3, B1..B3) of a Table I code as index maps i -> Pi(i), where
    Pi(i) is the column of the one in row i of the monomial matrix Pi."""
    t = codes.BB_TABLE[name]
    _, _, A_list, B_list = codes.bb_matrices(t["l"], t["m"], codes.BB_A, codes.BB_B)
    to_map = lambda P: np.argmax(P, axis=1).astype(np.int64)   # noqa: E731
    return t["n"], [to_map(P) for P in A_list], [to_map(P) for P in B_list]


def _inv(perm):
    out = np.empty_like(perm)
    out[perm] = np.arange(len(perm))
    return out


# Operation codes of the circuit.
CNOT, IDLE, INITZ, INITX, MEASZ, MEASX = range(6)


def syndrome_circuit(name: str, T: int):
    """The Appendix C.1 circuit as a list of steps; a step is a list of
    (op, qubit_a, qubit_b) with qubit_b = -1 for one-qubit operations.
    Qubits: L_i = i, R_i = n/2 + i, X_i = n + i, Z_i = 3n/2 + i (i < n/2).
    Returns (steps, n)."""
    n, (A1, A2, A3), (B1, B2, B3) = bb_perms(name)
    h = n // 2
    L = lambda i: int(i)                  # noqa: E731
    R = lambda i: h + int(i)              # noqa: E731
    X = lambda i: n + int(i)              # noqa: E731
    Z = lambda i: n + h + int(i)          # noqa: E731
    # Pi^T(i) = Pi^{-1}(i) for a permutation matrix
    A1t, A2t, A3t, B1t, B2t, B3t = (_inv(P) for P in (A1, A2, A3, B1, B2, B3))
    rng = range(h)
    step0 = [(IDLE, X(i), -1) for i in rng] + [(INITZ, Z(i), -1) for i in rng] + \
            [(IDLE, L(i), -1) for i in rng] + [(IDLE, R(i), -1) for i in rng]
    rnd = [
        [(INITX, X(i), -1) for i in rng] + [(CNOT, R(A1t[i]), Z(i)) for i in rng] + [(IDLE, L(i), -1) for i in rng],
        [(CNOT, X(i), L(A2[i])) for i in rng] + [(CNOT, R(A3t[i]), Z(i)) for i in rng],
        [(CNOT, X(i), R(B2[i])) for i in rng] + [(CNOT, L(B1t[i]), Z(i)) for i in rng],
        [(CNOT, X(i), R(B1[i])) for i in rng] + [(CNOT, L(B2t[i]), Z(i)) for i in rng],
        [(CNOT, X(i), R(B3[i])) for i in rng] + [(CNOT, L(B3t[i]), Z(i)) for i in rng],
        [(CNOT, X(i), L(A1[i])) for i in rng] + [(CNOT, R(A2t[i]), Z(i)) for i in rng],
        [(CNOT, X(i), L(A3[i])) for i in rng] + [(MEASZ, Z(i), -1) for i in rng] + [(IDLE, R(i), -1) for i in rng],
        [(MEASX, X(i), -1) for i in rng] + [(INITZ, Z(i), -1) for i in rng] + [(IDLE, L(i), -1) for i in rng] +
        [(IDLE, R(i), -1) for i in rng],
    ]
    return [step0] + rnd * T, n


def _fault_outcomes(steps, p):
    """Every outcome with an X part (or a flipped Z measurement) of every
    noise channel: (step, channel, X-flipped qubits, flipped measurement,
    probability).  Measurements are numbered in circuit order."""
    out = []
    ch = 0
    meas = 0
    for s, ops in enumerate(steps):
        for op, a, b in ops:
            if op == IDLE:                      # X or Y: p/3 each
                out.append((s, ch, (a,), -1, 2.0 * p / 3.0))
            elif op == CNOT:                    # 4 of the 15 Paulis for each X pattern
                for qs in ((a,), (b,), (a, b)):
                    out.append((s, ch, qs, -1, 4.0 * p / 15.0))
            elif op == INITZ:                   # |1> instead of |0>
                out.append((s, ch, (a,), -1, p))
            elif op == MEASZ:                   # flipped outcome
                out.append((s, ch, (), meas, p))
                meas += 1
            # INITX (|->) and MEASX flips have no X part on the Z record
            ch += 1
    return out, meas


def simulate_dem(name: str, T: int, p: float):
    """Merged circuit-level mechanisms: (detector matrix [mech, (T+1) n/2],
    observable matrix [mech, k], probabilities [mech]) as bool / float arrays."""
    steps, n = syndrome_circuit(name, T)
    h = n // 2
    hx, hz, oz = _bb(name)
    faults, n_meas = _fault_outcomes(steps, p)
    F = len(faults)
    nq = 2 * n
    frame = np.zeros((F, nq), dtype=bool)
    rec = np.zeros((F, n_meas), dtype=bool)
    by_step = {}
    for f, (s, _, qs, mi, _) in enumerate(faults):
        by_step.setdefault(s, []).append((f, qs, mi))
    meas = 0
    for s, ops in enumerate(steps):
        ctl = np.array([a for op, a, b in ops if op == CNOT], dtype=np.int64)
        tgt = np.array([b for op, a, b in ops if op == CNOT], dtype=np.int64)
        if ctl.size:                            # CNOTs of one step act on disjoint qubits
            frame[:, tgt] ^= frame[:, ctl]
        for op, a, _ in ops:
            if op in (INITZ, INITX):
                frame[:, a] = False
            elif op == MEASZ:
                rec[:, meas] = frame[:, a]
                meas += 1
        for f, qs, mi in by_step.get(s, ()):    # noise after the step's operations
            for q in qs:
                frame[f, q] ^= True
            if mi >= 0:
                rec[f, mi] ^= True
    m = rec.reshape(F, T, h)
    det = np.empty((F, T + 1, h), dtype=bool)
    det[:, 0] = m[:, 0]
    det[:, 1:T] = m[:, 1:] ^ m[:, :-1]
    data = frame[:, :n].astype(np.int64)
    det[:, T] = ((data @ hz.T.astype(np.int64)) % 2).astype(bool) ^ m[:, T - 1]
    obs = ((data @ oz.T.astype(np.int64)) % 2).astype(bool)
    sig = np.concatenate([det.reshape(F, -1), obs], axis=1)
    # merge: exclusive outcomes of one channel add, channels combine by odd parity
    keys = np.packbits(sig, axis=1)
    keys = np.ascontiguousarray(keys).view(np.dtype((np.void, keys.shape[1]))).ravel()
    uniq, first, inv = np.unique(keys, return_index=True, return_inverse=True)
    chan = np.array([c for _, c, _, _, _ in faults])
    prob = np.array([q for _, _, _, _, q in faults])
    per = {}
    for f in range(F):
        k = (int(inv[f]), int(chan[f]))
        per[k] = per.get(k, 0.0) + prob[f]
    keep_prob = np.ones(len(uniq))              # product of (1 - 2 p_channel)
    for (u, _), q in per.items():
        keep_prob[u] *= 1.0 - 2.0 * q
    pm = 0.5 * (1.0 - keep_prob)
    sig_u = sig[first]
    nz = sig_u.any(1)
    det_u = sig_u[nz, : (T + 1) * h]
    obs_u = sig_u[nz, (T + 1) * h:]
    assert det_u.any(1).all(), "a logical error that no detector sees"
    return det_u, obs_u, pm[nz]


@functools.lru_cache(maxsize=None)
def _bb(name):
    hx, hz = codes.bb_code(name)
    return hx, hz, codes.logical_basis(hx, hz)


def _perm_mat(perm):
    k = len(perm)
    M = np.zeros((k, k), dtype=np.int64)
    M[np.arange(k), perm] = 1
    return M


def _blocks(name):
    n, A, B = bb_perms(name)
    A1, A2, A3 = (_perm_mat(P) for P in A)
    B1, B2, B3 = (_perm_mat(P) for P in B)
    return n, dict(A1=A1, A2=A2, A3=A3, B1=B1, B2=B2, B3=B3, A=A1 + A2 + A3, B=B1 + B2 + B3,
                   Ab1=A2 + A3, Ab2=A3 + A1, Ab3=A1 + A2, Bb1=B2 + B3, Bb2=B3 + B1, Bb3=B1 + B2,
                   I=np.eye(n // 2, dtype=np.int64))


def dcm_block_form(name: str, T: int) -> np.ndarray:
    """H_DCM of Eq. C1: T copies of H'_DCM (n x 5n, ten column blocks of n/2)
    stacked with a shift of n/2 rows and 5n columns, then H_Z = (B^T | A^T) on
    the last n columns and last n/2 rows."""
    n, b = _blocks(name)
    h = n // 2
    t = lambda X: X.T                           # noqa: E731
    Z = np.zeros((h, h), dtype=np.int64)
    top = [t(b["B"]), t(b["A"]), b["I"], t(b["Bb1"]), t(b["Ab1"]), t(b["B3"]), t(b["A2"]),
           t(b["A2"]) @ t(b["Bb2"]), t(b["A2"]) @ t(b["B3"]), Z]
    bot = [Z, Z, b["I"], t(b["B1"]), t(b["A1"]), t(b["Bb3"]), t(b["Ab2"]),
           t(b["Ab2"]) @ t(b["B2"]), t(b["Ab2"]) @ t(b["Bb3"]), t(b["Ab2"]) @ t(b["B"])]
    Hp = np.block([top, bot]) % 2
    M, N = (T + 1) * h, T * 5 * n + n
    H = np.zeros((M, N), dtype=np.uint8)
    for r in range(T):
        H[r * h:(r + 2) * h, r * 5 * n:(r + 1) * 5 * n] ^= Hp.astype(np.uint8)
    H[T * h:, T * 5 * n:] ^= (np.hstack([t(b["B"]), t(b["A"])]) % 2).astype(np.uint8)
    return H


def ddm_block_form(name: str, T: int, extra_block: bool = False) -> np.ndarray:
    """H_DDM for w = 3 (Eq. D2): T copies of H'_DDM (11n/2 x 6n, twelve column
    blocks of n/2: the round's 5n columns plus the next round's first n)
    stacked with a shift of 11n/2 rows and 5n columns, then H_X = (A | B) on
    the last n columns.  ``extra_block`` appends the row block the paper adds
    for the [[108,8,10]] code."""
    n, b = _blocks(name)
    h = n // 2
    I = b["I"]
    Z = np.zeros((h, h), dtype=np.int64)

    def row(**cols):
        out = [Z] * 12
        for k, v in cols.items():
            out[int(k[1:]) - 1] = v
        return out
    rows = [
        row(c1=b["A"], c2=b["B"]),
        row(c1=I, c3=b["B1"], c4=I),
        row(c2=I, c3=b["A1"], c5=I),
        row(c3=b["B2"], c4=I, c6=I),
        row(c3=b["A3"], c5=I, c7=I),
        row(c3=b["B3"], c6=I, c11=I),
        row(c3=b["A2"], c7=I, c12=I),
        row(c1=b["A2"], c7=b["B2"], c8=I),
        row(c7=b["B1"], c8=I, c9=I),
        row(c7=b["B3"], c9=I, c10=I),
        row(c10=I, c11=b["Ab2"]),
    ]
    if extra_block:
        A1, A3 = b["A1"], b["A3"]
        rows.append(row(c10=(A1 @ A1 @ A3 + A1 @ A3 @ A3 + I)))
    Dp = (np.block(rows) % 2).astype(np.uint8)
    rb = Dp.shape[0]
    M, N = T * rb + h, T * 5 * n + n
    D = np.zeros((M, N), dtype=np.uint8)
    for r in range(T):
        D[r * rb:(r + 1) * rb, r * 5 * n:r * 5 * n + 6 * n] ^= Dp
    D[T * rb:, T * 5 * n:] ^= (np.hstack([b["A"], b["B"]]) % 2).astype(np.uint8)
    return D


@functools.lru_cache(maxsize=None)
def _dem_in_block_order(name: str, T: int, p: float):
    """Simulated mechanisms ordered like the columns of Eq. C1."""
    det, obs, pm = simulate_dem(name, T, p)
    H = dcm_block_form(name, T)
    col_key = {H[:, j].tobytes(): j for j in range(H.shape[1])}
    order = np.full(H.shape[1], -1, dtype=np.int64)
    for k in range(det.shape[0]):
        j = col_key.get(det[k].astype(np.uint8).tobytes())
        if j is None or order[j] >= 0:
            raise ValueError("simulated mechanism outside the block form (or repeated)")
        order[j] = k
    if (order < 0).any():
        raise ValueError("block-form column without a simulated mechanism")
    return H, obs[order].astype(np.uint8), pm[order]


def stabilizer_rows(name: str, T: int) -> np.ndarray:
    """The X-stabilizer rows of H_DDM: H_X = (A | B) on the data columns before
    every round and on the final data columns."""
    n, b = _blocks(name)
    h = n // 2
    N = T * 5 * n + n
    hx = (np.hstack([b["A"], b["B"]]) % 2).astype(np.uint8)
    D = np.zeros(((T + 1) * h, N), dtype=np.uint8)
    for r in range(T + 1):
        D[r * h:(r + 1) * h, r * 5 * n:r * 5 * n + n] = hx
    return D


@functools.lru_cache(maxsize=None)
def window_trivial_errors(name: str, w: int, t_loc: int = 3) -> tuple:
    """Trivial errors of weight <= w of the t_loc-round model (App. D's local
    temporal window), as sorted column tuples of that model."""
    from . import native
    H = dcm_block_form(name, t_loc)
    _, O, _ = _dem_in_block_order(name, t_loc, 1e-3)
    return tuple(sorted(native.trivial_errors(H, O.T, w)))


def ddm_local_window(name: str, T: int, w: int, t_loc: int = 3) -> sp.csr_matrix:
    """H_DDM from the stabilizers and every trivial error of weight <= w found
    in a t_loc-round window, translated to each of the T - t_loc + 1 start
    rounds (App. D).  Columns of the window's model map to the full model by a
    shift of 5n per round (the window's final data block becomes the next
    round's data-before-round block, or the final block)."""
    n = bb_perms(name)[0]
    if T < t_loc:
        raise ValueError("T must be at least t_loc")
    pats = window_trivial_errors(name, w, t_loc)
    rows = {tuple(np.nonzero(r)[0]) for r in stabilizer_rows(name, T)}
    for r in range(T - t_loc + 1):
        for pat in pats:
            rows.add(tuple(c + 5 * n * r for c in pat))
    rows = sorted(rows)
    N = T * 5 * n + n
    ptr = np.cumsum([0] + [len(r) for r in rows])
    col = np.fromiter((c for r in rows for c in r), dtype=np.int64, count=int(ptr[-1]))
    return sp.csr_matrix((np.ones(len(col), dtype=np.uint8), col, ptr), shape=(len(rows), N))


def circuit_level_problem(name: str, T: int, p: float, extra_block: bool | None = None,
                          w: int = 3) -> codes.Problem:
    """(H_DCM, H_DDM, O, priors) of the circuit-level model: the simulated
    mechanisms in the column order of Eq. C1 (verified equal as sets); D from
    Eq. D2 for w = 3, else from the local-window search for weight <= w."""
    H, O, pm = _dem_in_block_order(name, T, float(p))
    if extra_block is None:
        extra_block = name == "bb108"
    D = ddm_block_form(name, T, extra_block) if w == 3 else ddm_local_window(name, T, w)
    return codes.Problem(f"{name}_circuit_T{T}_p{p:g}_w{w}", codes._csr(H), codes._csr(D), codes._csr(O.T),
                         pm.astype(np.float64), dict(T=T, p=p, w=w, model="circuit"))
