"""Circuit-level detector error model (Appendix C / D): the Pauli-frame
simulation of the syndrome-extraction circuit against the matrices the paper
prints, their stated weights, the 8p/15 aggregation example, the degeneracy
identities and the weight-3 trivial-error claim."""
import numpy as np
import pytest

from bpdc_inputs import circuit


def _cols(H):
    return [H[:, j].astype(np.uint8).tobytes() for j in range(H.shape[1])]


@pytest.mark.parametrize("name,T", [("bb72", 1), ("bb72", 3), ("bb144", 2), ("bb108", 2)])
def test_simulated_model_is_the_printed_block_form(name, T):
    """Every merged mechanism of the simulated circuit is a column of the
    stacked H'_DCM of Eq. C1 and every column is one mechanism (no repeats)."""
    det, obs, pm = circuit.simulate_dem(name, T, 1e-3)
    H = circuit.dcm_block_form(name, T)
    sim = [det[k].astype(np.uint8).tobytes() for k in range(det.shape[0])]
    blk = _cols(H)
    assert len(set(sim)) == len(sim) and len(set(blk)) == len(blk)
    assert set(sim) == set(blk)
    n = circuit.bb_perms(name)[0]
    assert H.shape == ((T + 1) * n // 2, T * 5 * n + n)


def test_full_size_weights_and_counts():
    """BB[[144,12,12]], 12 rounds: M = 13 x 72 detectors, N = 12 x 720 + 144 =
    8784 mechanisms, interior row weight 35, column weight <= 6 (App. C.2)."""
    P = circuit.circuit_level_problem("bb144", 12, 1e-3)
    H = P.H.toarray()
    assert H.shape == (936, 8784)
    rw = H.sum(1)
    assert rw[72:-72].min() == rw[72:-72].max() == 35
    assert H.sum(0).max() == 6 and H.sum(0).min() >= 2
    assert P.L.shape == (12, 8784) and (P.priors > 0).all() and (P.priors < 0.5).all()


def test_aggregated_probabilities():
    """The paper's example: the bit flip of an R data qubit between the first
    and second Z-check CNOTs aggregates 4 + 4 Pauli outcomes of two CNOTs,
    8p/15 + O(p^2); exactly the odd-parity combination 2q(1-q), q = 4p/15.
    Column blocks 4-6 (L/R data between CNOTs, one Z-CNOT before and after)
    aggregate the same way; block 7 spans five CNOTs (20p/15 to first order)."""
    p = 1e-3
    P = circuit.circuit_level_problem("bb72", 3, p)
    n, h = 72, 36
    q = 4 * p / 15
    two = 2 * q * (1 - q)
    r = 5 * n   # a syndrome-extraction cycle away from the boundaries
    for blk in (4, 5, 6):
        np.testing.assert_allclose(P.priors[r + (blk - 1) * h:r + blk * h], two, rtol=1e-12)
    b7 = P.priors[r + 6 * h:r + 7 * h]
    np.testing.assert_allclose(b7, 0.5 * (1 - (1 - 2 * q) ** 5), rtol=1e-12)
    assert abs(b7[0] / p - 20 / 15) < 0.01


@pytest.mark.parametrize("name", ["bb72", "bb144", "bb108"])
def test_degeneracy_matrix_identities(name):
    """H_DDM H_DCM^T = 0 and H_DDM O^T = 0 over GF(2) (App. D), rows of weight
    6 (the X stabilizers) and 3 (the other ten row blocks)."""
    P = circuit.circuit_level_problem(name, 4, 1e-3)
    H, D, O = (m.toarray().astype(np.int64) for m in (P.H, P.D, P.L))
    assert not ((D @ H.T) % 2).any()
    assert not ((D @ O.T) % 2).any()
    assert set(np.unique(D.sum(1))) == {3, 6}
    n = circuit.bb_perms(name)[0]
    rb = (12 if name == "bb108" else 11) * n // 2
    assert D.shape[0] == 4 * rb + n // 2


def _weight3_trivial_errors(H, O):
    """All e with |e| = 3, e H^T = 0, e O^T = 0 (meet in the middle on pairs)."""
    N = H.shape[1]
    S = np.concatenate([H, O], axis=0).T.astype(np.uint8)      # [N, rows]
    key = np.packbits(S, axis=1)
    lookup = {}
    for j in range(N):
        lookup.setdefault(key[j].tobytes(), []).append(j)
    out = set()
    for a in range(N):
        x = np.packbits(S[a + 1:] ^ S[a], axis=1)
        for off in range(x.shape[0]):
            for c in lookup.get(x[off].tobytes(), ()):
                b = a + 1 + off
                if c != a and c != b:
                    out.add(tuple(sorted((a, b, c))))
    return out


@pytest.mark.slow
@pytest.mark.parametrize("name,extra,complete", [("bb72", False, True), ("bb144", False, True),
                                                 ("bb108", False, False), ("bb108", True, True)])
def test_every_weight3_trivial_error_is_a_row(name, extra, complete):
    """App. D: for w = 3 every weight-3 trivial error is a row of H_DDM for the
    BB codes, except [[108,8,10]], which needs the extra row block."""
    P = circuit.circuit_level_problem(name, 3, 1e-3, extra_block=extra)
    H, O, D = P.H.toarray(), P.L.toarray(), P.D.toarray()
    triv = _weight3_trivial_errors(H, O)
    rows = {tuple(np.nonzero(r)[0]) for r in D if r.sum() == 3}
    assert len(triv) > 0
    assert (triv <= rows) == complete, (len(triv), len(triv - rows))
    assert rows <= triv     # and every weight-3 row is a trivial error


# ---------------------------------------------------------------------------
# H_DDM for w = 4, 5 by the local-window search (App. D)

@pytest.mark.parametrize("name", ["bb72", "bb144", "bb108"])
def test_window_search_reproduces_the_printed_ddm(name):
    """Weight <= 3 trivial errors of a 3-round window, translated to every
    start round, plus the stabilizers, are exactly the rows of Eq. D2 (with
    the extra row block for [[108,8,10]])."""
    T = 5
    Dw = circuit.ddm_local_window(name, T, 3).toarray()
    Dp = circuit.ddm_block_form(name, T, name == "bb108")
    assert {tuple(np.nonzero(r)[0]) for r in Dw} == {tuple(np.nonzero(r)[0]) for r in Dp}


@pytest.mark.parametrize("w", [4, 5])
def test_window_translation_equals_direct_search(w):
    """App. D: every trivial error of weight <= 5 lies within 3 consecutive
    rounds, so the translated window patterns equal a direct search of the
    whole 5-round model."""
    from bpdc_inputs import native
    P = circuit.circuit_level_problem("bb72", 5, 1e-3)
    direct = native.trivial_errors(P.H, P.L, w)
    rows = {tuple(np.nonzero(r)[0]) for r in circuit.ddm_local_window("bb72", 5, w).toarray()}
    stab = {tuple(np.nonzero(r)[0]) for r in circuit.stabilizer_rows("bb72", 5)}
    assert direct == rows - stab


def _mitm_up_to_4(H, O):
    """Independent check: weight-3 and weight-4 trivial errors by meet in the
    middle over column pairs (column signature = its H and O column)."""
    S = np.concatenate([H, O], axis=0).T.astype(np.uint8)
    N = S.shape[0]
    key = [r.tobytes() for r in np.packbits(S, axis=1)]
    single = {}
    for j in range(N):
        single.setdefault(key[j], []).append(j)
    pairs = {}
    out = set()
    for a in range(N):
        x = np.packbits(S[a + 1:] ^ S[a], axis=1)
        for off in range(x.shape[0]):
            b = a + 1 + off
            kk = x[off].tobytes()
            pairs.setdefault(kk, []).append((a, b))
            for c in single.get(kk, ()):
                if c != a and c != b:
                    out.add(tuple(sorted((a, b, c))))
    for lst in pairs.values():
        for i in range(len(lst)):
            for k in range(i + 1, len(lst)):
                u = set(lst[i]) | set(lst[k])
                if len(u) == 4:
                    out.add(tuple(sorted(u)))
    return out


def test_native_search_matches_meet_in_the_middle():
    from bpdc_inputs import native
    P = circuit.circuit_level_problem("bb72", 2, 1e-3)
    H, O = P.H.toarray(), P.L.toarray()
    assert native.trivial_errors(P.H, P.L, 4) == _mitm_up_to_4(H, O)


def test_local_window_ddm_identities():
    P = circuit.circuit_level_problem("bb72", 4, 1e-3, w=5)
    H, D, O = (m.toarray().astype(np.int64) for m in (P.H, P.D, P.L))
    assert not ((D @ H.T) % 2).any() and not ((D @ O.T) % 2).any()
    assert set(np.unique(D.sum(1))) == {3, 4, 5, 6}
