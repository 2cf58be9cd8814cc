"""Pins for the seeded input generators: code constructions against Table I and
the identities of Sec. II.A / IV, and the counter-based sampler."""
import os

import numpy as np
import pytest

import bpdc_inputs as bi
from bpdc_inputs import codes, gf2, sampler

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.mark.parametrize("row", _table("table1_bb_codes.txt"), ids=lambda r: r[0])
def test_bb_codes_match_table1(row):
    name, n, k, _d, l, m = row[0], *map(int, row[1:])
    hx, hz = codes.bb_code(name)
    assert hx.shape == (l * m, n) and hz.shape == (l * m, n)
    # row weight r = 6, column weight c = 3 (Sec. II.B.2)
    assert set(hx.sum(1)) == {6} and set(hx.sum(0)) == {3}
    assert set(hz.sum(1)) == {6} and set(hz.sum(0)) == {3}
    # commutation H_Z H_X^T = 0 (Sec. II.A)
    assert not ((hz.astype(int) @ hx.T.astype(int)) % 2).any()
    # k = n - rank H_X - rank H_Z (Table I)
    assert n - gf2.rank(hx) - gf2.rank(hz) == k
    oz = codes.logical_basis(hx, hz)
    assert oz.shape[0] == k
    # O_Z H_X^T = 0 and O_Z independent of rowspace(H_Z)
    assert not ((oz.astype(int) @ hx.T.astype(int)) % 2).any()
    assert gf2.rank(np.vstack([hz, oz])) == gf2.rank(hz) + k


def test_bb_shift_definition():
    # (S_l)_{i,j} = 1 iff j = i + 1 mod l; x^l = y^m = I (Sec. II.B.2)
    s = codes.shift(5)
    assert s[0, 1] == 1 and s[4, 0] == 1 and s.sum() == 5
    l, m = 6, 6
    x = codes._monomial(l, m, "x", 1)
    y = codes._monomial(l, m, "y", 1)
    assert ((x @ y) % 2 == (y @ x) % 2).all()
    assert (codes._monomial(l, m, "x", l) == np.eye(l * m)).all()
    assert (codes._monomial(l, m, "y", m) == np.eye(l * m)).all()


def test_hgp_construction():
    h, hx, hz, oz = bi._hgp()
    assert h.shape == (30, 40)
    assert set(h.sum(0)) == {3} and set(h.sum(1)) == {4}
    assert hx.shape == (1200, 2500) and hz.shape == (1200, 2500)
    assert hz.nnz == 8400 and set(np.asarray(hz.sum(1)).ravel()) == {7}
    assert not gf2.matmul_mod2(hz, hx.T).any()
    r = gf2.rank(h)
    k_expected = (40 - r) ** 2 + (30 - r) ** 2      # k1*k2 + k1T*k2T
    assert oz.shape[0] == k_expected
    assert not gf2.matmul_mod2(oz, hx.T.toarray()).any()


def test_phenomenological_bb144_shapes_and_identities():
    P = bi.phenomenological_bb_problem("bb144", 12, 0.01)
    n, mz, T = 144, 72, 12
    assert P.H.shape == (mz * (T + 1), T * (n + mz) + n) == (936, 2736)
    assert P.H.nnz == 7344
    # row weight <= r + 2, column weight <= c (Sec. IV.C)
    assert np.asarray(P.H.sum(1)).max() == 8 and np.asarray(P.H.sum(0)).max() == 3
    assert P.D.shape == (T * (n + 72) + 72, 2736) and P.D.nnz == 14256
    # H_DDM rows and columns weigh at most max{r, c + 2} = 6 (Sec. IV.C)
    assert np.asarray(P.D.sum(1)).max() == 6 and np.asarray(P.D.sum(0)).max() == 6
    # H_DDM H_DCM^T = 0 and H_DDM O^T = 0 (Sec. IV.B)
    assert not gf2.matmul_mod2(P.D, P.H.T).any()
    assert not gf2.matmul_mod2(P.D, P.L.T).any()
    # priors: data p, measurement q
    assert P.priors.shape == (2736,) and np.isclose(P.priors, 0.01).all()


def test_phenomenological_detector_semantics():
    """A data error before round t flips only round-t detectors; a measurement
    error in round t flips detectors of rounds t and t+1 (Eq. 6)."""
    hx, hz = codes.bb_code("bb72")
    oz = codes.logical_basis(hx, hz)
    T = 3
    dcm, ddm, obs, is_meas = codes.phenomenological_matrices(hx, hz, oz, T)
    n, mz = 72, 36
    dcm = dcm.toarray()
    # simulate measurements m_{i,t} directly and form detectors
    rng = np.random.default_rng(1)
    for _ in range(20):
        e = (rng.random(dcm.shape[1]) < 0.05).astype(np.uint8)
        data_acc = np.zeros(n, np.uint8)
        meas = np.zeros((T + 1, mz), np.uint8)
        for t in range(1, T + 2):
            d0 = (t - 1) * (n + mz)
            data_acc ^= e[d0:d0 + n]
            meas[t - 1] = (hz.astype(int) @ data_acc) % 2
            if t <= T:
                meas[t - 1] ^= e[d0 + n:d0 + n + mz]
        det = meas.copy()
        det[1:] ^= meas[:-1]
        assert (det.ravel() == (dcm.astype(int) @ e) % 2).all()
        # logical readout at the end: O_Z applied to the accumulated data error
        assert ((oz.astype(int) @ data_acc) % 2 == (obs.toarray().astype(int) @ e) % 2).all()


def test_splitmix64_reference_stream():
    for c, v in _table("splitmix64.txt"):
        assert int(sampler.splitmix64_hash(0, int(c))) == int(v, 16)


def test_sampler_rates_and_determinism():
    pr = np.array([0.0, 0.01, 0.1, 0.5])
    e = sampler.sample_errors(pr, seed=7, shot_offset=0, B=200000)
    assert e[:, 0].sum() == 0
    for j in (1, 2, 3):
        mean = e[:, j].mean()
        sigma = np.sqrt(pr[j] * (1 - pr[j]) / e.shape[0])
        assert abs(mean - pr[j]) < 5 * sigma
    # shot offsets address the same stream
    e2 = sampler.sample_errors(pr, seed=7, shot_offset=1000, B=10)
    assert (e2 == e[1000:1010]).all()


def test_pack_roundtrip():
    rng = np.random.default_rng(0)
    for n in (1, 31, 32, 33, 100):
        bits = (rng.random((5, n)) < 0.5).astype(np.uint8)
        w = sampler.pack_bits(bits)
        assert w.shape == (5, (n + 31) // 32)
        assert (sampler.unpack_bits(w, n) == bits).all()
