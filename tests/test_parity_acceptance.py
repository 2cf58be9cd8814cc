"""The GPU-vs-oracle acceptance rules of tests/parity.py, checked on the CPU.

A rule that accepts everything proves nothing, and one that rejects rounding
cannot be met by any FP32 decoder.  So the rules are exercised with stand-ins
for the GPU built from the oracle itself: its output on priors perturbed by
1e-6 relative (a rounding-sized change of the computation) must pass, and its
output with a planted mistake (min-sum scale 0.63 instead of 0.625; priors
off by 0.2 % in product-sum) must fail.  The cut-set logic (which cuts the
selection rule of Algorithm 1 can make when values sit at the edge of the tie
window) is checked on hand-built rows."""
import numpy as np
import pytest
import scipy.sparse as sp

import bpdc_inputs as bi
from bpdc_inputs.sampler import sample_shots
import parity

SEED = 0x2510086950


def _winners(rows, post, tie_rel=1e-5, margin=1e-6, shot=0, hash64=lambda k, c: c):
    D = sp.csr_matrix((np.ones(sum(len(r) for r in rows)), np.concatenate(rows),
                       np.cumsum([0] + [len(r) for r in rows])), shape=(len(rows), len(post)))
    return parity.possible_winners(D, np.asarray(post, float), tie_rel, margin, shot, 0, hash64)


def test_possible_winners_single_candidate():
    # a clear maximum is the only winner
    w = _winners([[0, 1, 2]], [1.0, 5.0, 2.0])
    assert w == [{1}]


def test_possible_winners_window_edge_counts_both_ways():
    # L_max = 10 (window 1e-4 below it); column 2 sits 1e-10 from the edge, so
    # the candidate set is {1} or {1, 2}: rank h mod |set| with h = row index
    # (the stand-in hash) = 0 picks column 1 either way; with h = 1 the two
    # sets pick 1 and 2
    post = [1.0, 10.0, 10.0 - 1e-4 - 1e-10]
    assert _winners([[0, 1, 2]], post) == [{1}]
    assert _winners([[0, 1, 2]], post, hash64=lambda k, c: 1) == [{1, 2}]


def test_cut_is_possible():
    win = [{1}, {1, 2}, {3}]
    assert parity.cut_is_possible(win, np.array([0, 1, 0, 1]))        # row 1 picks 1
    assert parity.cut_is_possible(win, np.array([0, 1, 1, 1]))        # row 1 picks 2
    assert not parity.cut_is_possible(win, np.array([0, 1, 0, 0]))    # row 3 uncut
    assert not parity.cut_is_possible(win, np.array([1, 1, 0, 1]))    # 0 is nobody's pick
    # two cut variables that only one row can supply cannot both come from it
    assert not parity.cut_is_possible([{1, 2}], np.array([0, 1, 1]))


def _fake(oracle_mod, P, s, opts, eps=None, mutant=None):
    if mutant is not None:
        out = mutant()
    else:
        rng = np.random.default_rng(7)
        Q = P.with_priors(P.priors * (1 + eps * rng.standard_normal(P.N)))
        out = oracle_mod.decode_batch(Q, s, 0, opts, want_post=True)
    out["post"] = out["post"].astype(np.float32).astype(np.float64)   # FP32 outputs
    return out


@pytest.mark.parametrize("rule", ["min-sum", "product-sum"])
def test_rounding_sized_perturbation_passes(oracle_mod, rule):
    if rule == "min-sum":
        P, opts = bi.bb_problem("bb72", 0.06), oracle_mod.Options(alpha=0.625, max_iter=50)
    else:
        P, opts = bi.bb_problem("bb72", 0.05), oracle_mod.Options(variant=1, max_iter=50)
    _, s, o = sample_shots(P, SEED, 0, 1500)
    rep = parity.compare(oracle_mod, P, s, 0, opts, _fake(oracle_mod, P, s, opts, eps=1e-6), obs=o)
    print(parity.summary(rep))
    assert rep["unmatched_well"] == 0
    assert rep["unmatched_ill"] <= 0.01 * rep["B"]
    assert rep["posterior"]["failed"] == 0 and rep["posterior"]["inf_mismatch"] == 0
    assert rep["same"] >= 0.95 * rep["B"]


def test_planted_mistakes_fail(oracle_mod):
    P, opts = bi.bb_problem("bb72", 0.06), oracle_mod.Options(alpha=0.625, max_iter=50)
    _, s, o = sample_shots(P, SEED, 0, 1500)
    wrong_scale = oracle_mod.Options(alpha=0.63, max_iter=50)
    rep = parity.compare(oracle_mod, P, s, 0, opts,
                         _fake(oracle_mod, P, s, opts, mutant=lambda: oracle_mod.decode_batch(
                             P, s, 0, wrong_scale, want_post=True)), obs=o)
    assert rep["unmatched_well"] > 50 and rep["posterior"]["failed"] > 10000
    # product-sum with priors 0.2 % off: outcomes mostly survive, posteriors do not
    P2, opts2 = bi.bb_problem("bb72", 0.05), oracle_mod.Options(variant=1, max_iter=50)
    _, s2, _ = sample_shots(P2, SEED, 0, 1500)
    shifted = P2.with_priors(P2.priors * 1.002)
    rep2 = parity.compare(oracle_mod, P2, s2, 0, opts2,
                          _fake(oracle_mod, P2, s2, opts2, mutant=lambda: oracle_mod.decode_batch(
                              shifted, s2, 0, opts2, want_post=True)))
    assert rep2["posterior"]["failed"] > 10000
