"""Pins of the FP64 oracle to facts that do not come from the oracle itself:
exact marginals / min-energies on trees (BP is exact on trees), the decoding
invariants of Sec. II.C and Algorithm 1, Algorithm 1 == Algorithm 2
(Sec. III.A), and the tie-break definition."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

import bpdc_inputs as bi
from bpdc_inputs.codes import Problem
from bpdc_inputs.sampler import sample_shots, syndromes


def random_tree_problem(rng, n_checks, max_extra=3):
    """Random tree-shaped Tanner graph: every check has degree >= 2."""
    edges = []
    nvar = 1
    for c in range(n_checks):
        anchor = int(rng.integers(nvar))
        new = int(rng.integers(1, max_extra + 1))
        vs = [anchor] + list(range(nvar, nvar + new))
        nvar += new
        edges += [(c, v) for v in vs]
    H = np.zeros((n_checks, nvar), np.uint8)
    for c, v in edges:
        H[c, v] = 1
    # shuffle variable labels so the tree is not in construction order
    perm = rng.permutation(nvar)
    H = H[:, perm]
    p = rng.uniform(0.02, 0.45, size=nvar)
    Z = sp.csr_matrix((0, nvar), dtype=np.uint8)
    return Problem("tree", sp.csr_matrix(H), Z, Z, p)


def brute_force(H, p, s):
    """All syndrome-consistent errors with their probabilities."""
    N = H.shape[1]
    errs = np.array(list(itertools.product([0, 1], repeat=N)), dtype=np.uint8)
    ok = ((errs.astype(int) @ H.T.astype(int)) % 2 == s).all(1)
    errs = errs[ok]
    logw = (errs * np.log(p) + (1 - errs) * np.log1p(-p)).sum(1)
    return errs, logw


@pytest.mark.parametrize("seed", range(12))
def test_product_sum_exact_on_trees(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    P = random_tree_problem(rng, n_checks=int(rng.integers(2, 6)))
    H = P.H.toarray()
    e = (rng.random(P.N) < P.priors).astype(np.uint8)
    s = (H.astype(int) @ e) % 2
    errs, logw = brute_force(H, P.priors, s)
    w = np.exp(logw - logw.max())
    p1 = (w[:, None] * errs).sum(0) / w.sum()
    exact = np.log((1 - p1) / p1)
    opts = oracle_mod.Options(variant=1, max_iter=2 * P.N + 2)
    _, _, post, _ = oracle_mod.bp(P, s, opts=opts, early_stop=False)
    np.testing.assert_allclose(post, exact, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("seed", range(8))
def test_product_sum_exact_on_trees_at_huge_llrs(oracle_mod, seed):
    """Priors of 1e-300 .. 1e-200 (LLRs 460 .. 690) so that messages on the tree
    exceed 700, where -log tanh(x/2) underflows FP64; the exact marginals
    come from log-sum-exp over all syndrome-consistent errors."""
    from scipy.special import logsumexp
    rng = np.random.default_rng(500 + seed)
    P = random_tree_problem(rng, n_checks=int(rng.integers(2, 6)))
    P = P.with_priors(10.0 ** rng.uniform(-300, -200, size=P.N))
    H = P.H.toarray()
    e = np.zeros(P.N, np.uint8)
    e[rng.choice(P.N, size=seed % 2, replace=False)] = 1
    s = (H.astype(int) @ e) % 2
    errs, logw = brute_force(H, P.priors, s)
    exact = np.array([logsumexp(logw[errs[:, j] == 0]) - logsumexp(logw[errs[:, j] == 1])
                      for j in range(P.N)])
    assert np.abs(exact).max() > 709
    opts = oracle_mod.Options(variant=1, max_iter=2 * P.N + 2)
    _, _, post, _ = oracle_mod.bp(P, s, opts=opts, early_stop=False)
    np.testing.assert_allclose(post, exact, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("seed", range(12))
def test_min_sum_exact_min_energy_on_trees(oracle_mod, seed):
    rng = np.random.default_rng(100 + seed)
    P = random_tree_problem(rng, n_checks=int(rng.integers(2, 6)))
    H = P.H.toarray()
    e = (rng.random(P.N) < P.priors).astype(np.uint8)
    s = (H.astype(int) @ e) % 2
    errs, _ = brute_force(H, P.priors, s)
    lam = np.log((1 - P.priors) / P.priors)
    energy = errs @ lam
    exact = np.array([energy[errs[:, j] == 1].min() - energy[errs[:, j] == 0].min()
                      for j in range(P.N)])
    opts = oracle_mod.Options(variant=0, alpha=1.0, max_iter=2 * P.N + 2)
    _, _, post, _ = oracle_mod.bp(P, s, opts=opts, early_stop=False)
    np.testing.assert_allclose(post, exact, rtol=1e-12, atol=1e-12)


def test_min_sum_scale_multiplies_check_messages(oracle_mod):
    """One check, two variables: the check message is alpha * (-1)^s * sgn * |lam|."""
    H = sp.csr_matrix(np.array([[1, 1]], np.uint8))
    Z = sp.csr_matrix((0, 2), dtype=np.uint8)
    p = np.array([0.1, 0.3])
    P = Problem("pair", H, Z, Z, p)
    lam = np.log((1 - p) / p)
    for alpha in (1.0, 0.625):
        for s in (0, 1):
            opts = oracle_mod.Options(alpha=alpha, max_iter=1)
            _, _, post, _ = oracle_mod.bp(P, np.array([s]), opts=opts, early_stop=False)
            sign = -1.0 if s else 1.0
            np.testing.assert_allclose(post, [lam[0] + alpha * sign * lam[1],
                                              lam[1] + alpha * sign * lam[0]], rtol=1e-14)


def _shots(problem, B, seed):
    _, s, o = sample_shots(problem, seed, 0, B)
    return s, o


@pytest.mark.parametrize("name,p", [("bb72", 0.05), ("bb144", 0.06)])
def test_decoder_invariants(oracle_mod, name, p):
    P = bi.bb_problem(name, p)
    s, _ = _shots(P, 3000, 11)
    opts = oracle_mod.Options(max_iter=30)
    out = oracle_mod.decode_batch(P, s, 0, opts, want_post=True, want_post1=True, want_cut=True)
    st = out["status"]
    assert set(np.unique(st)) <= {0, 1, 2} and (st == 2).any() and (st == 1).any()
    conv = st < 2
    # converged => the correction reproduces the syndrome (Sec. II.C)
    assert (syndromes(out["e_hat"][conv], P.H) == s[conv]).all()
    # failed => it does not
    assert (syndromes(out["e_hat"][~conv], P.H) != s[~conv]).any(1).all()
    # iteration 0 convergence exactly for the zero syndrome (all priors < 1/2)
    zero = ~s.any(1)
    assert ((out["iters1"] == 0) == zero).all()
    assert (out["e_hat"][zero] == 0).all()
    # logical flips are e_hat L^T
    assert (out["obs_pred"] == syndromes(out["e_hat"], P.L)).all()
    D = P.D.toarray().astype(bool)
    post1, cut = out["post1"], out["cut"]
    ran_dc = st > 0
    assert (out["iters1"][ran_dc] == opts.max_iter).all()
    assert not cut[~ran_dc].any()
    for b in np.nonzero(ran_dc)[0]:
        c = cut[b].astype(bool)
        # every row of D has a cut variable in its support, and |Cut| <= rows(D)
        assert (D[:, c].any(1)).all() and c.sum() <= D.shape[0]
        # every cut variable is a (windowed) maximum of the first-run LLR in some row
        for row in D:
            sup = np.nonzero(row)[0]
            lmax = post1[b, sup].max()
            thr = lmax - opts.tie_rel * max(1.0, abs(lmax))
            chosen = sup[c[sup]]
            assert any(post1[b, j] >= thr for j in chosen)
        # cut variables are reported as e = 0 and posterior +inf (PadWithZeros)
        assert (out["e_hat"][b, c] == 0).all() and np.isposinf(out["post"][b, c]).all()


def test_cut_independent_of_row_order(oracle_mod):
    P = bi.bb_problem("bb144", 0.06)
    s, _ = _shots(P, 2000, 12)
    opts = oracle_mod.Options(max_iter=30)
    out = oracle_mod.decode_batch(P, s, 0, opts, want_post1=True, want_cut=True)
    failed = np.nonzero(out["status"] > 0)[0][:50]
    assert failed.size > 5
    # exact-tie mode: the hash keys on the row index, so only a pure argmax
    # rule can be row-order independent; use rows whose maximum is unique
    rng = np.random.default_rng(0)
    perm = rng.permutation(P.D.shape[0])
    Pp = Problem("perm", P.H, P.D[perm], P.L, P.priors)
    for b in failed:
        post = out["post1"][b]
        a = oracle_mod.dc_select(P, post, int(b), opts)
        bperm = oracle_mod.dc_select(Pp, post, int(b), opts)
        D = P.D.toarray()
        unique_rows = [all((post[np.nonzero(r)[0]] >= post[np.nonzero(r)[0]].max()
                            - opts.tie_rel * max(1, abs(post[np.nonzero(r)[0]].max()))).sum() == 1
                           for r in D)]
        if all(unique_rows):
            assert (a == bperm).all()
        # the union never depends on order for rows with a unique winner
        for r in D:
            sup = np.nonzero(r)[0]
            top = sup[np.argmax(post[sup])]
            lmax = post[top]
            if (post[sup] >= lmax - opts.tie_rel * max(1, abs(lmax))).sum() == 1:
                assert a[top] == 1 and bperm[top] == 1


def test_tie_break_rule(oracle_mod):
    """Candidates within the window are chosen by rank h(seed, shot*rows+row) mod |cand|."""
    P = bi.bb_problem("bb72", 0.05)
    D = P.D.tocsr()
    D.sort_indices()
    post = np.zeros(P.N)
    opts = oracle_mod.Options(tie_rel=1e-5, tie_seed=1234)
    shot = 77
    cut = oracle_mod.dc_select(P, post, shot, opts)
    expect = np.zeros(P.N, np.uint8)
    for row in range(D.shape[0]):
        sup = D.indices[D.indptr[row]:D.indptr[row + 1]]
        h = oracle_mod.hash64(opts.tie_seed, shot * D.shape[0] + row)
        expect[sup[h % len(sup)]] = 1
    assert (cut == expect).all()
    # window edges: inside at -0.5 tau, outside at -2 tau
    # every other variable is more reliable, so only row 0 picks inside its support
    post = np.full(P.N, 20.0)
    sup0 = D.indices[D.indptr[0]:D.indptr[1]]
    post[sup0] = 10.0 - np.array([0, 0.5e-4, 2e-4, 2e-4, 3e-4, 1.0])[:len(sup0)]
    opts1 = oracle_mod.Options(tie_rel=1e-5, tie_seed=99)
    c1 = oracle_mod.dc_select(P, post, 3, opts1)
    h = oracle_mod.hash64(99, 3 * D.shape[0] + 0)
    assert c1[sup0].sum() == 1 and c1[sup0[h % 2]] == 1


@pytest.mark.parametrize("name,p,prior", [("bb72", 0.05, 0), ("bb144", 0.07, 0), ("bb72", 0.05, 1)])
def test_algorithm1_equals_algorithm2(oracle_mod, name, p, prior):
    """Deleting the cut columns (Algorithm 1) and zeroing their priors
    (Algorithm 2) give identical results (Sec. III.A)."""
    P = bi.bb_problem(name, p)
    s, _ = _shots(P, 1500, 13)
    o1 = oracle_mod.Options(max_iter=40, cut_form=0, dc_prior=prior)
    o2 = oracle_mod.Options(max_iter=40, cut_form=1, dc_prior=prior)
    a = oracle_mod.decode_batch(P, s, 0, o1, want_post=True)
    b = oracle_mod.decode_batch(P, s, 0, o2, want_post=True)
    assert (a["status"] > 0).sum() > 20
    for k in ("e_hat", "status", "iters1", "iters2", "obs_pred"):
        assert (a[k] == b[k]).all(), k
    np.testing.assert_array_equal(a["post"], b["post"])


def test_dc_disabled_is_plain_bp(oracle_mod):
    P = bi.bb_problem("bb72", 0.06)
    s, _ = _shots(P, 800, 14)
    out = oracle_mod.decode_batch(P, s, 0, oracle_mod.Options(max_iter=25, dc_enable=0))
    assert set(np.unique(out["status"])) <= {0, 2}
    for b in range(0, 800, 97):
        ok, e, _, it = oracle_mod.bp(P, s[b], opts=oracle_mod.Options(max_iter=25))
        assert ok == (out["status"][b] == 0) and (e == out["e_hat"][b]).all() and it == out["iters1"][b]


def test_single_qubit_errors_are_corrected(oracle_mod):
    """Weight-1 errors are the unique most likely explanation on BB72 (d = 6)."""
    P = bi.bb_problem("bb72", 0.01)
    E = np.eye(P.N, dtype=np.uint8)
    s = syndromes(E, P.H)
    out = oracle_mod.decode_batch(P, s, 0, oracle_mod.Options(max_iter=50))
    assert (out["status"] == 0).all()
    assert (out["e_hat"] == E).all()
