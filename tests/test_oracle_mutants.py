"""Planted mistakes: each mutant copies the oracle source, changes one line the
way a plausible bug would, compiles it, and must fail at least one pin.  The
unmodified source must pass every pin.  All of this runs on the CPU."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import bpdc_inputs as bi
import oracle
from bpdc_inputs.sampler import sample_shots, syndromes
from test_oracle_pins import brute_force, random_tree_problem

SRC = os.path.join(os.path.dirname(oracle.__file__), "bpdc_oracle.c")

MUTANTS = {
    "syndrome_sign_dropped": ("double syn_sign = s_i ? -1.0 : 1.0;", "double syn_sign = 1.0;"),
    "variable_message_not_extrinsic": ("if (b != a) ext += r[g->col_edges[b]];",
                                       "ext += r[g->col_edges[b]];"),
    "check_message_includes_own_edge": ("if (f == e) continue;\n            sign *= sgn(q[f]);\n            if (fabs",
                                        "sign *= sgn(q[f]);\n            if (fabs"),
    "prior_llr_inverted": ("return log((1.0 - p) / p);", "return log(p / (1.0 - p));"),
    "min_sum_scale_dropped": ("return alpha * sign * mag;", "return sign * mag;"),
    "hard_decision_flipped": ("e_hat[j] = post[j] <= 0.0;   /* Eq. 4 */",
                              "e_hat[j] = post[j] >= 0.0;"),
    "cut_most_likely_error": ("if (post[P->d_col[a]] >= thr) cand[nc++] = P->d_col[a];",
                              "if (post[P->d_col[a]] < thr) cand[nc++] = P->d_col[a];"),
    "boxplus_of_signed_message": ("mag = boxplus(mag, fabs(q[f]));", "mag = boxplus(mag, q[f]);"),
    "boxplus_sign_of_correction": ("log1p(exp(-(a + b))) - log1p(exp(-d))", "log1p(exp(-(a + b))) + log1p(exp(-d))"),
    "second_bp_keeps_cut_columns": ("for (int j = 0; j < N; ++j) keep[j] = cut[j] ? -1 : nk++;",
                                    "for (int j = 0; j < N; ++j) keep[j] = nk++;"),
}


def _check_trees(orc, variant):
    for seed in range(4):
        rng = np.random.default_rng(seed + 7 * variant)
        P = random_tree_problem(rng, n_checks=4)
        H = P.H.toarray()
        e = (rng.random(P.N) < P.priors).astype(np.uint8)
        s = (H.astype(int) @ e) % 2
        errs, logw = brute_force(H, P.priors, s)
        if variant == 1:
            w = np.exp(logw - logw.max())
            p1 = (w[:, None] * errs).sum(0) / w.sum()
            exact = np.log((1 - p1) / p1)
        else:
            lam = np.log((1 - P.priors) / P.priors)
            en = errs @ lam
            exact = np.array([en[errs[:, j] == 1].min() - en[errs[:, j] == 0].min()
                              for j in range(P.N)])
        opts = orc.Options(variant=variant, alpha=1.0, max_iter=2 * P.N + 2)
        _, _, post, _ = orc.bp(P, s, opts=opts, early_stop=False)
        if not np.allclose(post, exact, rtol=1e-9, atol=1e-9):
            return False
    return True


def _check_scale(orc):
    import scipy.sparse as sp
    from bpdc_inputs.codes import Problem
    H = sp.csr_matrix(np.array([[1, 1]], np.uint8))
    Z = sp.csr_matrix((0, 2), dtype=np.uint8)
    p = np.array([0.1, 0.3])
    lam = np.log((1 - p) / p)
    _, _, post, _ = orc.bp(Problem("pair", H, Z, Z, p), np.array([1]),
                           opts=orc.Options(alpha=0.625, max_iter=1), early_stop=False)
    return np.allclose(post, [lam[0] - 0.625 * lam[1], lam[1] - 0.625 * lam[0]], rtol=1e-14)


def _check_invariants(orc):
    P = bi.bb_problem("bb72", 0.05)
    _, s, obs = sample_shots(P, 21, 0, 1500)
    opts = orc.Options(max_iter=30)
    out = orc.decode_batch(P, s, 0, opts, want_post=True, want_post1=True, want_cut=True)
    st = out["status"]
    conv = st < 2
    if not (syndromes(out["e_hat"][conv], P.H) == s[conv]).all():
        return False
    zero = ~s.any(1)
    if not (((out["iters1"] == 0) == zero).all() and (out["e_hat"][zero] == 0).all()):
        return False
    # the decoder must actually decode: BB72 at p = 0.05 fails on ~19% of shots
    fail = (st == 2) | (out["obs_pred"] != obs).any(1)
    if fail.mean() > 0.3:
        return False
    if not ((st == 1).any() and (st == 0).mean() > 0.5):
        return False
    D = P.D.toarray().astype(bool)
    for b in np.nonzero(st > 0)[0][:40]:
        c = out["cut"][b].astype(bool)
        if not D[:, c].any(1).all():
            return False
        if not (out["e_hat"][b, c] == 0).all():
            return False
        for row in D:
            sup = np.nonzero(row)[0]
            lmax = out["post1"][b, sup].max()
            thr = lmax - opts.tie_rel * max(1.0, abs(lmax))
            if not (out["post1"][b, sup[c[sup]]] >= thr).any():
                return False
    a = orc.decode_batch(P, s, 0, orc.Options(max_iter=30, cut_form=1))
    return all((a[k] == out[k]).all() for k in ("e_hat", "status", "iters2"))


def _all_pins(orc):
    return dict(trees_sum_product=_check_trees(orc, 1), trees_min_sum=_check_trees(orc, 0),
                scale=_check_scale(orc), invariants=_check_invariants(orc))


def test_unmodified_oracle_passes_every_pin(tmp_path):
    out = oracle.compile_oracle(SRC, str(tmp_path / "liborig.so"))
    res = _all_pins(oracle.Oracle(out))
    assert all(res.values()), res


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation target for {name} not found exactly once"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    lib = oracle.compile_oracle(str(path), str(tmp_path / f"lib{name}.so"))
    # run in a child process: a mutant may also crash (e.g. divide by zero)
    here = os.path.dirname(os.path.abspath(__file__))
    code = ("import sys, json; sys.path[:0] = [%r, %r]; import oracle; "
            "from test_oracle_mutants import _all_pins; "
            "print(json.dumps(_all_pins(oracle.Oracle(%r))))" % (here, os.path.dirname(here), lib))
    proc = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    if proc.returncode != 0:
        return  # the mutant crashed the pins: caught
    res = json.loads(proc.stdout.strip().splitlines()[-1])
    assert not all(res.values()), f"mutant {name} survived every pin: {res}"
