"""Shot-by-shot comparison of the CUDA decoder (FP32) with the FP64 oracle.

Every shot lands in exactly one class, and the counts of all classes are
reported:

  exempt_llr       the oracle's final posterior, or for a shot that ran
                   degeneracy cutting its first-run posterior, has some
                   |L_j| < 1e-3: hard decisions are exempt from bit-exactness
                   there (the one exemption the acceptance grants for them).
  same             status, corrections, logical flips and both iteration
                   counts equal the oracle's.
  same_cut         the first runs agree, the GPU cut a different set, that
                   set is a cut the selection rule makes from the oracle's
                   first-run posterior with values within the rounding margin
                   of the tie-window edge counted either way (the acceptance
                   exempts those rows: their probability gap is below 1e-6),
                   and the oracle's second BP on the GPU's cut set
                   (Algorithm 2 form) gives the GPU's status, corrections and
                   second iteration count.
  same_perturbed   the outcome equals the oracle's outcome on priors scaled
                   by 1 + eps * z_j (z_j standard normal, eps = 1e-7, 1e-6,
                   1e-5; a fixed sequence of draws): the FP32 run is one such
                   rounding-sized perturbation of the computation.
  unmatched_ill    no oracle outcome matches, and the oracle's own outcome
                   changes under those perturbations (the shot is decided by
                   rounding); bounded by the caller.
  unmatched_well   no oracle outcome matches and the oracle's outcome is
                   stable under every perturbation: a real disagreement,
                   never accepted.

Posterior LLRs (when the GPU returned them) are compared on `same` and
`same_cut` shots entry by entry: relative error |gpu - ref| / |ref| <= 1e-4
(cut variables +inf on both sides).  Where an entry exceeds that, the oracle
is rerun on priors scaled by 1 + 1e-5 z_j (three draws): the entry passes if
the GPU's error is at most twice the largest change of the oracle's own value
(the exact algorithm amplifies rounding there beyond 1e-4).  The counts of
both kinds are reported; no entry may fail both.

Calibration (tests/test_parity_acceptance.py): the oracle's own output on
priors perturbed by 3e-7 or 1e-6 relative passes every rule, and planted
mistakes (a min-sum scale of 0.63 instead of 0.625, priors off by 0.2 %) fail
the outcome or the posterior rules on thousands of shots or entries.
"""
from __future__ import annotations

import itertools

import numpy as np

from bpdc_inputs.sampler import pack_bits, unpack_bits

LLR_EPS = 1e-3
WINDOW_EPS = 1e-6
POST_REL = 1e-4
PERT_EPS = (1e-7, 1e-6, 1e-5)
SENS_EPS, SENS_DRAWS, SENS_FACTOR = 1e-5, 3, 2.0
CLASSES = ("exempt_llr", "same", "same_cut", "same_perturbed", "unmatched_ill", "unmatched_well")


def to_dev(bits_u8: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(pack_bits(bits_u8)).view(np.int32)).cuda()


def from_dev(words, n: int) -> np.ndarray:
    return unpack_bits(words.cpu().numpy().view(np.uint32), n)


def gpu_outcome(problem, out: dict) -> dict:
    """Host copy of a decode's outputs: status, e_hat [B,N], obs_pred [B,K],
    iters1 / iters2 and, when present, post [B,N] (float64)."""
    st = out["status"].cpu().numpy()
    res = dict(status=st, e_hat=from_dev(out["corrections"], problem.N))
    K = problem.K
    res["obs_pred"] = from_dev(out["logical_flips"], K) if K and "logical_flips" in out \
        else np.zeros((len(st), K), np.uint8)
    it = out["iterations"].cpu().numpy().view(np.uint32)
    res["iters1"] = (it & 0xFFFF).astype(np.int32)
    res["iters2"] = (it >> 16).astype(np.int32)
    if out.get("posterior_llr") is not None:
        res["post"] = out["posterior_llr"].cpu().numpy().astype(np.float64)
    return res


def concat(parts: list[dict]) -> dict:
    return {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}


def _same(a: dict, i: int, b: dict, j: int, iters: bool = True) -> bool:
    ok = a["status"][i] == b["status"][j] and bool((a["e_hat"][i] == b["e_hat"][j]).all())
    if iters:
        ok = ok and a["iters1"][i] == b["iters1"][j] and a["iters2"][i] == b["iters2"][j]
    return bool(ok)


def _perturbed_problem(problem, d: int):
    rng = np.random.default_rng(1000 + d)
    eps = PERT_EPS[d % len(PERT_EPS)]
    return problem.with_priors(np.clip(problem.priors * (1 + eps * rng.standard_normal(problem.N)),
                                       1e-300, 0.5))


def possible_winners(D, post1: np.ndarray, tie_rel: float, margin: float, shot: int, tie_seed: int,
                     hash64, max_ambiguous: int = 10):
    """Per row of D, the set of variables the cut selection can pick when every
    value within `margin` * max(1, |L_max|) of the tie-window edge may fall on
    either side; None when a row has more than max_ambiguous such values."""
    D = D.tocsr()
    Md = D.shape[0]
    out = []
    for r in range(Md):
        sup = D.indices[D.indptr[r]:D.indptr[r + 1]]
        if sup.size == 0:
            out.append(set())
            continue
        sup = np.sort(sup)
        v = post1[sup]
        lmax = v.max()
        scale = max(1.0, abs(lmax)) if np.isfinite(lmax) else 1.0
        thr = lmax - tie_rel * scale if np.isfinite(lmax) else lmax
        m = margin * scale
        sure = v >= thr + m
        amb = np.nonzero((np.abs(v - thr) < m) & ~sure)[0]
        if amb.size > max_ambiguous:
            return None
        h = hash64(tie_seed, shot * Md + r)
        win = set()
        for k in range(amb.size + 1):
            for extra in itertools.combinations(amb.tolist(), k):
                mask = sure.copy()
                mask[list(extra)] = True
                cand = sup[mask]
                if cand.size:
                    win.add(int(cand[h % cand.size]))
        out.append(win)
    return out


def cut_is_possible(winners, cut: np.ndarray) -> bool:
    """Whether `cut` (uint8/bool [N]) is the union of one winner per row, each
    taken from its row's possible winners (a matching that covers every cut
    variable with a distinct row that can pick it; the other rows pick any of
    their possible winners inside the cut)."""
    in_cut = set(np.nonzero(cut)[0].tolist())
    opts = []
    for w in winners:
        if not w:
            continue
        c = w & in_cut
        if not c:
            return False
        opts.append(c)
    covered = set()
    free_rows = []
    for c in opts:
        if len(c) == 1:
            covered |= c
        else:
            free_rows.append(c)
    need = list(in_cut - covered)
    if not need:
        return True
    match = {}   # row index -> variable

    def augment(x, seen):
        for ri, c in enumerate(free_rows):
            if x in c and ri not in seen:
                seen.add(ri)
                if ri not in match or augment(match[ri], seen):
                    match[ri] = x
                    return True
        return False

    return all(augment(x, set()) for x in need)


def compare(oracle_mod, problem, syn: np.ndarray, shot_offset: int, oo, gpu: dict, ref: dict | None = None,
            draws: int = 12, offsets: np.ndarray | None = None, obs: np.ndarray | None = None) -> dict:
    """Classifies every shot (see the module docstring) and returns the report:
    counts per class, the posterior check, up to five examples of each
    unmatched class and, given the true observables `obs`, the failure counts
    of both sides.  `gpu` is gpu_outcome(); `offsets` gives each shot's global
    index when the shots are not consecutive."""
    B = syn.shape[0]
    gidx = np.arange(shot_offset, shot_offset + B, dtype=np.int64) if offsets is None else np.asarray(offsets)
    if ref is None:
        if offsets is None:
            ref = oracle_mod.decode_batch(problem, syn, shot_offset, oo, want_post=True, want_post1=True)
        else:
            ref = concat([oracle_mod.decode_batch(problem, syn[b:b + 1], int(gidx[b]), oo, want_post=True,
                                                  want_post1=True) for b in range(B)])
    post, post1 = ref["post"], ref["post1"]
    fin = np.where(np.isinf(post), np.inf, np.abs(post))
    exempt = fin.min(1) < LLR_EPS
    dc = ref["status"] > 0
    exempt[dc] |= np.abs(post1[dc]).min(1) < LLR_EPS
    cls = np.full(B, "", dtype=object)
    cls[exempt] = "exempt_llr"
    lam0 = oracle_mod.prior_llr(problem.priors)
    alt_post = {}   # shot -> oracle posterior of the matching alternative (same_cut)
    for b in range(B):
        if cls[b]:
            continue
        # with posteriors the GPU's cut set is visible: +inf marks a cut variable
        cut_diff = False
        if "post" in gpu and dc[b] and gpu["status"][b] > 0:
            cut_g = np.isinf(gpu["post"][b])
            cut_diff = bool((cut_g != np.isinf(post[b])).any())
        if not cut_diff and _same(gpu, b, ref, b):
            cls[b] = "same"
            continue
        # a different cut after identical first runs
        if cut_diff and gpu["iters1"][b] == ref["iters1"][b]:
            margin = WINDOW_EPS * max(1.0, ref["iters1"][b] / 50.0)
            win = possible_winners(problem.D, post1[b], oo.tie_rel, margin, int(gidx[b]), oo.tie_seed,
                                   oracle_mod.hash64)
            if win is not None and cut_is_possible(win, cut_g):
                if oo.dc_prior:
                    lam2 = oracle_mod.prior_llr(np.clip(1.0 / (1.0 + np.exp(post1[b])), 1e-12, 0.5))
                else:
                    lam2 = lam0.copy()
                lam2 = np.where(cut_g, np.inf, lam2)
                ok, e2, p2, it2 = oracle_mod.bp(problem, syn[b], lam=lam2, opts=oo)
                fin2 = np.abs(p2[np.isfinite(p2)])
                if fin2.size and fin2.min() < LLR_EPS:
                    cls[b] = "exempt_llr"
                    continue
                if (gpu["status"][b] == (1 if ok else 2) and (gpu["e_hat"][b] == e2).all()
                        and gpu["iters2"][b] == it2):
                    cls[b] = "same_cut"
                    alt_post[b] = (p2, lam2)
                    continue
        # rounding-sized perturbations of the priors
        stable = True
        matched = False
        for d in range(draws):
            r = oracle_mod.decode_batch(_perturbed_problem(problem, d), syn[b:b + 1], int(gidx[b]), oo)
            if _same(gpu, b, r, 0):
                matched = True
                break
            if not _same(ref, b, r, 0):
                stable = False
        cls[b] = "same_perturbed" if matched else ("unmatched_ill" if not stable else "unmatched_well")
    rep = {c: int((cls == c).sum()) for c in CLASSES}
    rep["B"] = B
    rep["compared"] = B - rep["exempt_llr"]
    rep["status_gpu"] = np.bincount(gpu["status"], minlength=3).tolist()
    rep["status_ref"] = np.bincount(ref["status"], minlength=3).tolist()
    for c in ("unmatched_ill", "unmatched_well"):
        rep[c + "_examples"] = [dict(shot=int(gidx[b]), gpu=(int(gpu["status"][b]), int(gpu["iters1"][b]),
                                                             int(gpu["iters2"][b])),
                                     ref=(int(ref["status"][b]), int(ref["iters1"][b]), int(ref["iters2"][b])),
                                     e_diff=int((gpu["e_hat"][b] != ref["e_hat"][b]).sum()))
                                for b in np.nonzero(cls == c)[0][:5]]
    rep["classes"] = cls
    if obs is not None:
        rep["fail_gpu"], rep["fail_ref"] = failure_counts(problem, gpu, ref, obs)
    if "post" in gpu:
        rep["posterior"] = posterior_check(oracle_mod, problem, syn, gidx, oo, gpu, ref, cls, alt_post)
    return rep


def posterior_check(oracle_mod, problem, syn, gidx, oo, gpu, ref, cls, alt_post) -> dict:
    """Entry-by-entry posterior comparison on the `same` and `same_cut` shots.

    An entry passes when |gpu - ref| <= 1e-4 |ref|.  Where a shot has entries
    beyond that, the oracle is rerun on priors scaled by 1 + 1e-5 z_j (three
    draws, z_j standard normal) and such an
    entry passes when |gpu - ref| <= SENS_FACTOR times the largest change of the
    oracle's own value: the exact algorithm amplifies rounding there beyond
    1e-4, and no FP32 evaluation can do better than its own sensitivity."""
    shots = [b for b in range(len(cls)) if cls[b] in ("same", "same_cut")]
    n_ent = n_inf_bad = n_ok = n_sens = n_fail = 0
    worst = 0.0
    by_status = {0: 0, 1: 0, 2: 0}
    fails = []
    for b in shots:
        rp = alt_post[b][0] if b in alt_post else ref["post"][b]
        gp = gpu["post"][b]
        inf = np.isinf(rp)
        n_inf_bad += int((np.isinf(gp) != inf).sum())
        fin = ~inf
        err = np.abs(gp[fin] - rp[fin])
        rel = err / np.abs(rp[fin])
        n_ent += int(fin.sum())
        by_status[int(gpu["status"][b])] += 1
        bad = rel > POST_REL
        n_ok += int((~bad).sum())
        if (~bad).any():
            worst = max(worst, float(rel[~bad].max()))
        if not bad.any():
            continue
        cols = np.nonzero(fin)[0][bad]
        spread = np.zeros(cols.size)
        for d in range(SENS_DRAWS):
            z = np.random.default_rng(2000 + d).standard_normal(problem.N)
            if b in alt_post:   # the second BP on the GPU's cut: perturb its priors
                _, _, pp, _ = oracle_mod.bp(problem, syn[b], lam=alt_post[b][1] * (1 + SENS_EPS * z), opts=oo)
            else:
                Q = problem.with_priors(np.clip(problem.priors * (1 + SENS_EPS * z), 1e-300, 0.5))
                pp = oracle_mod.decode_batch(Q, syn[b:b + 1], int(gidx[b]), oo, want_post=True)["post"][0]
            spread = np.maximum(spread, np.abs(pp[cols] - rp[cols]))
        ok = err[bad] <= SENS_FACTOR * spread
        n_sens += int(ok.sum())
        n_fail += int((~ok).sum())
        for k in np.nonzero(~ok)[0][:1]:
            fails.append(dict(shot=int(gidx[b]), col=int(cols[k]), gpu=float(gp[cols[k]]), ref=float(rp[cols[k]]),
                              oracle_spread=float(spread[k])))
    return dict(shots=len(shots), shots_by_status=by_status, entries=n_ent, within_1e4=n_ok,
                within_sensitivity=n_sens, failed=n_fail, inf_mismatch=n_inf_bad,
                max_rel_within_1e4=worst, fail_examples=fails[:5])


def summary(rep: dict) -> dict:
    """The report without the per-shot class array (for printing)."""
    return {k: v for k, v in rep.items() if k != "classes"}


def failure_counts(problem, gpu: dict, ref: dict, obs: np.ndarray) -> tuple[int, int]:
    fail_g = (gpu["status"] == 2) | (gpu["obs_pred"] != obs).any(1)
    fail_o = (ref["status"] == 2) | (ref["obs_pred"] != obs).any(1)
    return int(fail_g.sum()), int(fail_o.sum())


def within_2_sigma(k1: int, k2: int, n: int) -> bool:
    p = max((k1 + k2) / (2.0 * n), 1.0 / n)
    sigma = np.sqrt(n * p * (1 - p))
    return abs(k1 - k2) <= 2 * sigma + 1
