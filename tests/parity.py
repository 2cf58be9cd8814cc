"""Helpers that compare the CUDA decoder with the FP64 oracle shot by shot.

Acceptance (FP32 GPU vs FP64 oracle):
  * a shot is *comparable* when the oracle's final posterior has |L_j| >= 1e-3
    for every variable and, if the shot ran degeneracy cutting, its first-run
    posterior also has |L_j| >= 1e-3 and every row of D is *robust*: no
    support variable lies within 1e-6 * max(1, |L_max|) of the tie-window
    edge L_max - tie_rel * max(1, |L_max|) (so FP32 rounding cannot change the
    candidate set; the margin grows as max(1, t / 50) with the t iterations
    of the first run, whose rounding drift accumulates);
  * and the shot is *well conditioned*: the oracle's outcome (status, e_hat,
    iteration counts) does not change when every prior is multiplied by
    1 + eps * z_j (z_j standard normal; three draws each at eps = 1e-7, 1e-6
    and 1e-5, the scale of FP32 rounding).  Min-sum
    with uniform priors is full of exact ties and exact zero messages; on the
    shots where such a tie decides the outcome, any rounding difference
    (FP32 against FP64) may decide it differently, so those shots are
    compared only through the failure statistics;
  * on comparable shots status, corrections, logical flips and iteration
    counts are bit-exact;
  * over all shots the failure counts agree within 2 binomial sigma.
"""
from __future__ import annotations

import numpy as np

from bpdc_inputs.sampler import pack_bits, unpack_bits

LLR_EPS = 1e-3
WINDOW_EPS = 1e-6


def to_dev(bits_u8: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(pack_bits(bits_u8)).view(np.int32)).cuda()


def from_dev(words, n: int) -> np.ndarray:
    return unpack_bits(words.cpu().numpy().view(np.uint32), n)


def robust_rows(D, post1: np.ndarray, tie_rel: float, margin=None) -> np.ndarray:
    """bool [B]: every row of D has its candidate set decided away from the
    window edge, by more than margin[b] * max(1, |L_max|) (default WINDOW_EPS)."""
    D = D.tocsr()
    ok = np.ones(post1.shape[0], dtype=bool)
    eps = np.full(post1.shape[0], WINDOW_EPS) if margin is None else np.asarray(margin, dtype=np.float64)
    for r in range(D.shape[0]):
        sup = D.indices[D.indptr[r]:D.indptr[r + 1]]
        if sup.size == 0:
            continue
        v = post1[:, sup]
        lmax = v.max(1)
        scale = np.maximum(1.0, np.abs(lmax))
        thr = lmax - tie_rel * scale
        near = (np.abs(v - thr[:, None]) <= (eps * scale)[:, None]) & (v != lmax[:, None])
        ok &= ~near.any(1)
    return ok


def well_conditioned(oracle_mod, problem, syn, shot_offset, opts, ref, draws: int = 3,
                     eps=(1e-7, 1e-6, 1e-5)) -> np.ndarray:
    """bool [B]: the oracle outcome survives tiny random relative prior
    perturbations (``draws`` draws at each relative size in ``eps``)."""
    ok = np.ones(syn.shape[0], dtype=bool)
    for d in range(draws * len(eps)):
        rng = np.random.default_rng(1000 + d)
        e = eps[d % len(eps)]
        q = problem.with_priors(np.clip(problem.priors * (1 + e * rng.standard_normal(problem.N)),
                                        1e-300, 0.5))
        pert = oracle_mod.decode_batch(q, syn, shot_offset, opts)
        ok &= ((pert["status"] == ref["status"]) & (pert["e_hat"] == ref["e_hat"]).all(1)
               & (pert["iters1"] == ref["iters1"]) & (pert["iters2"] == ref["iters2"]))
    return ok


def comparable(problem, ref: dict, tie_rel: float) -> np.ndarray:
    post = ref["post"]
    finite = np.where(np.isinf(post), np.inf, np.abs(post))
    ok = finite.min(1) >= LLR_EPS
    dc = ref["status"] > 0
    if dc.any():
        p1 = ref["post1"][dc]
        # FP32 rounding drift of the first-run posterior grows with the
        # iterations it ran: the margin scales with them beyond 50
        margin = WINDOW_EPS * np.maximum(1.0, ref["iters1"][dc] / 50.0)
        ok_dc = (np.abs(p1).min(1) >= LLR_EPS) & robust_rows(problem.D, p1, tie_rel, margin)
        ok[dc] &= ok_dc
    return ok


def compare(problem, gpu_out: dict, ref: dict, obs: np.ndarray | None, tie_rel: float) -> dict:
    """Returns counts and the indices of comparable shots that differ."""
    N, K = problem.N, problem.K
    st = gpu_out["status"].cpu().numpy()
    e = from_dev(gpu_out["corrections"], N)
    f = from_dev(gpu_out["logical_flips"], K) if K else np.zeros((len(st), 0), np.uint8)
    it = gpu_out["iterations"].cpu().numpy().view(np.uint32)
    it1, it2 = it & 0xFFFF, it >> 16
    comp = comparable(problem, ref, tie_rel)
    if "well_conditioned" in ref:
        comp &= ref["well_conditioned"]
    same = ((st == ref["status"]) & (e == ref["e_hat"]).all(1) & (f == ref["obs_pred"]).all(1)
            & (it1 == ref["iters1"]) & (it2 == ref["iters2"]))
    rep = dict(B=len(st), comparable=int(comp.sum()), mismatched=np.nonzero(comp & ~same)[0],
               identical_all=int(same.sum()), status_gpu=np.bincount(st, minlength=3),
               status_ref=np.bincount(ref["status"], minlength=3))
    # what differs on the first few mismatched shots (for the assertion message)
    rep["details"] = [dict(shot=int(b), status=(int(st[b]), int(ref["status"][b])),
                           iters=((int(it1[b]), int(it2[b])), (int(ref["iters1"][b]), int(ref["iters2"][b]))),
                           e_diff=np.nonzero(e[b] != ref["e_hat"][b])[0].tolist())
                      for b in rep["mismatched"][:5]]
    if obs is not None:
        fail_g = (st == 2) | (f != obs).any(1)
        fail_o = (ref["status"] == 2) | (ref["obs_pred"] != obs).any(1)
        rep["fail_gpu"], rep["fail_ref"] = int(fail_g.sum()), int(fail_o.sum())
    return rep


def within_2_sigma(k1: int, k2: int, n: int) -> bool:
    p = max((k1 + k2) / (2.0 * n), 1.0 / n)
    sigma = np.sqrt(n * p * (1 - p))
    return abs(k1 - k2) <= 2 * sigma + 1
