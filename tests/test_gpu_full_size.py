"""Parity at the full workload sizes, in the launch the benchmark times, on
sampled shots the oracle decodes one by one.

* Batched code capacity: BB[[144,12,12]], BB[[72,12,6]] and HGP-2500 at
  p = 0.01 .. 0.10, 10^6 shots per (code, p), all 30 batches in persistent
  multi-batch launches; inputs from the GPU sampler.
* Phenomenological BB[[144,12,12]], 12 noisy rounds + 1 perfect, p = q in
  {0.002 .. 0.010}, 10^6 shots per point, T_iter = 1000 (Sec. IV).

Sampled shot indices are spread over each 10^6-shot range; the counter
sampler regenerates any shot on the CPU from its global index."""
import numpy as np
import pytest
import torch

import bpdc_inputs as bi
from bpdc_inputs.sampler import sample_shots, unpack_bits
from parity import comparable, well_conditioned

pytestmark = pytest.mark.gpu

SEED = 0x2510086950
SHOTS = 1_000_000


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_08695_gb300 as pkg
    pkg.load()
    return pkg


def _sampled_parity(pkg, oracle_mod, items, probs, oo, picks_per_point, rng):
    """items: the decoded batches (outputs on the device); compares the picked
    shots of each batch with the oracle.  Returns (compared, picked)."""
    compared = total = 0
    for it, P in zip(items, probs):
        idx = np.sort(rng.choice(SHOTS, size=picks_per_point, replace=False))
        s = np.array([sample_shots(P, SEED, int(i), 1)[1][0] for i in idx])
        # the GPU sampler produced the same syndromes
        gs = unpack_bits(it["syndromes"][torch.as_tensor(idx, device="cuda")].cpu().numpy().view(np.uint32), P.M)
        assert (gs == s).all()
        refs = [oracle_mod.decode_batch(P, s[k:k + 1], int(i), oo, want_post=True, want_post1=True)
                for k, i in enumerate(idx)]
        ref = {key: np.concatenate([r[key] for r in refs]) for key in refs[0]}
        wc = np.array([well_conditioned(oracle_mod, P, s[k:k + 1], int(i), oo, refs[k], draws=1)[0]
                       for k, i in enumerate(idx)])
        comp = comparable(P, ref, oo.tie_rel) & wc
        sel = torch.as_tensor(idx, device="cuda")
        st = it["out"]["status"][sel].cpu().numpy()
        e = unpack_bits(it["out"]["corrections"][sel].cpu().numpy().view(np.uint32), P.N)
        iters = it["out"]["iterations"][sel].cpu().numpy().view(np.uint32)
        same = ((st == ref["status"]) & (e == ref["e_hat"]).all(1) & ((iters & 0xFFFF) == ref["iters1"])
                & ((iters >> 16) == ref["iters2"]))
        bad = np.nonzero(comp & ~same)[0]
        assert bad.size == 0, (P.name, idx[bad][:5])
        compared += int(comp.sum())
        total += len(idx)
    return compared, total


def test_batched_code_capacity_full_size(pkg, oracle_mod):
    probs = []
    for code in ("bb144", "bb72", "hgp2500"):
        for p in [round(0.01 * i, 2) for i in range(1, 11)]:
            probs.append(bi.hgp_problem(p) if code == "hgp2500" else bi.bb_problem(code, p))
    opts = pkg.Options(ms_scale=0.625, max_iter=50)
    items = []
    for P in probs:
        g = pkg.Graph.from_problem(P, opts)
        syn, obs, _ = g.sample(SHOTS, SEED, 0)
        items.append(dict(graph=g, syndromes=syn, shot_offset=0, out=g.alloc_outputs(SHOTS), obs_true=obs))
    by_kernel = {}
    for it in items:
        by_kernel.setdefault(it["graph"].info["kernel_id"], []).append(it)
    for group in by_kernel.values():
        pkg.decode_multi(group)
    torch.cuda.synchronize()
    rng = np.random.default_rng(17)
    oo = oracle_mod.Options(alpha=0.625, max_iter=50)
    picks = [60 if "hgp" in P.name else 150 for P in probs]
    compared = total = 0
    for it, P, k in zip(items, probs, picks):
        c, t = _sampled_parity(pkg, oracle_mod, [it], [P], oo, k, rng)
        compared += c
        total += t
    assert compared >= 0.5 * total, (compared, total)


def test_phenomenological_full_size(pkg, oracle_mod):
    probs = [bi.phenomenological_bb_problem("bb144", 12, p) for p in (0.002, 0.004, 0.006, 0.008, 0.010)]
    opts = pkg.Options(ms_scale=0.625, max_iter=1000)
    items = []
    for P in probs:
        g = pkg.Graph.from_problem(P, opts)
        syn, obs, _ = g.sample(SHOTS, SEED, 0)
        items.append(dict(graph=g, syndromes=syn, shot_offset=0, out=g.alloc_outputs(SHOTS), obs_true=obs))
    pkg.decode_multi(items)
    torch.cuda.synchronize()
    rng = np.random.default_rng(18)
    oo = oracle_mod.Options(alpha=0.625, max_iter=1000)
    compared, total = _sampled_parity(pkg, oracle_mod, items, probs, oo, 40, rng)
    assert compared >= 0.5 * total, (compared, total)
