"""GPU parity: the CUDA decoder, called through the C-ABI, against the FP64
oracle on the same seeded shots (acceptance rules and their calibration in
tests/parity.py and tests/test_parity_acceptance.py).

Every case decodes twice, through the production launch (no posterior) and
with posterior output (the guarded path), asserts that both give identical
outcomes, and classifies every shot.  Each case asserts: no well-conditioned
mismatch; at most MAX_ILL of the shots decided differently where the oracle's
own outcome changes under rounding-sized prior perturbations; at least
`min_compared` of the shots outside the |L| < 1e-3 exemption (0.8 unless the
case states the measured reason); failure counts within two binomial sigma;
every posterior entry within 1e-4 relative or, where the oracle amplifies
rounding beyond that, within twice the oracle's own spread."""
import ctypes

import numpy as np
import pytest

import bpdc_inputs as bi
import parity
from bpdc_inputs.sampler import sample_shots, syndromes, unpack_bits
from parity import from_dev, to_dev, within_2_sigma

pytestmark = pytest.mark.gpu

SEED = 0x2510086950
MAX_ILL = 0.02
OUTCOME_KEYS = ("corrections", "status", "logical_flips", "iterations")


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def pkg(torch_cuda):
    import paper_2510_08695_gb300 as pkg
    pkg.load()
    return pkg


def oracle_options(oracle_mod, opts):
    return oracle_mod.Options(variant=opts.variant, alpha=opts.ms_scale, max_iter=opts.max_iter,
                              dc_enable=opts.dc_enable, dc_prior=opts.dc_prior, tie_rel=opts.tie_rel,
                              tie_seed=opts.tie_seed)


def _run(pkg, oracle_mod, P, B, opts_kw, seed=SEED, offset=0, G=None, persistent=True, kernel=None):
    """Decodes B seeded shots both ways and classifies them against the oracle."""
    _, s, o = sample_shots(P, seed, offset, B)
    opts = pkg.Options(**opts_kw)
    g = pkg.Graph.from_problem(P, opts)
    if G:
        g.set_plan(G)
    if kernel is not None:
        g.set_kernel(kernel)
    fast = g.decode(to_dev(s), offset, obs_true=to_dev(o), persistent=persistent)
    out = g.decode(to_dev(s), offset, obs_true=to_dev(o), persistent=persistent, posterior=True)
    g.sync_status()
    for k in OUTCOME_KEYS:
        assert bool((fast[k] == out[k]).all()), f"production and posterior paths differ in {k}"
    rep = parity.compare(oracle_mod, P, s, offset, oracle_options(oracle_mod, opts),
                         parity.gpu_outcome(P, out), obs=o)
    return g, rep


def _assert_parity(rep, min_compared=0.8, max_ill=MAX_ILL):
    sm = parity.summary(rep)
    print(sm)
    B = rep["B"]
    assert rep["unmatched_well"] == 0, sm
    assert rep["unmatched_ill"] <= max_ill * B, sm
    assert rep["compared"] >= min_compared * B, sm
    assert within_2_sigma(rep["fail_gpu"], rep["fail_ref"], B), sm
    post = rep.get("posterior")
    if post is not None:
        assert post["failed"] == 0 and post["inf_mismatch"] == 0, post
    return rep


# ---------------------------------------------------------------------------
# sampler

@pytest.mark.parametrize("name", ["bb72", "hgp", "phen"])
def test_gpu_sampler_bit_exact(pkg, name):
    P = {"bb72": lambda: bi.bb_problem("bb72", 0.05), "hgp": lambda: bi.hgp_problem(0.07),
         "phen": lambda: bi.phenomenological_bb_problem("bb72", 3, 0.02)}[name]()
    g = pkg.Graph.from_problem(P)
    B, off = 3000, 12345
    syn, obs, err = g.sample(B, SEED + 7, off, errors=True)
    e, s, o = sample_shots(P, SEED + 7, off, B)
    assert (from_dev(err, P.N) == e).all()
    assert (from_dev(syn, P.M) == s).all()
    assert (from_dev(obs, P.K) == o).all()


# ---------------------------------------------------------------------------
# full BP+DC against the oracle

def test_cfg_bb72_code_capacity_parity(pkg, oracle_mod):
    """BB [[72,12,6]], p = 0.05, 10^4 shots, alpha = 0.625, T_iter = 50, on the
    automatic variant (19: the shared last check pass)."""
    P = bi.bb_problem("bb72", 0.05)
    g, rep = _run(pkg, oracle_mod, P, 10000, dict(ms_scale=0.625, max_iter=50))
    assert g.info["kernel_id"] == 19
    _assert_parity(rep, min_compared=0.99)
    assert rep["status_ref"][1] > 50 and rep["status_ref"][2] > 50
    assert rep["posterior"]["shots_by_status"][1] > 100   # posteriors after the cut


def test_bb144_parity(pkg, oracle_mod):
    P = bi.bb_problem("bb144", 0.06)
    g, rep = _run(pkg, oracle_mod, P, 3000, dict(ms_scale=0.625, max_iter=50), G=32)
    assert g.info["threads_per_shot"] == 32 and g.info["kernel_id"] == 20   # the shared last check pass
    _assert_parity(rep, min_compared=0.99)


@pytest.mark.parametrize("p,min_compared", [(0.03, 0.99), (0.06, 0.95), (0.09, 0.7)])
def test_hgp_parity(pkg, oracle_mod, p, min_compared):
    """HGP-2500 (the dominant graph of the batched workload), 3000 shots per p,
    the automatic kernel (variant 15, the one the bench times).  At p = 0.09
    every shot fails and about 28 % of the failed runs end with some
    |L_j| < 1e-3 among the 2500 posteriors: those shots are exempt from
    bit-exactness, the rest must match."""
    P = bi.hgp_problem(p)
    g, rep = _run(pkg, oracle_mod, P, 3000, dict(ms_scale=0.625, max_iter=50))
    assert g.info["kernel_id"] == 15
    _assert_parity(rep, min_compared=min_compared)
    if p == 0.03:
        assert rep["same_cut"] > 100   # the cut-set path is exercised


@pytest.mark.parametrize("G", [128, 512])
def test_hgp_parity_other_group_sizes(pkg, oracle_mod, G):
    P = bi.hgp_problem(0.06)
    g, rep = _run(pkg, oracle_mod, P, 1000, dict(ms_scale=0.625, max_iter=50), G=G)
    assert g.info["threads_per_shot"] == G
    _assert_parity(rep, min_compared=0.95)


def test_phenomenological_parity_512(pkg, oracle_mod):
    P = bi.phenomenological_bb_problem("bb72", 6, 0.02)
    g, rep = _run(pkg, oracle_mod, P, 600, dict(ms_scale=0.625, max_iter=100), G=512)
    _assert_parity(rep, min_compared=0.99)


@pytest.mark.parametrize("p,T,B", [(0.006, 200, 400), (0.010, 1000, 600)])
def test_phenomenological_parity(pkg, oracle_mod, p, T, B):
    """Phenomenological BB[[144,12,12]], 12 noisy rounds + 1 perfect; the
    second case has the workload's p = q = 0.01 and T_iter = 1000."""
    P = bi.phenomenological_bb_problem("bb144", 12, p)
    g, rep = _run(pkg, oracle_mod, P, B, dict(ms_scale=0.625, max_iter=T))
    _assert_parity(rep, min_compared=0.99)


def test_posterior_prior_parity(pkg, oracle_mod):
    """Second BP on the first-run posterior (Algorithm 1 as printed).  Every
    variable with L <= 0 after the first run gets prior LLR 0, so the second
    run is full of exact ties; about 1.3 % of the shots are decided by
    rounding there (unmatched_ill, bounded at 2 %)."""
    P = bi.bb_problem("bb72", 0.06)
    g, rep = _run(pkg, oracle_mod, P, 4000, dict(ms_scale=0.625, max_iter=40, dc_prior=1))
    _assert_parity(rep, min_compared=0.99)


def test_alpha_one_parity(pkg, oracle_mod):
    """Plain min-sum (alpha = 1) on uniform priors keeps exact symmetric ties
    in exact-tie arithmetic: about 60 % of the shots end with some L_j = 0
    (exempt), and the FP64 oracle fails twice as often as under a 1e-9
    relative perturbation of the priors; FP32 rounding acts like such a
    perturbation.  Bit-exactness on the shots the oracle decides stably;
    unmatched rounding-decided shots bounded at 8 %; failure statistics against
    the perturbed oracle."""
    P = bi.bb_problem("bb72", 0.06)
    g, rep = _run(pkg, oracle_mod, P, 4000, dict(ms_scale=1.0, max_iter=72))
    sm = parity.summary(rep)
    print(sm)
    assert rep["unmatched_well"] == 0 and rep["unmatched_ill"] <= 0.08 * rep["B"], sm
    assert rep["compared"] >= 0.35 * rep["B"], sm
    assert rep["posterior"]["failed"] == 0, sm
    _, s, o = sample_shots(P, SEED, 0, 4000)
    rng = np.random.default_rng(5)
    Q = P.with_priors(P.priors * (1 + 1e-9 * rng.standard_normal(P.N)))
    pert = oracle_mod.decode_batch(Q, s, 0, oracle_mod.Options(alpha=1.0, max_iter=72))
    fail_p = int(((pert["status"] == 2) | (pert["obs_pred"] != o).any(1)).sum())
    assert within_2_sigma(rep["fail_gpu"], fail_p, rep["B"]), (rep["fail_gpu"], fail_p)


@pytest.mark.parametrize("d,p,prior", [(7, 0.01, 1), (7, 0.05, 1), (5, 0.06, 0)])
def test_surface_code_product_sum_parity(pkg, oracle_mod, d, p, prior):
    """The paper's surface-code setting: product-sum BP, T_iter = n, second BP
    on the first-run posterior (Sec. III.B).  Weight-2 boundary checks give
    exact posterior zeros (|L| < 1e-3, exempt) on 4 % (d = 7, p = 0.05) to
    17 % (d = 5, p = 0.06) of the shots."""
    P = bi.surface_problem(d, p)
    g, rep = _run(pkg, oracle_mod, P, 6000, dict(variant=1, max_iter=d * d, dc_prior=prior))
    assert g.info["kernel_id"] == 11
    _assert_parity(rep, min_compared=0.8)


def test_bb72_product_sum_parity(pkg, oracle_mod):
    P = bi.bb_problem("bb72", 0.05)
    g, rep = _run(pkg, oracle_mod, P, 4000, dict(variant=1, max_iter=50))
    assert g.info["kernel_id"] == 12
    _assert_parity(rep, min_compared=0.99)


def test_surface_code_min_sum_parity(pkg, oracle_mod):
    P = bi.surface_problem(7, 0.04)
    g, rep = _run(pkg, oracle_mod, P, 4000, dict(ms_scale=0.625, max_iter=49, dc_prior=1))
    _assert_parity(rep, min_compared=0.99)


# ---------------------------------------------------------------------------
# single steps

def test_cut_select_matches_oracle(pkg, oracle_mod, torch_cuda):
    """The selection step of Algorithm 1 alone, on the oracle's first-run
    posteriors rounded to FP32: every GPU cut set is one the rule makes when
    values within 1e-6 of a tie-window edge may fall either way, and nearly
    all equal the oracle's."""
    torch = torch_cuda
    P = bi.bb_problem("bb144", 0.07)
    _, s, _ = sample_shots(P, SEED + 3, 0, 3000)
    ref = oracle_mod.decode_batch(P, s, 0, oracle_mod.Options(max_iter=30), want_post1=True, want_cut=True)
    idx = np.nonzero(ref["status"] > 0)[0]
    assert idx.size > 50
    post = ref["post1"][idx].astype(np.float32)
    g = pkg.Graph.from_problem(P)
    # shot offsets must match the oracle's (global index = position in the batch)
    same = 0
    for k, b in enumerate(idx):
        cut = from_dev(g.cut_select(torch.from_numpy(post[k][None, :]).cuda(), int(b)), P.N)[0]
        win = parity.possible_winners(P.D, post[k].astype(np.float64), 1e-5, 1e-6, int(b), 0x2510086950,
                                      oracle_mod.hash64)
        assert win is not None and parity.cut_is_possible(win, cut), b
        same += int((cut == ref["cut"][b]).all())
    assert same >= 0.95 * idx.size, (same, idx.size)


def test_bp_on_given_cut_matches_oracle(pkg, oracle_mod):
    """BP #2 alone: the oracle's cut sets fed to the GPU (cut_in) and to the
    oracle's BP with +inf priors on the cut (Algorithm 2)."""
    P = bi.bb_problem("bb72", 0.06)
    _, s, _ = sample_shots(P, SEED + 4, 0, 4000)
    oo = oracle_mod.Options(max_iter=40)
    ref = oracle_mod.decode_batch(P, s, 0, oo, want_cut=True)
    idx = np.nonzero(ref["status"] > 0)[0][:300]
    g = pkg.Graph.from_problem(P, pkg.Options(max_iter=40))
    out = g.decode(to_dev(s[idx]), 0, cut_in=to_dev(ref["cut"][idx]))
    st = out["status"].cpu().numpy()
    e = from_dev(out["corrections"], P.N)
    it = out["iterations"].cpu().numpy() & 0xFFFF
    lam0 = oracle_mod.prior_llr(P.priors)
    n_cmp = 0
    for k, b in enumerate(idx):
        lam = np.where(ref["cut"][b] > 0, np.inf, lam0)
        ok, e_o, post, its = oracle_mod.bp(P, s[b], lam=lam, opts=oo)
        fin = np.abs(post[np.isfinite(post)])
        if fin.size and fin.min() < 1e-3:
            continue
        n_cmp += 1
        assert st[k] == (0 if ok else 2) and (e[k] == e_o).all() and it[k] == its, b
    assert n_cmp > 0.8 * len(idx)


# ---------------------------------------------------------------------------
# launch forms, splitting, edge cases

def test_plain_and_persistent_identical_and_offsets(pkg):
    P = bi.bb_problem("bb144", 0.06)
    _, s, o = sample_shots(P, SEED + 5, 1000, 2500)
    g = pkg.Graph.from_problem(P)
    a = g.decode(to_dev(s), 1000, persistent=True)
    b = g.decode(to_dev(s), 1000, persistent=False)
    c1 = g.decode(to_dev(s[:777]), 1000)
    c2 = g.decode(to_dev(s[777:]), 1777)
    for k in ("corrections", "status", "logical_flips", "iterations"):
        assert (a[k] == b[k]).all(), k
        import torch
        assert (a[k] == torch.cat([c1[k], c2[k]])).all(), k


@pytest.mark.parametrize("name,kernel", [("bb144", None), ("hgp", None), ("phen", None), ("hgp", 15),
                                         ("bb144", 20), ("circuit", 16)])
def test_layouts_give_identical_results(pkg, name, kernel):
    """The bank-conflict-aware layout changes no arithmetic: bit-identical
    outputs; also for the slot-profile variants, whose identity placement
    sorts variables by degree into the passes."""
    from bpdc_inputs import circuit
    P = {"bb144": lambda: bi.bb_problem("bb144", 0.07), "hgp": lambda: bi.hgp_problem(0.06),
         "phen": lambda: bi.phenomenological_bb_problem("bb144", 12, 0.008),
         "circuit": lambda: circuit.circuit_level_problem("bb72", 6, 2e-3)}[name]()
    _, s, o = sample_shots(P, SEED + 21, 0, 1500 if P.N < 1000 else 400)
    g = pkg.Graph.from_problem(P, pkg.Options(max_iter=200) if name == "circuit" else None)
    if kernel is not None:
        g.set_kernel(kernel)
    outs = []
    for mode in (1, 0):
        g.set_layout(mode)
        outs.append(g.decode(to_dev(s), 0, obs_true=to_dev(o), posterior=True))
    for k in ("corrections", "status", "logical_flips", "iterations", "posterior_llr"):
        a, b = outs[0][k], outs[1][k]
        assert (a == b).all() or (k == "posterior_llr" and bool(((a == b) | (a.isnan() & b.isnan())).all())), k


@pytest.mark.parametrize("name", ["bb72", "bb144", "hgp", "phen"])
def test_every_variant_gives_identical_results(pkg, name):
    """Every compiled kernel variant that accepts a graph (as the autotuner
    tries them, including the circuit-level one on small codes) decodes it
    bit-identically: min-sum takes order-free minima, and each variable sums
    its edges in ascending check order whatever the variant."""
    P = {"bb72": lambda: bi.bb_problem("bb72", 0.06), "bb144": lambda: bi.bb_problem("bb144", 0.07),
         "hgp": lambda: bi.hgp_problem(0.06),
         "phen": lambda: bi.phenomenological_bb_problem("bb144", 12, 0.01)}[name]()
    _, s, o = sample_shots(P, SEED + 22, 0, 1200 if P.N < 1000 else 300)
    g = pkg.Graph.from_problem(P)
    ks = g.kernels()
    assert len(ks) >= 2
    outs = {}
    for k in ks:
        g.set_kernel(k)
        outs[k] = g.decode(to_dev(s), 0, obs_true=to_dev(o))
    g.sync_status()
    k0 = ks[0]
    for k in ks[1:]:
        for key in ("corrections", "status", "logical_flips", "iterations"):
            assert torch_equal(outs[k][key], outs[k0][key]), (k, key)


def test_autotune_choice(pkg):
    """The autotuner times every accepting variant, keeps the automatic one
    within its margin and otherwise takes the fastest."""
    from paper_2510_08695_gb300.autotune import autotune
    P = bi.bb_problem("bb72", 0.06)
    _, s, _ = sample_shots(P, SEED + 23, 0, 2000)
    g = pkg.Graph.from_problem(P)
    k0 = g.info["kernel_id"]
    ks = g.kernels()
    res = autotune(g, to_dev(s), 0, margin=1.0)
    assert set(res["ms"]) == set(ks) and res["best"] == k0 and g.info["kernel_id"] == k0
    res = autotune(g, to_dev(s), 0, margin=0.0)
    assert res["best"] == min(res["ms"], key=res["ms"].get) and g.info["kernel_id"] == res["best"]


def torch_equal(a, b):
    return bool((a == b).all())


def test_decode_multi_equals_single(pkg):
    import torch
    probs = [bi.bb_problem("bb72", 0.04), bi.bb_problem("bb144", 0.05), bi.hgp_problem(0.05),
             bi.bb_problem("bb72", 0.08)]
    items, singles = [], []
    for i, P in enumerate(probs):
        _, s, o = sample_shots(P, SEED + 10 + i, 0, 700 if P.N > 200 else 2000)
        g = pkg.Graph.from_problem(P)
        syn, obs = to_dev(s), to_dev(o)
        singles.append(g.decode(syn, 0, obs_true=obs))
        items.append(dict(graph=g, syndromes=syn, shot_offset=0, obs_true=obs,
                          out=g.alloc_outputs(s.shape[0]),
                          counters=torch.zeros(4, dtype=torch.int64, device="cuda")))
    pkg.decode_multi(items)
    torch.cuda.synchronize()
    for it, ref in zip(items, singles):
        for k in ("corrections", "status", "logical_flips", "iterations"):
            assert (it["out"][k] == ref[k]).all(), k
        cnt = it["counters"].cpu().numpy()
        st = ref["status"].cpu().numpy()
        assert cnt[0] == len(st) and cnt[3] == (st > 0).sum()


def test_edge_cases(pkg, oracle_mod, torch_cuda):
    torch = torch_cuda
    P = bi.bb_problem("bb72", 0.05)
    g = pkg.Graph.from_problem(P)
    # B = 0 is a no-op
    out = g.decode(torch.zeros((0, g.MW), dtype=torch.int32, device="cuda"), 0)
    assert out["status"].numel() == 0
    # zero syndromes decode to zero at iteration 0
    z = g.decode(torch.zeros((64, g.MW), dtype=torch.int32, device="cuda"), 0)
    assert (z["corrections"] == 0).all() and (z["status"] == 0).all() and (z["iterations"] == 0).all()
    # a single shot, every single-qubit error of BB72
    E = np.eye(P.N, dtype=np.uint8)
    s = syndromes(E, P.H)
    one = g.decode(to_dev(s[:1]), 0)
    assert (from_dev(one["corrections"], P.N)[0] == E[0]).all()
    allq = g.decode(to_dev(s), 0)
    assert (from_dev(allq["corrections"], P.N) == E).all() and (allq["status"] == 0).all()
    # T_iter = 0: nonzero syndromes fail BP at once, DC runs on the priors
    _, s2, _ = sample_shots(P, SEED + 6, 0, 500)
    g0 = pkg.Graph.from_problem(P, pkg.Options(max_iter=0))
    r0 = g0.decode(to_dev(s2), 0)
    ref0 = oracle_mod.decode_batch(P, s2, 0, oracle_mod.Options(max_iter=0))
    assert (r0["status"].cpu().numpy() == ref0["status"]).all()
    # DC disabled: status is 0 or 2 only
    gd = pkg.Graph.from_problem(P, pkg.Options(dc_enable=0))
    rd = gd.decode(to_dev(s2), 0)
    assert set(np.unique(rd["status"].cpu().numpy())) <= {0, 2}
    # converged shots reproduce their syndrome
    rs = g.decode(to_dev(s2), 0)
    st = rs["status"].cpu().numpy()
    e = from_dev(rs["corrections"], P.N)
    assert (syndromes(e[st < 2], P.H) == s2[st < 2]).all()


def test_shot_limit_per_launch(pkg, torch_cuda):
    """One launch takes at most 2^32 - 2^24 shots (groups wider than a warp
    pass their work tickets through a 32-bit shared word): a larger call is
    refused with UNSUPPORTED before anything is launched or read (the buffers
    here hold one shot), and the library stays usable."""
    torch = torch_cuda
    from paper_2510_08695_gb300 import _bpdc
    P = bi.bb_problem("bb72", 0.05)
    g = pkg.Graph.from_problem(P)
    syn = torch.zeros((1, g.MW), dtype=torch.int32, device="cuda")
    out = g.alloc_outputs(1)
    o = g._outputs(out)
    big = (1 << 32) - (1 << 24) + 1
    rc = _bpdc._lib.bpdc_decode(g.handle, big, syn.data_ptr(), 0, ctypes.byref(o), 1, None)
    assert rc == _bpdc.ERR_UNSUPPORTED
    assert b"shots per launch" in _bpdc._lib.bpdc_last_error()
    ok = g.decode(syn, 0)
    torch.cuda.synchronize()
    assert int(ok["status"][0]) == 0


def test_smem_peak_microbenchmark(pkg):
    """The roof the bench divides by: conflict-free 4-byte shared-memory
    traffic moves at most 128 B per SM clock (32 banks x 4 B); GB300 SMs run
    at up to 2.07 GHz."""
    import torch
    m = pkg.measure_smem_peak(0, reps=4000)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert m["num_sms"] == sms
    assert 0.3 * 128 * sms * 2.07e9 < m["bytes_per_s"] <= 1.02 * 128 * sms * 2.07e9, m


# ---------------------------------------------------------------------------
# circuit-level detector error models (Appendix C / D; kernels 13 and 14)

@pytest.mark.parametrize("kernel", [16, 14, 13])
def test_circuit_level_parity_bb72(pkg, oracle_mod, kernel):
    """BB[[72,12,6]], 6 noisy rounds, p = 2e-3: H_DCM 252 x 2232 with rows of
    up to 35 edges, H_DDM for w = 3, T_iter = 1000 (Sec. IV), priors p for
    the second BP; every circuit-level kernel (16: 512 threads per shot with
    the row's q held in registers; 14: 1024 threads, degree-sorted passes and a
    shared edge table; 13: uniform passes)."""
    from bpdc_inputs import circuit
    P = circuit.circuit_level_problem("bb72", 6, 2e-3)
    g, rep = _run(pkg, oracle_mod, P, 400, dict(ms_scale=0.625, max_iter=1000), kernel=kernel)
    assert g.info["kernel_id"] == kernel
    _assert_parity(rep, min_compared=0.99)
    assert rep["status_ref"][1] > 20


def test_circuit_level_parity_bb144_full_size(pkg, oracle_mod):
    """The circuit-level serving model at full size: BB[[144,12,12]], 12
    rounds, p = 1e-3 (H_DCM 936 x 8784), on shots at global offsets spread
    over a 10^6-shot range, in the multi-batch launch the server uses."""
    import torch
    from bpdc_inputs import circuit
    P = circuit.circuit_level_problem("bb144", 12, 1e-3)
    opts = pkg.Options(ms_scale=0.625, max_iter=1000)
    g = pkg.Graph.from_problem(P, opts)
    assert g.info["kernel_id"] in (14, 16)
    offs, n = [0, 333_333, 999_900], 70
    s = np.concatenate([sample_shots(P, SEED + 20, off, n)[1] for off in offs])
    o = np.concatenate([sample_shots(P, SEED + 20, off, n)[2] for off in offs])
    outs = {}
    for post in (False, True):
        items = [dict(graph=g, syndromes=to_dev(s[i * n:(i + 1) * n]), shot_offset=off,
                      obs_true=to_dev(o[i * n:(i + 1) * n]), out=g.alloc_outputs(n, posterior=post))
                 for i, off in enumerate(offs)]
        pkg.decode_multi(items)      # one persistent launch over the three batches
        g.sync_status()
        outs[post] = {k: torch.cat([it["out"][k] for it in items]) for k in items[0]["out"]}
    for k in OUTCOME_KEYS:
        assert bool((outs[False][k] == outs[True][k]).all()), k
    gidx = np.concatenate([np.arange(off, off + n) for off in offs])
    rep = parity.compare(oracle_mod, P, s, 0, oracle_options(oracle_mod, opts), parity.gpu_outcome(P, outs[True]),
                         offsets=gidx, obs=o)
    _assert_parity(rep, min_compared=0.99)
    assert rep["status_ref"][1] > 10


def test_circuit_level_parity_bb72_w5(pkg, oracle_mod):
    """H_DDM from the local-window search for trivial errors of weight <= 5
    (App. D; the paper's circuit-level setting): 60 696 rows on BB72, 6 rounds."""
    from bpdc_inputs import circuit
    P = circuit.circuit_level_problem("bb72", 6, 3e-3, w=5)
    g, rep = _run(pkg, oracle_mod, P, 300, dict(ms_scale=0.625, max_iter=1000))
    assert g.info["kernel_id"] in (14, 16) and P.D.shape[0] > 50000
    _assert_parity(rep, min_compared=0.99)
    assert rep["status_ref"][1] > 20
