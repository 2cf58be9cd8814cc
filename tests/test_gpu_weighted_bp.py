"""Weighted BP on the GPU (forward kernel + hand-written adjoint behind a
torch.autograd.Function) against the plain-PyTorch FP64 reference
(oracle/weighted_bp.py, itself pinned to the FP64 oracle) and against finite
differences of the GPU forward."""
import numpy as np
import pytest
import torch

import bpdc_inputs as bi
from bpdc_inputs.sampler import sample_shots
from oracle import weighted_bp as ref
from parity import to_dev

pytestmark = pytest.mark.gpu

SEED = 0x2510086950


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_08695_gb300 as pkg
    from paper_2510_08695_gb300 import wbp
    P = bi.bb_problem("bb144", 0.06)
    g = pkg.Graph.from_problem(P, pkg.Options(variant=1, max_iter=20))
    e, s, _ = sample_shots(P, SEED + 40, 0, 64)
    T = 8
    rng = np.random.default_rng(9)
    W = rng.uniform(0.7, 1.3, size=(2, T, P.E))
    return pkg, wbp, P, g, e, s, T, W


def _gpu_post(wbp, g, s, W, clip=20.0, k=3):
    Wt = torch.tensor(W, dtype=torch.float32, device="cuda")
    return wbp.weighted_bp(Wt, g, to_dev(s), clip, k)


def test_forward_matches_reference(setup):
    pkg, wbp, P, g, e, s, T, W = setup
    post = _gpu_post(wbp, g, s, W).double().cpu().numpy()
    rp = ref.forward(P.H, P.priors, s, torch.tensor(W)).numpy()
    rel = np.abs(post - rp) / np.maximum(np.abs(rp), 1.0)
    assert rel.max() < 1e-4, rel.max()


def test_unit_weights_give_the_decoders_posterior(setup):
    """Unit weights and T iterations reproduce the product-sum posterior of the
    reference (pinned to the oracle) for every iteration."""
    pkg, wbp, P, g, e, s, T, W = setup
    post = _gpu_post(wbp, g, s, np.ones_like(W), clip=30.0).double().cpu().numpy()
    rp = ref.forward(P.H, P.priors, s, torch.ones(2, T, P.E, dtype=torch.float64), clip=30.0).numpy()
    assert (np.abs(post - rp) / np.maximum(np.abs(rp), 1.0)).max() < 1e-4


def test_adjoint_matches_reference_autograd(setup):
    pkg, wbp, P, g, e, s, T, W = setup
    Wg = torch.tensor(W, dtype=torch.float32, device="cuda", requires_grad=True)
    err = torch.tensor(e, dtype=torch.float32, device="cuda")
    wbp.bce_loss(wbp.weighted_bp(Wg, g, to_dev(s), 20.0, 3), err).backward()
    gg = Wg.grad.double().cpu().numpy()
    Wr = torch.tensor(W, requires_grad=True)
    ref.bce_loss(ref.forward(P.H, P.priors, s, Wr), e).backward()
    gr = Wr.grad.numpy()
    scale = np.abs(gr).max()
    assert scale > 0
    assert np.abs(gg - gr).max() <= 1e-3 * scale, (np.abs(gg - gr).max(), scale)


def test_adjoint_matches_finite_differences(setup):
    """Central differences (h = 1e-3) of the GPU forward's summed loss at the
    weights with the largest gradients; FP32 forward noise bounds the
    agreement at a few percent."""
    pkg, wbp, P, g, e, s, T, W = setup
    err = torch.tensor(e, dtype=torch.float64, device="cuda")

    def loss(Wn):
        post = _gpu_post(wbp, g, s, Wn).double()
        ee = err[:, None, :]
        return float((ee * torch.nn.functional.softplus(post) + (1 - ee) * torch.nn.functional.softplus(-post)).sum())

    Wg = torch.tensor(W, dtype=torch.float32, device="cuda", requires_grad=True)
    post = wbp.weighted_bp(Wg, g, to_dev(s), 20.0, 3)
    ee = err.float()[:, None, :]
    (ee * torch.nn.functional.softplus(post) + (1 - ee) * torch.nn.functional.softplus(-post)).sum().backward()
    gg = Wg.grad.double().cpu().numpy()
    h = 1e-3
    for k in np.argsort(-np.abs(gg).ravel())[:8]:
        idx = np.unravel_index(k, gg.shape)
        Wp, Wm = W.copy(), W.copy()
        Wp[idx] += h
        Wm[idx] -= h
        fd = (loss(Wp) - loss(Wm)) / (2 * h)
        assert abs(fd - gg[idx]) <= 5e-2 * abs(gg[idx]) + 1e-3, (idx, fd, gg[idx])


def test_coset_objective_gradient_matches_finite_differences(setup):
    """The coset-aware objective (probability that each iteration's residual
    flips a logical operator, plus missed syndrome bits) through the
    hand-written adjoint against central differences (h = 1e-3) of the GPU
    forward, at the weights with the largest gradients."""
    pkg, wbp, P, g, e, s, T, W = setup
    err = torch.tensor(e, dtype=torch.float64, device="cuda")
    syn = torch.tensor(s, dtype=torch.float64, device="cuda")
    H = torch.tensor(P.H.toarray(), dtype=torch.float64, device="cuda")
    O = torch.tensor(P.L.toarray(), dtype=torch.float64, device="cuda")

    scale = float(s.shape[0] * P.K)   # a sum over shots and observables, like the BCE check's

    def loss(Wn):
        return scale * float(wbp.coset_loss(_gpu_post(wbp, g, s, Wn).double(), err, syn, H, O))

    Wg = torch.tensor(W, dtype=torch.float32, device="cuda", requires_grad=True)
    post = wbp.weighted_bp(Wg, g, to_dev(s), 20.0, 3)
    (scale * wbp.coset_loss(post.double(), err, syn, H, O)).backward()
    gg = Wg.grad.double().cpu().numpy()
    assert np.abs(gg).max() > 0
    h = 1e-3
    for k in np.argsort(-np.abs(gg).ravel())[:8]:
        idx = np.unravel_index(k, gg.shape)
        Wp, Wm = W.copy(), W.copy()
        Wp[idx] += h
        Wm[idx] -= h
        fd = (loss(Wp) - loss(Wm)) / (2 * h)
        assert abs(fd - gg[idx]) <= 5e-2 * abs(gg[idx]) + 1e-3, (idx, fd, gg[idx])


def test_checkpoint_interval_does_not_change_results(setup):
    """Segments are recomputed with the forward's own arithmetic, so the
    posteriors and gradients are bit-identical for every interval k, and the
    fixed-order reduction makes repeated runs identical."""
    pkg, wbp, P, g, e, s, T, W = setup
    err = torch.tensor(e, dtype=torch.float32, device="cuda")
    res = []
    for k in (1, 3, T, 3):
        Wg = torch.tensor(W, dtype=torch.float32, device="cuda", requires_grad=True)
        post = wbp.weighted_bp(Wg, g, to_dev(s), 20.0, k)
        wbp.bce_loss(post, err).backward()
        res.append((post.detach().cpu(), Wg.grad.cpu()))
    for p, gr in res[1:]:
        assert torch.equal(p, res[0][0]) and torch.equal(gr, res[0][1])


def test_training_lowers_the_loss(setup):
    pkg, wbp, P, g, e, s, T, W = setup
    Wt, hist = wbp.train_weights(g, T=10, steps=12, batch=1024, lr=0.02, seed=SEED + 41)
    assert Wt.shape == (2, 10, P.E)
    assert np.mean(hist[-3:]) < hist[0], hist


def test_weighted_decode_matches_reference(setup):
    """BP (no DC) with learned weights inside the decoder: the iteration at
    which the hard decision first reproduces the syndrome and the posterior
    there equal the reference's, on shots whose reference posteriors stay
    away from 0 up to that iteration."""
    pkg, wbp, P, g, e, s, T, W = setup
    gd = pkg.Graph.from_problem(P, pkg.Options(variant=1, max_iter=T, dc_enable=0))
    gd.set_weights(torch.tensor(W, dtype=torch.float32), clip=20.0)
    out = gd.decode(to_dev(s), 0, posterior=True)
    it = out["iterations"].cpu().numpy() & 0xFFFF
    st = out["status"].cpu().numpy()
    post = out["posterior_llr"].cpu().numpy().astype(np.float64)
    rp = ref.forward(P.H, P.priors, s, torch.tensor(W)).numpy()       # [B, T, N]
    H = P.H.toarray().astype(np.int64)
    lam = np.log((1 - P.priors) / P.priors)
    checked = 0
    for b in range(s.shape[0]):
        hist = [lam] + [rp[b, t] for t in range(T)]                   # posterior after 0..T iterations
        conv = [t for t in range(T + 1) if (((H @ (hist[t] <= 0)) % 2) == s[b]).all()]
        t_ref = conv[0] if conv else None
        upto = (t_ref if t_ref is not None else T)
        if min(np.abs(h).min() for h in hist[1:upto + 1] or [lam]) < 1e-3:
            continue
        checked += 1
        if t_ref is None:
            assert st[b] == 2 and it[b] == T
            ref_post = hist[T]
        else:
            assert st[b] == 0 and it[b] == t_ref, (b, st[b], it[b], t_ref)
            ref_post = hist[t_ref]
        assert (np.abs(post[b] - ref_post) / np.maximum(np.abs(ref_post), 1.0)).max() < 1e-4
    assert checked > 40


def test_weights_need_the_product_sum_rule(setup):
    pkg, wbp, P, g, e, s, T, W = setup
    gm = pkg.Graph.from_problem(P, pkg.Options(variant=0))
    with pytest.raises(pkg.BpdcError):
        gm.set_weights(torch.ones(2, T, P.E), clip=20.0)


def test_learned_weights_are_kept_only_when_no_worse(setup):
    pkg, wbp, P, g, e, s, T, W = setup
    gd = pkg.Graph.from_problem(P, pkg.Options(variant=1, max_iter=50))
    Wt, _ = wbp.train_weights(gd, T=10, steps=8, batch=1024, lr=0.02, seed=SEED + 42)
    kept, ler_w, ler_p = wbp.select_weights(gd, Wt, shots=20000)
    assert kept == (ler_w <= ler_p)
    # the graph is left with the better setting
    ler_now = wbp.logical_error_rate(gd, 20000, 99, 1 << 40)
    assert ler_now == min(ler_w, ler_p) if kept else ler_now == ler_p
