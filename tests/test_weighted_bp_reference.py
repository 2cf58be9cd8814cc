"""Pins of the plain-PyTorch weighted-BP reference (oracle/weighted_bp.py),
which the CUDA forward and adjoint are checked against: unit weights reproduce the FP64 oracle's
product-sum BP iteration by iteration, zero check weights leave the priors,
a two-edge check has a closed form, and autograd agrees with central finite
differences."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import bpdc_inputs as bi
from bpdc_inputs.sampler import sample_shots
from oracle import weighted_bp as wbp


def test_unit_weights_are_the_oracle_product_sum(oracle_mod):
    P = bi.bb_problem("bb72", 0.05)
    _, s, _ = sample_shots(P, 0x2510086950 + 30, 0, 6)
    T = 5
    W = torch.ones(2, T, P.E, dtype=torch.float64)
    post = wbp.forward(P.H, P.priors, s, W, clip=float("inf"), qmin=0.0).numpy()
    for b in range(s.shape[0]):
        for t in range(1, T + 1):
            _, _, ref, _ = oracle_mod.bp(P, s[b], opts=oracle_mod.Options(variant=1, max_iter=t),
                                         early_stop=False)
            np.testing.assert_allclose(post[b, t - 1], ref, rtol=1e-9, atol=1e-9)


def test_zero_check_weights_leave_the_priors():
    P = bi.bb_problem("bb72", 0.05)
    _, s, _ = sample_shots(P, 0x2510086950 + 31, 0, 4)
    W = torch.ones(2, 3, P.E, dtype=torch.float64)
    W[0] = 0.0
    post = wbp.forward(P.H, P.priors, s, W).numpy()
    lam = np.log((1 - P.priors) / P.priors)
    np.testing.assert_allclose(post, np.broadcast_to(lam, post.shape), rtol=0, atol=0)


def test_two_edge_check_closed_form():
    """One check on two variables: the product-sum of a single message is the
    message itself, so L_0(1) = lambda_0 + wc_0 (-1)^s clip(wv_1 lambda_1)."""
    H = sp.csr_matrix(np.array([[1, 1]], np.uint8))
    p = np.array([0.1, 0.2])
    lam = np.log((1 - p) / p)
    W = torch.tensor([[[0.7, 1.3]], [[0.9, 1.1]]], dtype=torch.float64)   # [2, T=1, E=2]
    for s in (0, 1):
        post = wbp.forward(H, p, np.array([[s]], np.uint8), W, clip=20.0).numpy()[0, 0]
        sig = -1.0 if s else 1.0
        np.testing.assert_allclose(post[0], lam[0] + 0.7 * sig * (1.1 * lam[1]), rtol=1e-12)
        np.testing.assert_allclose(post[1], lam[1] + 1.3 * sig * (0.9 * lam[0]), rtol=1e-12)


def test_autograd_matches_finite_differences():
    P = bi.bb_problem("bb72", 0.06)
    e, s, _ = sample_shots(P, 0x2510086950 + 32, 0, 8)
    T = 4
    rng = np.random.default_rng(3)
    W0 = torch.tensor(rng.uniform(0.6, 1.4, size=(2, T, P.E)))
    tb = wbp.edge_tables(P.H)

    def loss(W):
        return wbp.bce_loss(wbp.forward(P.H, P.priors, s, W, tables=tb), e)

    W = W0.clone().requires_grad_(True)
    loss(W).backward()
    g = W.grad.numpy()
    h = 1e-6
    for _ in range(12):
        k = (int(rng.integers(2)), int(rng.integers(T)), int(rng.integers(P.E)))
        Wp, Wm = W0.clone(), W0.clone()
        Wp[k] += h
        Wm[k] -= h
        fd = (loss(Wp).item() - loss(Wm).item()) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (k, fd, g[k])
