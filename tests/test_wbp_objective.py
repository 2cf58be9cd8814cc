"""The coset-aware weighted-BP objective (paper_2510_08695_gb300/wbp.py) on the
CPU: the soft parity against brute-force enumeration, and the loss at its
limits (a decoder that returns the error, one that returns an error of the
same coset, one that flips a logical operator)."""
import itertools

import numpy as np
import pytest
import torch

import bpdc_inputs as bi
from paper_2510_08695_gb300 import wbp


def test_odd_parity_probability_brute_force():
    rng = np.random.default_rng(3)
    N, R = 7, 4
    x = torch.tensor(rng.uniform(0, 1, size=(3, N)))
    A = torch.tensor((rng.uniform(size=(R, N)) < 0.5).astype(np.float64))
    got = wbp.odd_parity_probability(x, A).numpy()
    for b in range(3):
        for r in range(R):
            tot = 0.0
            for bits in itertools.product([0, 1], repeat=N):
                pr = np.prod([x[b, j].item() if bits[j] else 1 - x[b, j].item() for j in range(N)])
                if sum(bits[j] for j in range(N) if A[r, j] > 0) % 2:
                    tot += pr
            assert abs(got[b, r] - tot) < 1e-12


def test_coset_loss_limits():
    P = bi.bb_problem("bb72", 0.05)
    H = torch.tensor(P.H.toarray(), dtype=torch.float64)
    O = torch.tensor(P.L.toarray(), dtype=torch.float64)
    rng = np.random.default_rng(4)
    e = (rng.uniform(size=(1, P.N)) < 0.05).astype(np.float64)
    s = (e @ P.H.toarray().T) % 2
    big = 60.0

    def post_of(ehat):   # confident posteriors with decision ehat
        return torch.tensor(np.where(ehat > 0, -big, big)[:, None, :])

    E, S = torch.tensor(e), torch.tensor(s)
    # the error itself and the error times a stabilizer (a row of H_X): no loss
    assert wbp.coset_loss(post_of(e), E, S, H, O).item() < 1e-12
    stab = P.D.toarray()[0]
    assert wbp.coset_loss(post_of((e + stab) % 2), E, S, H, O).item() < 1e-12
    # the error times a logical operator of the other type flips a logical
    # observable: a logical X operator anticommutes with some row of O_Z
    Lx = None
    from bpdc_inputs import gf2
    K = gf2.nullspace(P.H.toarray() % 2)           # candidates commuting with H
    for v in K:
        if ((O.numpy() @ v) % 2).any():
            Lx = v
            break
    assert Lx is not None
    lost = wbp.coset_loss(post_of((e + Lx) % 2), E, S, H, O).item()
    assert lost > 1.0 / P.K - 1e-9
    # an undecided posterior (L = 0) scores half a flip per observable and row
    flat = torch.zeros((1, 1, P.N), dtype=torch.float64)
    assert abs(wbp.coset_loss(flat, E, S, H, O).item() - 1.0) < 1e-9


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_coset_loss_gradient_finite_differences(dtype):
    P = bi.bb_problem("bb72", 0.05)
    H = torch.tensor(P.H.toarray(), dtype=dtype)
    O = torch.tensor(P.L.toarray(), dtype=dtype)
    rng = np.random.default_rng(5)
    e = torch.tensor((rng.uniform(size=(2, P.N)) < 0.05).astype(np.float64), dtype=dtype)
    s = torch.remainder(e @ H.T, 2)
    post = torch.tensor(rng.normal(2.0, 2.0, size=(2, 3, P.N)), dtype=torch.float64, requires_grad=True)
    # every iteration enters the loss: perturb the middle and the last one
    loss = wbp.coset_loss(post, e.double(), s.double(), H.double(), O.double())
    loss.backward()
    g = post.grad.numpy()
    h = 1e-6
    for (b, t, j) in [(0, 2, 0), (1, 1, 5), (0, 2, 40), (1, 0, 7)]:
        p1 = post.detach().clone()
        p1[b, t, j] += h
        p2 = post.detach().clone()
        p2[b, t, j] -= h
        fd = (wbp.coset_loss(p1, e.double(), s.double(), H.double(), O.double())
              - wbp.coset_loss(p2, e.double(), s.double(), H.double(), O.double())).item() / (2 * h)
        assert abs(fd - g[b, t, j]) < 1e-6 * max(1.0, abs(fd))
