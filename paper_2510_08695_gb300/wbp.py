"""Differentiable weighted BP on the GPU.

``weighted_bp(weights, graph, syndromes)`` is a ``torch.autograd.Function``
over the library's forward kernel (``bpdc_wbp_forward``) and hand-written
adjoint (``bpdc_decode_backward``): posterior LLRs [B, T, N] of T unrolled
product-sum iterations with per-edge, per-iteration weights [2, T, E]
(definition in include/bpdc.h).  Messages are checkpointed every
``ckpt_every`` iterations and recomputed per segment in the backward pass.

``train_weights`` fits the weights on shots the library samples itself, with
the binary cross-entropy of the posteriors against the sampled errors, or
with ``coset_loss``: the soft probability that the residual of each
iteration's decision flips a logical operator (the right target on a
degenerate code, where any correction in the error's coset succeeds) plus a
soft syndrome-mismatch term.
"""
from __future__ import annotations

import torch

from . import _bpdc


class WeightedBP(torch.autograd.Function):
    @staticmethod
    def forward(ctx, weights, graph, syndromes, clip: float = 20.0, ckpt_every: int = 5):
        T = int(weights.shape[1])
        w = weights.detach().contiguous()
        ws = _bpdc.wbp_workspace(graph, syndromes.shape[0], T, ckpt_every)
        post = _bpdc.wbp_forward(graph, syndromes, w, T, clip, ckpt_every, ws)
        ctx.save_for_backward(w)
        ctx.graph, ctx.syn, ctx.ws, ctx.clip, ctx.k = graph, syndromes, ws, clip, ckpt_every
        return post

    @staticmethod
    def backward(ctx, grad_post):
        (w,) = ctx.saved_tensors
        g = _bpdc.decode_backward(ctx.graph, ctx.syn, w, int(w.shape[1]), ctx.clip, ctx.k,
                                  grad_post.contiguous(), ctx.ws)
        return g, None, None, None, None


def weighted_bp(weights, graph, syndromes, clip: float = 20.0, ckpt_every: int = 5):
    return WeightedBP.apply(weights, graph, syndromes, clip, ckpt_every)


def bce_loss(post, errors):
    """Mean binary cross-entropy of sigma(-L) against the errors (float [B, N]),
    over shots, iterations and variables."""
    e = errors[:, None, :]
    return (e * torch.nn.functional.softplus(post) + (1 - e) * torch.nn.functional.softplus(-post)).mean()


def odd_parity_probability(x, A):
    """P(odd parity) of independent bits with probabilities x [B, N] over each
    row of the 0/1 matrix A [R, N]: (1 - prod_j (1 - 2 x_j)) / 2, the product
    taken in the log domain (magnitudes summed by a matmul, signs counted)."""
    t = 1 - 2 * x
    logabs = torch.log(t.abs().clamp_min(1e-30))
    negatives = torch.remainder((t < 0).to(x.dtype) @ A.T, 2)
    prod = torch.exp(logabs @ A.T) * (1 - 2 * negatives)
    return (1 - prod) / 2


def coset_loss(post, errors, syndromes, H, O, syndrome_weight: float = 1.0):
    """An objective tied to the decoder's success on a degenerate code, taken
    at every unrolled iteration (post [B, T, N]) like the BCE objective: with
    flip probabilities p_j = sigma(-L_j), the residual e + e_hat has bit j odd
    with probability q_j = e_j + p_j - 2 e_j p_j; the loss is the mean
    probability that the residual flips a logical operator (rows of O: a
    correction in the right coset scores 0 whatever its weight) plus
    syndrome_weight times the mean probability that the hard decision misses a
    syndrome bit (rows of H).  errors [B, N] and syndromes [B, M] are float
    {0, 1}; H, O dense float."""
    B, T, N = post.shape
    p = torch.sigmoid(-post).reshape(B * T, N)
    e = errors[:, None, :].expand(B, T, N).reshape(B * T, N)
    s = syndromes[:, None, :].expand(B, T, syndromes.shape[1]).reshape(B * T, -1)
    q = e + p - 2 * e * p
    logical = odd_parity_probability(q, O).mean()
    odd = odd_parity_probability(p, H)
    miss = (s * (1 - odd) + (1 - s) * odd).mean()
    return logical + syndrome_weight * miss


def unpack_words(words, n: int):
    """int32 bit words [B, ceil(n/32)] -> float32 {0, 1} [B, n] on the same device."""
    w = words.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    bits = (w[:, :, None] >> torch.arange(32, device=w.device)) & 1
    return bits.reshape(w.shape[0], -1)[:, :n].to(torch.float32)


def train_weights(graph, T: int = 20, steps: int = 50, batch: int = 4096, lr: float = 0.01, seed: int = 11,
                  clip: float = 20.0, ckpt_every: int = 5, weights=None, objective: str = "bce", problem=None):
    """Adam over freshly sampled batches (shot offsets advance every step) on
    the mean BCE of every iteration's posteriors against the sampled errors
    (objective "bce") or on coset_loss (objective "coset"; needs the problem
    for its H and L).  Returns (weights [2, T, E], list of losses)."""
    dev = torch.device("cuda", graph.device)
    W = (torch.ones((2, T, graph.E), dtype=torch.float32, device=dev) if weights is None
         else weights.detach().clone()).requires_grad_(True)
    opt = torch.optim.Adam([W], lr=lr)
    if objective == "coset":
        H = torch.tensor(problem.H.toarray(), dtype=torch.float32, device=dev)
        O = torch.tensor(problem.L.toarray(), dtype=torch.float32, device=dev)
    elif objective != "bce":
        raise ValueError(f"unknown objective {objective!r}")
    hist = []
    for s in range(steps):
        syn, _, err = graph.sample(batch, seed, s * batch, errors=True)
        post = weighted_bp(W, graph, syn, clip, ckpt_every)
        e = unpack_words(err, graph.N)
        if objective == "bce":
            loss = bce_loss(post, e)
        else:
            loss = coset_loss(post, e, unpack_words(syn, graph.M), H, O)
        opt.zero_grad()
        loss.backward()
        opt.step()
        hist.append(float(loss.detach()))
    return W.detach(), hist


def logical_error_rate(graph, shots: int, seed: int, shot_offset: int = 0, chunk: int = 100000) -> float:
    """BP+DC logical error rate of the graph's current setting (with or
    without learned weights) on seeded shots sampled by the library."""
    fails = 0
    done = 0
    dev = torch.device("cuda", graph.device)
    while done < shots:
        n = min(chunk, shots - done)
        syn, obs, _ = graph.sample(n, seed, shot_offset + done)
        cnt = torch.zeros(4, dtype=torch.int64, device=dev)
        graph.decode(syn, shot_offset + done, obs_true=obs, counters=cnt)
        fails += int(cnt[1])
        done += n
    return fails / shots


def binomial_interval(k: int, n: int, z: float = 1.96):
    """Wilson score interval of a binomial proportion k / n."""
    if n == 0:
        return 0.0, 1.0
    ph = k / n
    den = 1 + z * z / n
    c = (ph + z * z / (2 * n)) / den
    h = z * (ph * (1 - ph) / n + z * z / (4 * n * n)) ** 0.5 / den
    return c - h, c + h


def select_weights(graph, weights, clip: float = 20.0, shots: int = 100000, seed: int = 99,
                   shot_offset: int = 1 << 40):
    """Keeps learned weights only where they do no worse: BP+DC logical error
    rates with and without them on the same held-out shots (offsets far from
    the training shots); the graph is left with the better setting.  Returns
    (kept, ler_weighted, ler_plain)."""
    graph.set_weights(None)
    ler_plain = logical_error_rate(graph, shots, seed, shot_offset)
    graph.set_weights(weights, clip)
    ler_w = logical_error_rate(graph, shots, seed, shot_offset)
    kept = ler_w <= ler_plain
    if not kept:
        graph.set_weights(None)
    return kept, ler_w, ler_plain
