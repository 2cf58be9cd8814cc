"""Plain PyTorch (float64, CPU) reference of weighted product-sum BP.

TEST INFRASTRUCTURE: only the test suite imports this module.  It shares no
code with the CUDA path.

Weighted BP is not part of the paper; it generalises the product-sum rule
that Sec. II.C.1 cites by one trainable weight per edge, per iteration and
per direction.  With every weight 1 and no clipping it is the flooding
product-sum BP of the oracle (a pin in the tests).  Definition, for
iterations t = 1..T over the edges e = (i, j) of H in CSR order:

    q_e(t) = clip( wv[t, e] * (lambda_j + sum_{e' in M(j), e' != e} r_e'(t-1)), -Q, Q ),  r(0) = 0
    r_e(t) = wc[t, e] * (-1)^{s_i} * prod_{e' in N(i), e' != e} sgn(q_e'(t))
                       * phi( sum_{e' in N(i), e' != e} phi( max(|q_e'(t)|, qmin) ) )
    L_j(t) = lambda_j + sum_{e in M(j)} r_e(t)

with phi(x) = -log tanh(x / 2) = log(1 + 2 / (e^x - 1)), sgn(0) = +1 and
lambda_j = ln((1 - p_j) / p_j).  Every step is written per edge with explicit
neighbour lists (no prefix sums, no subtraction of a total), so that it reads
against the definition; autograd provides the reference gradients.
"""
from __future__ import annotations

import numpy as np
import torch


def edge_tables(H):
    """Edge lists of a 0/1 matrix (scipy sparse or dense): rows, cols of the
    edges in CSR order; for every edge the other edges of its check and of its
    variable (padded with E, an extra slot); for every variable its edges
    (padded with E)."""
    import scipy.sparse as sp
    Hc = sp.csr_matrix(H)
    Hc.sort_indices()
    M, N = Hc.shape
    rows = np.repeat(np.arange(M), np.diff(Hc.indptr))
    cols = Hc.indices.astype(np.int64)
    E = len(cols)
    by_row = [list(range(Hc.indptr[i], Hc.indptr[i + 1])) for i in range(M)]
    by_col = [[] for _ in range(N)]
    for e in range(E):
        by_col[cols[e]].append(e)
    dmax = max(len(r) for r in by_row)
    cmax = max(len(c) for c in by_col)
    chk_others = np.full((E, max(dmax - 1, 1)), E, dtype=np.int64)
    var_others = np.full((E, max(cmax - 1, 1)), E, dtype=np.int64)
    for e in range(E):
        o = [x for x in by_row[rows[e]] if x != e]
        chk_others[e, :len(o)] = o
        o = [x for x in by_col[cols[e]] if x != e]
        var_others[e, :len(o)] = o
    var_edges = np.full((N, cmax), E, dtype=np.int64)
    for j in range(N):
        var_edges[j, :len(by_col[j])] = by_col[j]
    return dict(rows=rows, cols=cols, E=E, M=M, N=N, chk_others=chk_others, var_others=var_others,
                var_edges=var_edges)


def phi(x):
    return torch.log1p(2.0 / torch.expm1(x))


def forward(H, priors, syndromes, weights, clip: float = 20.0, qmin: float = 1e-6, tables=None):
    """Posterior LLRs [B, T, N] of weighted BP.

    syndromes: uint8 [B, M]; weights: float64 tensor [2, T, E] (wc = weights[0],
    wv = weights[1]); clip = Q (float('inf') for none)."""
    tb = tables or edge_tables(H)
    E, N = tb["E"], tb["N"]
    lam = torch.as_tensor(np.log((1.0 - priors) / priors), dtype=torch.float64)
    s = torch.as_tensor(np.asarray(syndromes, dtype=np.int64))
    B = s.shape[0]
    T = weights.shape[1]
    rows = torch.as_tensor(tb["rows"])
    cols = torch.as_tensor(tb["cols"])
    co = torch.as_tensor(tb["chk_others"])
    vo = torch.as_tensor(tb["var_others"])
    ve = torch.as_tensor(tb["var_edges"])
    syn_sign = 1.0 - 2.0 * s[:, rows].to(torch.float64)               # (-1)^{s_i} per edge
    lam_e = lam[cols]
    zero = torch.zeros(B, 1, dtype=torch.float64)
    r = torch.zeros(B, E, dtype=torch.float64)
    posts = []
    for t in range(T):
        # variable -> check: prior plus the other incoming check messages
        r_pad = torch.cat([r, zero], dim=1)
        a = lam_e + r_pad[:, vo].sum(dim=2)
        q = weights[1, t] * a
        if np.isfinite(clip):
            q = torch.clamp(q, -clip, clip)
        # check -> variable: product-sum over the other edges of the check
        f = phi(torch.clamp(q.abs(), min=qmin))
        sg = torch.where(q < 0, -1.0, 1.0).to(torch.float64)
        f_pad = torch.cat([f, zero], dim=1)                           # padding adds phi = 0
        sg_pad = torch.cat([sg, torch.ones(B, 1, dtype=torch.float64)], dim=1)
        S = f_pad[:, co].sum(dim=2)
        sign = syn_sign * sg_pad[:, co].prod(dim=2)
        r = weights[0, t] * sign * phi(S)
        # posterior
        r_pad = torch.cat([r, zero], dim=1)
        posts.append(lam[None, :] + r_pad[:, ve].sum(dim=2))
    return torch.stack(posts, dim=1)


def bce_loss(post, errors):
    """Mean binary cross-entropy of the posterior error probabilities
    sigma(-L) against the true errors, over shots, iterations and variables."""
    e = torch.as_tensor(np.asarray(errors), dtype=post.dtype)[:, None, :]
    # -[e log sigma(-L) + (1 - e) log sigma(L)] = e softplus(L) + (1 - e) softplus(-L)
    return (e * torch.nn.functional.softplus(post) + (1 - e) * torch.nn.functional.softplus(-post)).mean()
