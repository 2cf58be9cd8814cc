"""The allocation-free multi-batch decode captured into a CUDA graph: every
replay decodes the syndromes currently in the captured buffers, identically
to a direct call."""
import numpy as np
import pytest
import torch

import bpdc_inputs as bi

pytestmark = pytest.mark.gpu

SEED = 0x2510086950


def test_captured_decode_replays_new_syndromes():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_08695_gb300 as pkg
    gs = [pkg.Graph.from_problem(bi.bb_problem("bb72", 0.05)), pkg.Graph.from_problem(bi.bb_problem("bb144", 0.05))]
    for g in gs:   # one call takes one kernel variant: variant 7's shape takes both codes
        g.set_kernel(7)
    assert gs[0].info["kernel_id"] == gs[1].info["kernel_id"]
    B = [700, 300]
    syn = [torch.empty((b, g.MW), dtype=torch.int32, device="cuda") for b, g in zip(B, gs)]
    out = [g.alloc_outputs(b) for b, g in zip(B, gs)]
    items = [dict(graph=g, syndromes=s, shot_offset=5000 * k, out=o) for k, (g, s, o) in enumerate(zip(gs, syn, out))]
    for s, g, b in zip(syn, gs, B):
        s.copy_(g.sample(b, SEED, 0)[0])
    pkg.decode_multi_noalloc(items)          # first call outside the capture
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        pkg.decode_multi_noalloc(items)
    for rep in range(3):
        for s, g, b in zip(syn, gs, B):
            s.copy_(g.sample(b, SEED + 100 + rep, 0)[0])
        graph.replay()
        torch.cuda.synchronize()
        for k, (g, s, b) in enumerate(zip(gs, syn, B)):
            ref = g.decode(s, 5000 * k)
            for key in ("corrections", "status", "logical_flips", "iterations"):
                assert torch.equal(out[k][key], ref[key]), (rep, k, key)
