"""The allocation-free decode entry point against the ordinary one.

Some callers cannot allocate device memory while they decode: a real-time
decoding loop that must never wait on an allocator, a plugin inside a host
framework whose allocator owns the device memory, or a stream that is being
captured into a CUDA graph.  For them ``bpdc_decode_multi_noalloc`` takes the
persistent kernel's scratch (work counter, batch descriptors) from a fixed
device array of the library instead of allocated memory.  Its results must
equal ``bpdc_decode_multi``'s, bit for bit, on consecutive calls: the array is
shared by every call and keeps the previous call's contents.

This file is collected last on purpose; it passes alone in a fresh process
(the first call looks the array up) and after every other test.
"""
import numpy as np
import pytest

import bpdc_inputs as bi
from bpdc_inputs.sampler import sample_shots
from parity import to_dev

pytestmark = pytest.mark.gpu

KEYS = ("corrections", "status", "logical_flips", "iterations")


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_08695_gb300 as pkg
    pkg.load()
    return torch, pkg


def _items(torch, pkg, graphs, problems, seed):
    items = []
    for k, (g, P) in enumerate(zip(graphs, problems)):
        _, s, o = sample_shots(P, seed + k, 1000 * k, 1500)
        items.append(dict(graph=g, syndromes=to_dev(s), obs_true=to_dev(o), shot_offset=1000 * k,
                          out=g.alloc_outputs(s.shape[0]),
                          counters=torch.zeros(4, dtype=torch.int64, device="cuda")))
    return items


def _fresh_outputs(torch, items):
    return [dict(it, out=it["graph"].alloc_outputs(it["syndromes"].shape[0]),
                 counters=torch.zeros(4, dtype=torch.int64, device="cuda")) for it in items]


def test_noalloc_equals_decode_multi_on_consecutive_calls(env):
    torch, pkg = env
    problems = [bi.bb_problem("bb72", 0.05), bi.bb_problem("bb144", 0.06), bi.bb_problem("bb72", 0.08)]
    graphs = [pkg.Graph.from_problem(P, pkg.Options(max_iter=50)) for P in problems]
    for g in graphs:   # one call takes one kernel variant: variant 7's shape takes both codes
        g.set_kernel(7)
    assert len({g.info["kernel_id"] for g in graphs}) == 1
    for call, seed in enumerate((0x51, 0x52)):
        items = _items(torch, pkg, graphs, problems, seed)
        ref = _fresh_outputs(torch, items)
        pkg.decode_multi(ref)
        pkg.decode_multi_noalloc(items)
        torch.cuda.synchronize()
        for it, r in zip(items, ref):
            for k in KEYS:
                assert torch.equal(it["out"][k], r["out"][k]), (call, k)
            assert torch.equal(it["counters"], r["counters"]), call
            st = it["out"]["status"].cpu().numpy()
            assert (st == 1).any() or (st == 2).any()   # DC ran in this mix


def test_noalloc_rejects_what_its_scratch_cannot_hold(env):
    torch, pkg = env
    P = bi.bb_problem("bb72", 0.05)
    g = pkg.Graph.from_problem(P)
    _, s, _ = sample_shots(P, 3, 0, 8)
    syn = to_dev(s)
    too_many = [dict(graph=g, syndromes=syn, shot_offset=0, out=g.alloc_outputs(8)) for _ in range(17)]
    with pytest.raises(pkg.BpdcError) as err:
        pkg.decode_multi_noalloc(too_many)
    assert "at most 16 batches" in str(err.value)
    h = pkg.Graph.from_problem(bi.hgp_problem(0.05))
    _, sh, _ = sample_shots(bi.hgp_problem(0.05), 3, 0, 8)
    mixed = [dict(graph=g, syndromes=syn, shot_offset=0, out=g.alloc_outputs(8)),
             dict(graph=h, syndromes=to_dev(sh), shot_offset=0, out=h.alloc_outputs(8))]
    with pytest.raises(pkg.BpdcError):
        pkg.decode_multi_noalloc(mixed)
