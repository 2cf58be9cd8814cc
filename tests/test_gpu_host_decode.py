"""Decoding from host memory (bpdc_decode_host): the pipelined copy-in /
decode / copy-out path gives the outputs of the device path, for page-locked
and pageable host tensors, several graphs and kernel variants in one call,
pieces that split batches, and empty batches."""
import pytest

import bpdc_inputs as bi
from bpdc_inputs.sampler import sample_shots
from parity import to_dev

pytestmark = pytest.mark.gpu

SEED = 0x2510086950
KEYS = ("corrections", "status", "logical_flips", "iterations")


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_08695_gb300 as pkg
    pkg.load()
    return pkg


@pytest.fixture(scope="module")
def problems(pkg):
    probs = [bi.bb_problem("bb72", 0.06), bi.bb_problem("bb144", 0.07), bi.hgp_problem(0.05)]
    out = []
    for i, (P, B) in enumerate(zip(probs, (3001, 1500, 403))):
        _, s, o = sample_shots(P, SEED + 70 + i, 1000 * i, B)
        out.append((pkg.Graph.from_problem(P), to_dev(s), to_dev(o), 1000 * i))
    return out


def _device_reference(pkg, problems):
    import torch
    items = [dict(graph=g, syndromes=s, shot_offset=off, obs_true=o, out=g.alloc_outputs(s.shape[0]))
             for g, s, o, off in problems]
    pkg.decode_multi(items)
    torch.cuda.synchronize()
    return [it["out"] for it in items]


def _host_items(problems, pinned):
    import torch
    items = []
    for g, s, o, off in problems:
        B = s.shape[0]
        if pinned:
            sh, oh, out = s.cpu().pin_memory(), o.cpu().pin_memory(), g.alloc_host_outputs(B)
        else:
            sh, oh = s.cpu(), o.cpu()
            out = {k: torch.zeros(v.shape, dtype=v.dtype) for k, v in g.alloc_outputs(B).items()}
        items.append(dict(graph=g, syndromes=sh, shot_offset=off, obs_true=oh, out=out))
    return items


@pytest.mark.parametrize("pinned,chunk", [(True, 512), (True, 0), (False, 777)])
def test_host_decode_equals_device_decode(pkg, problems, pinned, chunk):
    ref = _device_reference(pkg, problems)
    items = _host_items(problems, pinned)
    pkg.decode_host(items, chunk_shots=chunk)
    for it, r in zip(items, ref):
        for k in KEYS:
            assert (it["out"][k] == r[k].cpu()).all(), k


def test_host_decode_empty_batches_and_required_outputs_only(pkg, problems):
    import torch
    ref = _device_reference(pkg, problems)
    g, s, o, off = problems[0]
    empty = dict(graph=g, syndromes=torch.empty((0, g.MW), dtype=torch.int32), shot_offset=0,
                 out=g.alloc_host_outputs(0))
    sh = s.cpu().pin_memory()
    out = g.alloc_host_outputs(s.shape[0], iterations=False, logical=False)
    pkg.decode_host([empty, dict(graph=g, syndromes=sh, shot_offset=off, out=out), empty], chunk_shots=1000)
    assert (out["corrections"] == ref[0]["corrections"].cpu()).all()
    assert (out["status"] == ref[0]["status"].cpu()).all()


def test_host_decode_rejects_device_tensors_and_posteriors(pkg, problems):
    import torch
    g, s, o, off = problems[0]
    with pytest.raises(ValueError):
        pkg.decode_host([dict(graph=g, syndromes=s, shot_offset=off, out=g.alloc_host_outputs(s.shape[0]))])
    out = g.alloc_host_outputs(s.shape[0])
    out["posterior_llr"] = torch.empty((s.shape[0], g.N), dtype=torch.float32)
    with pytest.raises(pkg.BpdcError):
        pkg.decode_host([dict(graph=g, syndromes=s.cpu(), shot_offset=off, out=out)])
