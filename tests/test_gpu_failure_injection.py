"""Allocation failures injected on the host (bpdc_debug_fail_allocations, no
GPU fault): graph creation fails with BPDC_ERR_OOM at each of its allocations
and leaves no graph; a failed re-plan keeps the graph decoding as before; a
failed host-decode staging allocation reports BPDC_ERR_OOM and the next call
works.  The injection is switched off again whatever happens."""
import pytest

import bpdc_inputs as bi
from bpdc_inputs.sampler import sample_shots
from parity import to_dev

pytestmark = pytest.mark.gpu

SEED = 0x2510086950
ERR_OOM = -3
KEYS = ("corrections", "status", "logical_flips", "iterations")


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_08695_gb300 as pkg
    pkg.load()
    yield pkg
    pkg.debug_fail_allocations(0, 0)


def _same(a, b):
    return all(bool((a[k].cpu() == b[k].cpu()).all()) for k in KEYS)


@pytest.mark.parametrize("skip", [0, 1, 2])   # the graph arena, the launch ring, its page-locked mirror
def test_graph_creation_reports_oom_at_every_allocation(pkg, skip):
    P = bi.bb_problem("bb72", 0.05)
    pkg.debug_fail_allocations(skip, 1)
    try:
        with pytest.raises(pkg.BpdcError) as ei:
            pkg.Graph.from_problem(P)
        assert ei.value.code == ERR_OOM
    finally:
        pkg.debug_fail_allocations(0, 0)
    _, s, o = sample_shots(P, SEED + 80, 0, 500)
    g = pkg.Graph.from_problem(P)
    out = g.decode(to_dev(s), 0, obs_true=to_dev(o))
    g.sync_status()
    assert out["status"].shape[0] == 500


def test_failed_replan_keeps_the_graph(pkg):
    P = bi.bb_problem("bb72", 0.06)
    _, s, o = sample_shots(P, SEED + 81, 0, 800)
    g = pkg.Graph.from_problem(P)
    ref = g.decode(to_dev(s), 0, obs_true=to_dev(o))
    k0 = g.info["kernel_id"]
    other = [k for k in g.kernels() if k != k0][0]
    g.set_kernel(k0)
    pkg.debug_fail_allocations(0, 1)
    try:
        with pytest.raises(pkg.BpdcError) as ei:
            g.set_kernel(other)
        assert ei.value.code == ERR_OOM
    finally:
        pkg.debug_fail_allocations(0, 0)
    assert g.info["kernel_id"] == k0
    assert _same(g.decode(to_dev(s), 0, obs_true=to_dev(o)), ref)


def test_host_decode_staging_failure(pkg):
    P = bi.bb_problem("bb144", 0.06)
    _, s, o = sample_shots(P, SEED + 82, 0, 1000)
    g = pkg.Graph.from_problem(P)
    ref = g.decode(to_dev(s), 0)
    items = [dict(graph=g, syndromes=to_dev(s).cpu().pin_memory(), shot_offset=0, out=g.alloc_host_outputs(1000))]
    pkg.debug_fail_allocations(0, 1)
    try:
        with pytest.raises(pkg.BpdcError) as ei:
            pkg.decode_host(items, chunk_shots=256)
        assert ei.value.code == ERR_OOM
    finally:
        pkg.debug_fail_allocations(0, 0)
    pkg.decode_host(items, chunk_shots=256)
    assert _same(items[0]["out"], ref)
