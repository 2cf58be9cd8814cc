"""Continuous-batching server: under a dense seeded Poisson trace of requests
from several codes, requests share launches and overlap on the device, and
every result equals decoding that request alone."""
import numpy as np
import pytest

import bpdc_inputs as bi
from bpdc_inputs.sampler import sample_shots
from parity import to_dev

pytestmark = pytest.mark.gpu


def test_server_results_equal_alone_and_requests_overlap():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_08695_gb300 as pkg
    from paper_2510_08695_gb300 import serving
    probs = [bi.bb_problem("bb72", 0.05), bi.bb_problem("bb144", 0.05), bi.hgp_problem(0.03)]
    graphs = [pkg.Graph.from_problem(P) for P in probs]
    pools = []
    for k, P in enumerate(probs):
        _, s, _ = sample_shots(P, 0x5E + k, 0, 6000 if P.N < 1000 else 1500)
        pools.append(to_dev(s).cpu().pin_memory())
    trace = serving.poisson_trace(300, rate_per_s=20000.0, n_graphs=3, seed=3, max_shots=512)
    server = serving.Server(graphs, slots=4, max_shots=2048)
    reqs = serving.replay(server, trace, pools)
    assert all(r.result is not None for r in reqs)
    assert max(server.requests_per_launch) > 1 and server.max_busy > 1
    for r in reqs:
        alone = graphs[r.graph_id].decode(r.syndromes.cuda(), r.shot_offset)
        for k in ("corrections", "status", "logical_flips", "iterations"):
            assert torch.equal(r.result[k], alone[k].cpu()), (r.rid, k)
    lat = np.array([r.done - r.arrival for r in reqs])
    assert (lat > 0).all()
