"""The bounds-checked build (libbpdc_checked.so, compiled with -DBPDC_CHECKS)
runs a spread of decodes without a failed check and with the outputs of the
normal library: every kernel variant that accepts BB[[72,12,6]] (the wide
circuit-level variant included), BB[[144,12,12]] and HGP-2500, product-sum with posteriors on
a surface code, a circuit-level detector model, learned weights, and the
host-memory path.  The checked decodes run in a child process, since a
process loads one of the two libraries."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# Runs the cases with whichever library the environment selects and saves
# every output array to the .npz file named by argv[1].
CASES = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[2]); sys.path.insert(0, sys.argv[2] + "/tests")
import paper_2510_08695_gb300 as pkg, bpdc_inputs as bi
from bpdc_inputs import circuit
from bpdc_inputs.sampler import sample_shots
from parity import to_dev
pkg.load(build_if_missing=False)
SEED = 0x2510086950
res = {}

def keep(tag, out):
    for k, v in out.items():
        res[f"{tag}/{k}"] = v.cpu().numpy()

def run(tag, P, B, opts=None, kernels=True, posterior=False, weights=None):
    _, s, o = sample_shots(P, SEED + 90, 0, B)
    g = pkg.Graph.from_problem(P, opts or pkg.Options())
    if weights is not None:
        g.set_weights(weights, clip=20.0)
    ks = g.kernels() if kernels else [g.info["kernel_id"]]
    for k in ks:
        g.set_kernel(k)
        keep(f"{tag}/k{k}", g.decode(to_dev(s), 0, obs_true=to_dev(o), posterior=posterior))
    return g, s

g, s = run("bb72", bi.bb_problem("bb72", 0.06), 600)
run("bb144", bi.bb_problem("bb144", 0.06), 300)
run("hgp", bi.hgp_problem(0.06), 200)
run("surface", bi.surface_problem(5, 0.05), 500, pkg.Options(variant=1, max_iter=25, dc_prior=1), posterior=True)
run("circuit", circuit.circuit_level_problem("bb72", 3, 0.003), 200, pkg.Options(max_iter=200), kernels=False)
P = bi.bb_problem("bb144", 0.06)
W = torch.tensor(np.random.default_rng(3).uniform(0.8, 1.2, size=(2, 5, P.E)), dtype=torch.float32)
run("weighted", P, 300, pkg.Options(variant=1, max_iter=10), kernels=False, weights=W)
host = [dict(graph=g, syndromes=to_dev(s).cpu(), shot_offset=0, out=g.alloc_host_outputs(s.shape[0]))]
pkg.decode_host(host, chunk_shots=128)
keep("host", host[0]["out"])
torch.cuda.synchronize()
if pkg.library_path().endswith("libbpdc_checked.so"):
    st = pkg.check_status(0)
    assert st is None, f"bounds check failed: site {st[0]}, index {st[1]}"
np.savez(sys.argv[1], **res)
"""


def _run(tmp_path, checked):
    if not __import__("torch").cuda.is_available():
        pytest.skip("no CUDA device")
    out = tmp_path / ("checked.npz" if checked else "normal.npz")
    env = dict(os.environ, BPDC_CHECKED="1" if checked else "0")
    r = subprocess.run([sys.executable, "-c", CASES, str(out), ROOT], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    return np.load(out)


def test_checked_build_runs_clean_and_matches(tmp_path):
    from paper_2510_08695_gb300 import build
    build.build()
    checked = _run(tmp_path, True)
    normal = _run(tmp_path, False)
    assert sorted(checked.files) == sorted(normal.files) and len(normal.files) > 30
    bad = [k for k in normal.files if not np.array_equal(checked[k], normal[k], equal_nan=True)]
    assert not bad, json.dumps(bad[:10])
