"""Host-side logic that needs no GPU: the autotuner's choice rule and the
tensor checks of the host-memory decode binding."""
import types

import pytest
import torch

from paper_2510_08695_gb300 import _bpdc
from paper_2510_08695_gb300.autotune import choose


def test_autotune_keeps_the_incumbent_within_the_margin():
    assert choose({0: 1.00, 7: 0.99}, incumbent=0) == 0          # 1 % faster: keep
    assert choose({0: 1.00, 7: 0.97}, incumbent=0) == 7          # 3 % faster: switch
    assert choose({0: 1.00, 7: 0.99}, incumbent=0, margin=0.0) == 7
    assert choose({1: 2.0, 8: 1.0}, incumbent=5) == 8            # incumbent not timed
    assert choose({3: 1.0}, incumbent=3) == 3


def _fake_graph():
    return types.SimpleNamespace(MW=2, NW=5, KW=1, handle=None)


def _item(**over):
    g = _fake_graph()
    it = dict(graph=g, syndromes=torch.zeros((4, 2), dtype=torch.int32), shot_offset=0,
              out=dict(corrections=torch.zeros((4, 5), dtype=torch.int32), status=torch.zeros(4, dtype=torch.uint8)))
    for k, v in over.items():
        if k in ("corrections", "status", "logical_flips", "iterations"):
            it["out"][k] = v
        else:
            it[k] = v
    return it


@pytest.mark.parametrize("bad", [
    dict(syndromes=torch.zeros((4, 3), dtype=torch.int32)),                  # wrong row width
    dict(syndromes=torch.zeros((4, 2), dtype=torch.int64)),                  # wrong dtype
    dict(syndromes=torch.zeros((2, 4), dtype=torch.int32).t()),              # not contiguous
    dict(corrections=torch.zeros((4, 4), dtype=torch.int32)),                # wrong output width
    dict(status=torch.zeros(3, dtype=torch.uint8)),                          # wrong batch size
    dict(obs_true=torch.zeros((4, 2), dtype=torch.int32)),                   # wrong logical width
    dict(logical_flips=torch.zeros((4, 1), dtype=torch.float32)),            # wrong dtype
])
def test_host_decode_rejects_malformed_tensors_before_the_library(bad):
    with pytest.raises(ValueError):
        _bpdc.decode_host([_item(**bad)])
