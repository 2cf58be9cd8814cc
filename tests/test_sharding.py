"""Multi-rank host logic of bench.py on the CPU: two gloo ranks shard the shots
of every (code, p) point by global index, their ranges are disjoint, the
elapsed time is the max over ranks, and decoding results do not depend on the
sharding (the tie-break hash keys on the global shot index)."""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, spp, result_dir):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import torch
    import bench
    import bpdc_inputs as bi
    import oracle
    from bpdc_inputs.sampler import sample_shots

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    off = bench.shard_offset(rank, spp)
    offs = [None] * world
    dist.all_gather_object(offs, off)
    # elapsed-time aggregation: max over ranks
    t = torch.tensor([float(rank + 1) * 1.5])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    # every rank decodes its own shard with the oracle
    P = bi.bb_problem("bb72", 0.07)
    _, s, _ = sample_shots(P, 99, off, spp)
    out = oracle.decode_batch(P, s, off, oracle.Options(max_iter=30), want_cut=True)
    np.savez(os.path.join(result_dir, f"rank{rank}.npz"), offs=np.array(offs), tmax=t.numpy(),
             e_hat=out["e_hat"], status=out["status"], cut=out["cut"])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_by_global_index(tmp_path, oracle_mod):
    import torch.multiprocessing as mp
    spp, world = 400, 2
    mp.start_processes(_rank_main, args=(world, _free_port(), spp, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    r = [np.load(tmp_path / f"rank{k}.npz") for k in range(world)]
    offs = r[0]["offs"]
    assert list(offs) == [0, spp]
    assert all(float(x["tmax"][0]) == 3.0 for x in r)   # max over ranks
    # one process decoding all global shots gives the same results
    import bpdc_inputs as bi
    from bpdc_inputs.sampler import sample_shots
    P = bi.bb_problem("bb72", 0.07)
    _, s, _ = sample_shots(P, 99, 0, world * spp)
    ref = oracle_mod.decode_batch(P, s, 0, oracle_mod.Options(max_iter=30), want_cut=True)
    for k in range(world):
        sl = slice(k * spp, (k + 1) * spp)
        assert (r[k]["status"] == ref["status"][sl]).all()
        assert (r[k]["e_hat"] == ref["e_hat"][sl]).all()
        assert (r[k]["cut"] == ref["cut"][sl]).all()
    assert (ref["status"] > 0).sum() > 10   # DC ran, so the hash keying was exercised
