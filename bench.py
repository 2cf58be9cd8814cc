#!/usr/bin/env python3
"""Throughput benchmark of the BP+DC hot path (one JSON line on rank 0).

Workload (batched code capacity across uneven codes): BB [[144,12,12]],
BB [[72,12,6]] and the hypergraph product of a seeded (3,4)-regular n = 40
code (n = 2500, k = 148); bit-flip rate p = 0.01 .. 0.10 (10 values);
10^6 shots per (code, p); normalized min-sum, alpha = 0.625, T_iter = 50,
FP32 messages, degeneracy cutting on BP failure, second BP on the priors.
A step decodes all 3 * 10 * 10^6 shots; shots are sampled on the GPU by the
seeded counter sampler before timing (they stay resident in HBM; at ~2 GB
of syndromes they exceed L2, so no flush is needed).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --gpus N > 1 the script runs under torch.distributed.run, one process
per GPU; every rank decodes its own 3 * 10^7 shots (disjoint global shot
indices), so per-GPU work is fixed (weak scaling); the only cross-rank
operations are a barrier and a max of the elapsed times.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "BP+DC shots/s and p99 us/shot at matched LER vs plain kernel, 1 GB300"
UNIT = "shots/s"
SEED = 0x2510086950 + 1          # workload seed (second workload configuration)
P_VALUES = [round(0.01 * i, 2) for i in range(1, 11)]
CODES = ["bb144", "bb72", "hgp2500"]
ALPHA, T_ITER = 0.625, 50
SMEM_BYTES_PER_CLK_PER_SM = 128   # 32 banks x 4 B
SERVE_ROUNDS, SERVE_P, SERVE_T_ITER, SERVE_REQUESTS = 12, 1e-3, 1000, 300
SERVE_LOADS, SERVE_SLOTS = (0.5, 0.7, 0.9, 1.2, 2.0, 3.0), 8
WBP_T, WBP_BATCH, WBP_STEPS, WBP_LR, WBP_EVAL_SHOTS = 50, 4096, 60, 0.01, 2_000_000
WBP_EVAL_P = (0.04, 0.06, 0.08)
EDGE_UPDATE_BYTES = 16            # 2 x 4 B read + 2 x 4 B written per edge and iteration
# phenomenological workload: BB[[144,12,12]], 12 noisy rounds + 1 perfect, p = q
PHEN_ROUNDS, PHEN_P, PHEN_T_ITER = 12, [0.002, 0.004, 0.006, 0.008, 0.010], 1000
PHEN_SEED = 0x2510086950 + 2
# single-code workload: BB[[72,12,6]] at p = 0.05
BB72_P, BB72_SHOTS, BB72_SEED = 0.05, 10_000_000, 0x2510086950


# ---------------------------------------------------------------------------
# host helpers (no GPU needed)

def shard_offset(rank: int, shots_per_point: int) -> int:
    """First global shot index of a rank's share of every (code, p) point."""
    return rank * shots_per_point


# restricted profiling case outside the default workload: the circuit-level
# model of the serving leg on its own (kernel variant 13)
CIRCUIT_CASE = "circuit_bb144"
# and the phenomenological workload's points on their own (the kernel variant
# its leg autotunes to)
PHEN_CASE = "phen_bb144"


E2E_CHUNK = 262144   # shots per pipelined piece of the end-to-end leg


def case_t_iter(only) -> int:
    return {CIRCUIT_CASE: SERVE_T_ITER, PHEN_CASE: PHEN_T_ITER}.get(only, T_ITER)


def workload_problems(only=None, p_only=None):
    import bpdc_inputs as bi
    if only == CIRCUIT_CASE:
        from bpdc_inputs import circuit
        return [(CIRCUIT_CASE, SERVE_P, circuit.circuit_level_problem("bb144", SERVE_ROUNDS, SERVE_P))]
    if only == PHEN_CASE:
        return [(PHEN_CASE, p, bi.phenomenological_bb_problem("bb144", PHEN_ROUNDS, p)) for p in PHEN_P
                if p_only is None or abs(p - p_only) < 1e-9]
    probs = []
    for code in CODES:
        if only and code != only:
            continue
        for p in P_VALUES:
            if p_only is not None and abs(p - p_only) > 1e-9:
                continue
            if code == "hgp2500":
                probs.append((code, p, bi.hgp_problem(p)))
            else:
                probs.append((code, p, bi.bb_problem(code, p)))
    return probs


def extrapolate_cpu(samples, shots_per_point: int) -> float:
    """CPU shots/s for the full workload from per-point (shots, seconds) samples."""
    total_time = sum(shots_per_point * t / n for n, t in samples)
    return len(samples) * shots_per_point / total_time


def oracle_sample_plan(code: str) -> int:
    """Shots of each (code, p) point the CPU baseline decodes (about 10 s of
    work on 16 cores); the reference arm decodes a quarter of it per step."""
    return 1600 if code == "hgp2500" else 16000


def kernel_source_hash(kernel_id: int) -> str:
    """SHA-256 (16 hex digits) of what a kernel variant is built from: the device
    code of bpdc_kernels.cu (everything before the variant table) and the
    variant's own row of that table, without comments, blank lines and the
    checked build's guard blocks.  Other variants' rows do not enter it."""
    import hashlib
    import re
    src = os.path.join(ROOT, "paper_2510_08695_gb300", "csrc", "bpdc_kernels.cu")
    text = open(src).read()
    cut = text.index("#define BPDC_VARIANTS")
    code = re.sub(r"#ifdef BPDC_CHECKS\n.*?#endif\n", "", text[:cut], flags=re.S)
    code = re.sub(r"//[^\n]*", "", re.sub(r"/\*.*?\*/", "", code, flags=re.S))
    code = "\n".join(line.rstrip() for line in code.splitlines() if line.strip())
    row = re.search(r"X\(%d,[^)]*\)" % kernel_id, text[cut:])
    code += "\n" + (re.sub(r"\s+", "", row.group(0)) if row else "")
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def profiled_traffic(kernel_id: int, shots: int, edge_updates: int):
    """DRAM bytes per launch of a kernel variant, scaled from its committed ncu
    summary (profiles/decode_kernel_*.json) by the shots the launch processes
    (DRAM traffic is syndromes in, corrections out: it grows with shots, not
    iterations), and the shared-memory wavefront bytes scaled by edge-updates.
    (None, None, name) when no summary was taken from the current kernel
    source."""
    import glob
    cur = kernel_source_hash(kernel_id)
    stale = None
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "decode_kernel_*.json"))):
        prof = json.load(open(path))
        if prof.get("kernel_id") != kernel_id:
            continue
        if prof.get("kernel_device_source_sha256_16") != cur:
            stale = os.path.basename(path)
            continue
        smem = prof.get("smem_wavefront_bytes_per_edge_update")
        return (prof["traffic_bytes_per_shot"] * shots, None if smem is None else smem * edge_updates,
                os.path.basename(path))
    return None, None, stale


def smem_roofline(edge_updates: int, ms: float, peak_gbs: float, kernel_id: int, shots: int) -> dict:
    """Roofline of one decode launch against the shared-memory roof: 16
    algorithmic bytes per edge-update over the launch's CUDA-event time."""
    achieved = edge_updates * EDGE_UPDATE_BYTES / (ms / 1e3) / 1e9
    traffic, smem_traffic, prof_file = profiled_traffic(kernel_id, shots, edge_updates)
    return {"bound": "smem", "achieved": achieved, "peak": peak_gbs, "unit": "GB/s", "frac": achieved / peak_gbs,
            "traffic": traffic, "smem_wavefront_bytes": smem_traffic,
            "traffic_source": (f"DRAM bytes from profiles/{prof_file}, scaled by shots per launch"
                               if traffic is not None else "no ncu summary of the current kernel"),
            "kernel": f"decode_kernel variant {kernel_id}",
            "algorithmic_bytes": f"{EDGE_UPDATE_BYTES} B per edge-update x {edge_updates} edge-updates per launch"}


def timed(torch, stream, fn, reps: int) -> float:
    """Mean milliseconds of fn() over reps calls, CUDA events on `stream`."""
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def same_outputs(a: dict, b: dict) -> bool:
    return all(bool((a[k] == b[k]).all()) for k in ("corrections", "status", "logical_flips", "iterations") if k in a)


def phenomenological_leg(args, pkg, torch, stream, peak_gbs) -> dict:
    """Phenomenological BB[[144,12,12]] (12 noisy rounds + 1 perfect, Eq. 12-15;
    H_DDM of Sec. IV.B), p = q in {0.002 .. 0.010}, shots_per_point shots per
    point, T_iter = 1000: one persistent multi-batch launch over the five
    points against the plain per-batch kernel and against CUDA-graph replay of
    the allocation-free launch, identical outputs required."""
    import bpdc_inputs as bi
    from paper_2510_08695_gb300.autotune import autotune
    spp = args.shots_per_point
    opts = pkg.Options(ms_scale=ALPHA, max_iter=PHEN_T_ITER)
    items = []
    for p in PHEN_P:
        P = bi.phenomenological_bb_problem("bb144", PHEN_ROUNDS, p)
        g = pkg.Graph.from_problem(P, opts)
        syn, obs, _ = g.sample(spp, PHEN_SEED, 0)
        items.append(dict(graph=g, syndromes=syn, obs_true=obs, shot_offset=0, out=g.alloc_outputs(spp),
                          counters=torch.zeros(4, dtype=torch.int64, device="cuda"), p=p))
    torch.cuda.synchronize()
    # the probe: 10^5 shots of the p = 0.010 point, enough that the few shots
    # running all 1000 + 1000 iterations do not decide the launch's length alone
    probe = items[-1]
    tune = autotune(probe["graph"], probe["syndromes"][:min(100000, spp)].contiguous(), 0)
    for it in items:
        it["graph"].set_kernel(tune["best"])
    vid = tune["best"]
    reps = max(1, min(args.steps, 3))
    pkg.decode_multi(items, stream)           # warm-up
    for it in items:
        it["counters"].zero_()
    pkg.decode_multi(items, stream)           # counted pass
    torch.cuda.synchronize()
    cnt = [it["counters"].cpu().tolist() for it in items]
    ref = [{k: v.clone() for k, v in it["out"].items()} for it in items]
    counted = [dict(it, counters=None) for it in items]
    ms_persist = timed(torch, stream, lambda: pkg.decode_multi(counted, stream), reps)
    same_p = all(same_outputs(it["out"], r) for it, r in zip(items, ref))

    def plain():
        for it in items:
            it["graph"].decode(it["syndromes"], 0, obs_true=it["obs_true"], out=it["out"], persistent=False,
                               stream=stream)
    ms_plain = timed(torch, stream, plain, reps)
    same_plain = all(same_outputs(it["out"], r) for it, r in zip(items, ref))
    # CUDA graph of the allocation-free launch (descriptors captured as kernel
    # parameters; the first call resolves the scratch address outside capture)
    pkg.decode_multi_noalloc(counted, stream)
    torch.cuda.synchronize()
    cs = torch.cuda.Stream()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=cs):
        pkg.decode_multi_noalloc(counted, cs)
    ms_graph = timed(torch, stream, cg.replay, reps)
    same_graph = all(same_outputs(it["out"], r) for it, r in zip(items, ref))
    shots = spp * len(items)
    eu = sum(c[2] for c in cnt) * items[0]["graph"].E
    return {"workload": (f"phenomenological BB[[144,12,12]], {PHEN_ROUNDS} noisy rounds + 1 perfect, p=q in "
                         f"{PHEN_P}, detector check matrix {probe['graph'].M}x{probe['graph'].N}, H_DDM "
                         f"{items[0]['graph'].info['Md']} rows; {spp} shots per point; normalized min-sum alpha=0.625, "
                         f"T_iter={PHEN_T_ITER}, DC on failure, second BP on priors"),
            "metric": "shots/s", "value": shots / (ms_persist / 1e3), "ms_per_step": ms_persist,
            "edge_updates_per_s": eu / (ms_persist / 1e3),
            "plain_kernel": {"value": shots / (ms_plain / 1e3), "ms_per_step": ms_plain, "identical_outputs": same_plain},
            "cuda_graph_replay": {"value": shots / (ms_graph / 1e3), "ms_per_step": ms_graph,
                                  "identical_outputs": same_graph, "api": "bpdc_decode_multi_noalloc captured"},
            "persistent_identical_over_repeats": same_p,
            "ler": {f"p={it['p']}": c[1] / spp for it, c in zip(items, cnt)},
            "dc_fraction": {f"p={it['p']}": c[3] / spp for it, c in zip(items, cnt)},
            "autotune": {"kernel": vid, "ms_per_variant": {str(k): round(v, 3) for k, v in tune["ms"].items()}},
            "roofline": smem_roofline(eu, ms_persist, peak_gbs, vid, shots),
            "timing": f"CUDA events on the launching stream, mean of {reps} steps after a warm-up step"}


def bb72_leg(args, pkg, torch, stream, peak_gbs) -> dict:
    """BB[[72,12,6]] code capacity at p = 0.05, 10^7 shots per step (the
    single-code workload: alpha = 0.625, T_iter = 50, DC on failure)."""
    import bpdc_inputs as bi
    from paper_2510_08695_gb300.autotune import autotune
    P = bi.bb_problem("bb72", BB72_P)
    g = pkg.Graph.from_problem(P, pkg.Options(ms_scale=ALPHA, max_iter=T_ITER))
    syn, obs, _ = g.sample(BB72_SHOTS, BB72_SEED, 0)
    tune = autotune(g, syn[:20000].contiguous(), 0)
    g.set_kernel(tune["best"])
    out = g.alloc_outputs(BB72_SHOTS)
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    g.decode(syn, 0, obs_true=obs, out=out, stream=stream)
    g.decode(syn, 0, obs_true=obs, out=out, counters=cnt, stream=stream)
    torch.cuda.synchronize()
    c = cnt.cpu().tolist()
    reps = max(1, min(args.steps, 5))
    ms = timed(torch, stream, lambda: g.decode(syn, 0, obs_true=obs, out=out, stream=stream), reps)
    eu = c[2] * g.E
    return {"workload": f"BB[[72,12,6]] code capacity, p={BB72_P}, {BB72_SHOTS} shots per step, normalized min-sum "
                        "alpha=0.625, T_iter=50, DC on failure, second BP on priors",
            "metric": "shots/s", "value": BB72_SHOTS / (ms / 1e3), "ms_per_step": ms,
            "edge_updates_per_s": eu / (ms / 1e3), "ler": c[1] / BB72_SHOTS, "dc_fraction": c[3] / BB72_SHOTS,
            "autotune": {"kernel": tune["best"], "ms_per_variant": {str(k): round(v, 3) for k, v in tune["ms"].items()}},
            "roofline": smem_roofline(eu, ms, peak_gbs, tune["best"], BB72_SHOTS),
            "timing": f"CUDA events on the launching stream, mean of {reps} steps after a warm-up step"}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        under_load = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(under_load) if under_load else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def run_reference(args, world, rank):
    """The FP64 CPU oracle timed on bounded samples of the same workload."""
    if rank != 0:
        return
    import numpy as np
    import oracle
    from bpdc_inputs.sampler import sample_shots
    oracle.build()
    cores = oracle.max_threads()
    probs = workload_problems()
    opts = oracle.Options(alpha=ALPHA, max_iter=T_ITER)
    inputs = []
    for i, (code, p, P) in enumerate(probs):
        n = max(1, oracle_sample_plan(code) // 4)
        _, s, _ = sample_shots(P, SEED, 0, n)
        inputs.append((P, s))
    per_step = []
    for step in range(args.warmup + args.steps):
        samples = []
        for P, s in inputs:
            t0 = time.perf_counter()
            oracle.decode_batch(P, s, 0, opts)
            samples.append((s.shape[0], time.perf_counter() - t0))
        if step >= args.warmup:
            per_step.append(extrapolate_cpu(samples, args.shots_per_point))
    value = statistics.median(per_step)
    sample_desc = (f"{sum(s.shape[0] for _, s in inputs)} shots per step: first "
                   f"{oracle_sample_plan('bb72') // 4} (BB) / {oracle_sample_plan('hgp2500') // 4} (HGP) shots of "
                   "each (code, p) point, extrapolated per point to 1e6 shots")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded counter sampler)",
            "config": config_dict(args, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample_desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(args, world):
    n_points = len(workload_problems(getattr(args, "only", None), getattr(args, "p", None)))
    restricted = "" if n_points == len(CODES) * len(P_VALUES) else \
        f" [restricted to code={getattr(args, 'only', None)} p={getattr(args, 'p', None)}]"
    if getattr(args, "only", None) == PHEN_CASE:
        text = (f"phenomenological BB[[144,12,12]], {PHEN_ROUNDS} noisy rounds + 1 perfect, p=q in {PHEN_P}"
                f"{restricted}; {args.shots_per_point} shots per point per GPU; normalized min-sum alpha=0.625, "
                f"T_iter={PHEN_T_ITER}, DC on failure [profiling case]")
    elif getattr(args, "only", None) == CIRCUIT_CASE:
        text = (f"circuit-level BB[[144,12,12]], {SERVE_ROUNDS} rounds, p={SERVE_P:g} (detector model derived from "
                f"the depth-8 syndrome circuit, H_DDM w=3); {args.shots_per_point} shots per GPU; normalized "
                f"min-sum alpha=0.625, T_iter={SERVE_T_ITER}, DC on failure [restricted profiling case]")
    else:
        text = ("batched code capacity across uneven codes: BB[[144,12,12]], BB[[72,12,6]], "
                "HGP of a seeded (3,4)-regular n=40 code (n=2500, k=148); p=0.01..0.10 (10 values); "
                f"{args.shots_per_point} shots per (code,p) per GPU; normalized min-sum alpha=0.625, "
                "T_iter=50, DC on failure, second BP on priors p" + restricted)
    return {"workload": text,
            "shots_per_step": n_points * args.shots_per_point * world,
            "launch": "persistent multi-batch launches (one per kernel variant), device work counter, kernel variant "
                      "per code autotuned before the timed region",
            "l2": getattr(args, "l2_note", "inputs larger than L2 (no flush)"),
            "parallelism": f"dp{world}"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--shots-per-point", type=int, default=1_000_000)
    ap.add_argument("--no-extras", action="store_true", help="skip plain/e2e/latency/cpu legs")
    ap.add_argument("--only", choices=CODES + [CIRCUIT_CASE, PHEN_CASE], default=None,
                    help="restrict the workload to one code (small profiling cases; not a bench line)")
    ap.add_argument("--p", type=float, default=None, help="restrict the workload to one error rate")
    ap.add_argument("--kernel", type=int, default=None,
                    help="pin this kernel variant for every code instead of autotuning (profiling cases)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2510_08695_gb300 as pkg
    from paper_2510_08695_gb300 import build as pbuild
    if rank == 0:
        pbuild.build()
    if world > 1:
        dist.barrier()
    pkg.load(build_if_missing=False)

    spp = args.shots_per_point
    off = shard_offset(rank, spp)
    probs = workload_problems(args.only, args.p)
    opts = pkg.Options(ms_scale=ALPHA, max_iter=case_t_iter(args.only))
    batches = []
    for code, p, P in probs:
        g = pkg.Graph.from_problem(P, opts, device=local)
        syn, obs, _ = g.sample(spp, SEED, off)
        cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
        batches.append(dict(code=code, p=p, P=P, graph=g, syndromes=syn, obs_true=obs, shot_offset=off,
                            out=g.alloc_outputs(spp), counters=cnt))
    torch.cuda.synchronize()
    # autotuned mapping (untimed): per code, every kernel variant that accepts
    # its graph is timed on 20000 shots of the code's highest-p point, and all
    # points of the code take the fastest
    from paper_2510_08695_gb300.autotune import autotune
    tuned = {}
    for code in sorted({b["code"] for b in batches} if args.kernel is None else ()):
        probe = max((b for b in batches if b["code"] == code), key=lambda b: b["p"])
        n = min(20000, spp)
        res = autotune(probe["graph"], probe["syndromes"][:n].contiguous(), probe["shot_offset"])
        for b in batches:
            if b["code"] == code:
                b["graph"].set_kernel(res["best"])
        tuned[code] = {"kernel": res["best"], "ms_per_variant": {str(k): round(v, 3) for k, v in res["ms"].items()}}
    if args.kernel is not None:
        for b in batches:
            b["graph"].set_kernel(args.kernel)
        tuned = {code: {"kernel": args.kernel, "pinned": True} for code in {b["code"] for b in batches}}
    torch.cuda.synchronize()
    groups = {}
    for b in batches:
        groups.setdefault(b["graph"].info["kernel_id"], []).append(b)
    stream = torch.cuda.current_stream()

    # inputs and outputs resident in HBM; below a few L2 sizes (129 MB) a
    # restricted profiling case writes a 256 MB buffer before every step, so
    # that each step starts with its syndromes out of L2
    resident = sum(t.numel() * t.element_size() for b in batches
                   for t in [b["syndromes"], b["obs_true"]] + list(b["out"].values()))
    flush = torch.empty(64 << 20, dtype=torch.int32, device="cuda") if resident < (512 << 20) else None
    args.l2_note = ("L2 flushed before each step (a 256 MB write outside the decode events)" if flush is not None
                    else "inputs larger than L2 (no flush)")

    def step(events=None):
        if flush is not None:
            flush.zero_()
        for gi, (vid, items) in enumerate(sorted(groups.items())):
            if events is not None:
                events[gi][0].record(stream)
            pkg.decode_multi(items, stream)
            if events is not None:
                events[gi][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    for b in batches:
        b["counters"].zero_()
    step()     # one counted step: iterations and failures per batch
    torch.cuda.synchronize()
    iters = {id(b): int(b["counters"][2]) for b in batches}
    fails = {id(b): int(b["counters"][1]) for b in batches}

    # the roof: shared-memory bandwidth per SM clock, measured by the library's
    # microbenchmark before the timed region
    try:
        smem_peak = pkg.measure_smem_peak(local)
    except pkg.BpdcError as exc:
        smem_peak = {"error": str(exc)}

    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in groups] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        step(ev[k])
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = t0.elapsed_time(t1)
    if world > 1:
        tt = torch.tensor([ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    shots_per_step = len(batches) * spp * world
    if args.only or args.p is not None or args.kernel is not None:
        line_note = "restricted workload or pinned kernel variant (profiling case)"
    else:
        line_note = None
    value = shots_per_step * args.steps / (ms / 1e3)

    # dominant launch: per-variant average duration and algorithmic bytes
    per_variant = []
    for gi, (vid, items) in enumerate(sorted(groups.items())):
        d_ms = statistics.mean(ev[k][gi][0].elapsed_time(ev[k][gi][1]) for k in range(args.steps))
        eu = sum(iters[id(b)] * b["graph"].E for b in items)
        per_variant.append(dict(kernel_id=vid, ms=d_ms, edge_updates=eu, codes=sorted({b["code"] for b in items}),
                                shots=len(items) * spp))
    dom = max(per_variant, key=lambda v: v["ms"])
    sm_mhz = clk.get("sm_mhz") or 2070.0
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    nominal_gbs = nsm * SMEM_BYTES_PER_CLK_PER_SM * sm_mhz * 1e6 / 1e9
    if smem_peak.get("bytes_per_s"):
        peak_gbs = smem_peak["bytes_per_s"] / 1e9
        peak_src = (f"measured: shared-memory microbenchmark (bpdc_measure_smem_peak) before the timed region, "
                    f"{peak_gbs / nominal_gbs:.3f} of the nominal {nsm} SMs x {SMEM_BYTES_PER_CLK_PER_SM} B/clk "
                    f"x median sampled SM clock {sm_mhz:.0f} MHz = {nominal_gbs:.0f} GB/s")
    else:
        peak_gbs = nominal_gbs
        peak_src = (f"nominal: {nsm} SMs x {SMEM_BYTES_PER_CLK_PER_SM} B/clk x median sampled SM clock "
                    f"{sm_mhz:.0f} MHz (microbenchmark failed)")
    achieved_gbs = dom["edge_updates"] * EDGE_UPDATE_BYTES / (dom["ms"] / 1e3) / 1e9
    total_eu = sum(v["edge_updates"] for v in per_variant)
    traffic, smem_traffic, prof_file = profiled_traffic(dom["kernel_id"], dom["shots"], dom["edge_updates"])

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded counter sampler on the GPU, bit-identical to the CPU sampler)",
            "config": config_dict(args, world),
            "edge_updates_per_s": total_eu * world / (ms / args.steps / 1e3),
            "roofline": {"bound": "smem", "achieved": achieved_gbs, "peak": peak_gbs, "unit": "GB/s",
                         "frac": achieved_gbs / peak_gbs, "traffic": traffic,
                         "traffic_source": (f"DRAM bytes from profiles/{prof_file}, scaled by shots per launch"
                                            if traffic is not None else "no ncu summary of the current kernel"),
                         "smem_wavefront_bytes": smem_traffic,
                         "kernel": f"decode_kernel variant {dom['kernel_id']} ({'+'.join(dom['codes'])})",
                         "peak_source": peak_src,
                         "smem_microbenchmark": smem_peak,
                         "algorithmic_bytes": f"{EDGE_UPDATE_BYTES} B per edge-update x "
                                              f"{dom['edge_updates']} edge-updates per launch"},
            "per_variant_ms": {str(v["kernel_id"]): round(v["ms"], 3) for v in per_variant},
            "autotune": tuned,
            "note": line_note,
            "gpu_launches": args.steps * len(groups),
            "clocks": clk}

    if not args.no_extras:
        line["e2e"] = e2e_leg(args, pkg, torch, batches, groups, stream, world)
    # the remaining legs characterise one GPU (and the host CPU): N = 1 only
    if rank == 0 and world == 1 and not args.no_extras:
        extras(args, pkg, torch, batches, groups, stream, line, value, fails)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def e2e_leg(args, pkg, torch, batches, groups, stream, world):
    """The metric end to end through the public API: every step decodes this
    rank's shots from page-locked host syndromes into page-locked host
    corrections, status and logical flips with bpdc_decode_host (inside the
    library the copies of one piece of shots overlap the decoding of its
    neighbours); barrier and max over ranks.  The outputs are compared with
    those of the device-resident run."""
    host = []
    for b in batches:
        B = int(b["syndromes"].shape[0])
        host.append(dict(graph=b["graph"], syndromes=b["syndromes"].cpu().pin_memory(), shot_offset=b["shot_offset"],
                         out=b["graph"].alloc_host_outputs(B, iterations=False, logical=True)))
    h2d = sum(it["syndromes"].numel() * it["syndromes"].element_size() for it in host)
    d2h = sum(t.numel() * t.element_size() for it in host for t in it["out"].values())
    pkg.decode_host(host, chunk_shots=E2E_CHUNK, stream=stream)   # warm-up: staging allocation
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(args.steps):
        pkg.decode_host(host, chunk_shots=E2E_CHUNK, stream=stream)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    if world > 1:
        tt = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        ms = float(tt.item())
    same = all(bool((it["out"][k] == b["out"][k].cpu()).all()) for it, b in zip(host, batches)
               for k in ("corrections", "status", "logical_flips"))
    e2e = len(batches) * args.shots_per_point * args.steps * world / (ms / 1e3)
    return {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d * world, "d2h_bytes_per_step": d2h * world,
            "api": "bpdc_decode_host (page-locked host buffers, pieces of %d shots)" % E2E_CHUNK,
            "identical_outputs": same}


def extras(args, pkg, torch, batches, groups, stream, line, value, fails):
    import numpy as np

    # ---- the other two workload configurations: one line each, beside the headline
    peak_gbs = line["roofline"]["peak"]
    line["phenomenological"] = phenomenological_leg(args, pkg, torch, stream, peak_gbs)
    line["bb72_code_capacity"] = bb72_leg(args, pkg, torch, stream, peak_gbs)

    # ---- plain per-batch kernel on the same shots: throughput and identical results
    ref_out = {id(b): {k: v.clone() for k, v in b["out"].items()} for b in batches}
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    reps = max(1, min(args.steps, 3))
    t0.record(stream)
    for _ in range(reps):
        for b in batches:
            b["graph"].decode(b["syndromes"], b["shot_offset"], obs_true=b["obs_true"], out=b["out"],
                              persistent=False)
    t1.record(stream)
    torch.cuda.synchronize()
    plain = len(batches) * args.shots_per_point * reps / (t0.elapsed_time(t1) / 1e3)
    same = all(bool((b["out"][k] == ref_out[id(b)][k]).all()) for b in batches
               for k in ("corrections", "status", "logical_flips"))
    tot_fail = sum(fails.values())
    line["plain_kernel"] = {"value": plain, "unit": UNIT, "launches_per_step": len(batches),
                            "identical_outputs": same}
    line["ler"] = {f"{b['code']}@{b['p']}": fails[id(b)] / args.shots_per_point for b in batches}
    line["failures_per_step"] = tot_fail

    # ---- serving: seeded Poisson trace mixing circuit-level BB[[144,12,12]]
    # requests (12 rounds, p = 1e-3, T_iter = 1000) with code-capacity
    # BB[[72,12,6]] requests (p = 0.05), 1..1024 shots each
    from paper_2510_08695_gb300 import serving
    from bpdc_inputs import circuit
    Pc = circuit.circuit_level_problem("bb144", SERVE_ROUNDS, SERVE_P)
    gc = pkg.Graph.from_problem(Pc, pkg.Options(ms_scale=ALPHA, max_iter=SERVE_T_ITER))
    bb72 = [b for b in batches if b["code"] == "bb72" and b["p"] == 0.05][0]
    graphs = [gc, bb72["graph"]]
    pools = [gc.sample(60000, SEED + 50, 0)[0].cpu().pin_memory(),
             bb72["syndromes"][:200000].cpu().pin_memory()]
    calib = serving.poisson_trace(60, rate_per_s=1e9, n_graphs=len(graphs), seed=11)
    cal = serving.replay(serving.PlainDecoder(graphs), calib, pools)
    service_s = (max(r.done for r in cal) - min(r.arrival for r in cal)) / len(cal)

    def stats(reqs):
        l_us = np.array([(r.done - r.arrival) * 1e6 for r in reqs])
        n = np.array([r.syndromes.shape[0] for r in reqs])
        per_shot = np.repeat(l_us, n)     # every shot inherits its request's latency
        span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
        return {"p50_us": float(np.percentile(l_us, 50)), "p99_us": float(np.percentile(l_us, 99)),
                "p50_us_per_shot": float(np.percentile(per_shot, 50)),
                "p99_us_per_shot": float(np.percentile(per_shot, 99)), "shots_per_s": float(n.sum() / span)}

    sweep = []
    same = True
    status_counts = None
    for k, load in enumerate(SERVE_LOADS):
        rate = load / service_s
        trace = serving.poisson_trace(SERVE_REQUESTS, rate_per_s=rate, n_graphs=len(graphs), seed=12 + k)
        served = {}
        for name, eng in (("plain", serving.PlainDecoder(graphs)),
                          ("server", serving.Server(graphs, slots=SERVE_SLOTS))):
            served[name] = serving.replay(eng, trace, pools)
        same &= all(torch.equal(a.result[x], b.result[x]) for a, b in zip(served["plain"], served["server"])
                    for x in ("corrections", "status", "logical_flips"))
        sweep.append({"offered_load": load, "requests_per_s": rate,
                      "plain_per_request_kernel": stats(served["plain"]),
                      "continuous_batching_server": stats(served["server"])})
        if status_counts is None:
            st = torch.cat([r.result["status"] for r in served["server"] if r.graph_id == 0])
            status_counts = torch.bincount(st.long(), minlength=3).tolist()
    line["serving"] = {"trace": f"{SERVE_REQUESTS} Poisson requests of 1..1024 shots per load, half circuit-level "
                                f"BB[[144,12,12]] ({SERVE_ROUNDS} rounds, p={SERVE_P:g}, detector model "
                                f"{Pc.M}x{Pc.N} derived from the depth-8 syndrome circuit, H_DDM w=3, "
                                f"T_iter={SERVE_T_ITER}) and half code-capacity BB[[72,12,6]] at p=0.05; offered "
                                "load as a multiple of the plain decoder's measured capacity "
                                f"({1 / service_s:.1f} requests/s); latency = arrival to results on the host; "
                                "per shot: every shot takes its request's latency",
                       "sweep": sweep, "server_slots": SERVE_SLOTS, "identical_results": same,
                       "circuit_level_status_counts": status_counts}
    ref_load = min(sweep, key=lambda x: abs(x["offered_load"] - 0.7))
    line["p99_us_per_shot"] = ref_load["continuous_batching_server"]["p99_us_per_shot"]

    # ---- CUDA graph: a small request decoded by a direct multi-batch call
    # against the same allocation-free call replayed from a captured graph
    bb72b = [b for b in batches if b["code"] == "bb72" and b["p"] == 0.05][0]
    gg = bb72b["graph"]
    nb = 64
    sb = bb72b["syndromes"][:nb].clone()
    ob = gg.alloc_outputs(nb)
    it = [dict(graph=gg, syndromes=sb, shot_offset=0, out=ob)]
    pkg.decode_multi_noalloc(it)
    torch.cuda.synchronize()
    cs = torch.cuda.Stream()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=cs):
        pkg.decode_multi_noalloc(it)
    lat_g = {}
    for name, fn in (("direct_call", lambda: pkg.decode_multi_noalloc(it)), ("graph_replay", cg.replay)):
        for _ in range(20):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(300):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        lat_g[name] = {"p50_us": float(np.percentile(ts, 50) * 1e6), "p99_us": float(np.percentile(ts, 99) * 1e6)}
    line["cuda_graph"] = {"request": f"{nb} BB[[72,12,6]] shots at p=0.05, call to results on the device",
                          **lat_g}

    # ---- differentiable weighted BP: training throughput (forward + adjoint
    # kernels, batches of 4096 sampled shots, T = T_iter = 50 unrolled
    # iterations) for two objectives, and BP+DC with each set of learned
    # weights against plain BP+DC on 10^6 held-out shots per p
    import bpdc_inputs as bi
    from paper_2510_08695_gb300 import wbp
    P6 = bi.bb_problem("bb144", 0.06)
    gw = pkg.Graph.from_problem(P6, pkg.Options(variant=1, max_iter=T_ITER))
    wbp.train_weights(gw, T=WBP_T, steps=2, batch=WBP_BATCH, lr=WBP_LR, seed=SEED + 60)   # warm-up
    objectives = {}
    evals = {pp: pkg.Graph.from_problem(bi.bb_problem("bb144", pp), pkg.Options(variant=1, max_iter=T_ITER))
             for pp in WBP_EVAL_P}
    plain_ler = {}
    for pp, ge in evals.items():
        ge.set_weights(None)
        plain_ler[pp] = wbp.logical_error_rate(ge, WBP_EVAL_SHOTS, SEED + 62, 1 << 40)
    for obj in ("bce", "coset"):
        wbp.train_weights(gw, T=WBP_T, steps=2, batch=WBP_BATCH, lr=WBP_LR, seed=SEED + 60, objective=obj,
                          problem=P6)   # warm-up of the objective's own kernels
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        W, hist = wbp.train_weights(gw, T=WBP_T, steps=WBP_STEPS, batch=WBP_BATCH, lr=WBP_LR, seed=SEED + 61,
                                    objective=obj, problem=P6)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        ler = {}
        for pp, ge in evals.items():
            ge.set_weights(W)
            lw = wbp.logical_error_rate(ge, WBP_EVAL_SHOTS, SEED + 62, 1 << 40)
            ge.set_weights(None)
            lp = plain_ler[pp]
            kw, kp = round(lw * WBP_EVAL_SHOTS), round(lp * WBP_EVAL_SHOTS)
            # difference of two binomial proportions on the same number of shots
            sd = ((lw * (1 - lw) + lp * (1 - lp)) / WBP_EVAL_SHOTS) ** 0.5
            ler[f"bb144@{pp:g}"] = {"learned": lw, "plain": lp,
                                    "learned_ci95": wbp.binomial_interval(kw, WBP_EVAL_SHOTS),
                                    "plain_ci95": wbp.binomial_interval(kp, WBP_EVAL_SHOTS),
                                    "difference_sigmas": (lw - lp) / sd if sd > 0 else 0.0,
                                    "learned_weights_used": lw <= lp}
        objectives[obj] = {"train_s": t_train, "train_shots_per_s": WBP_STEPS * WBP_BATCH / t_train,
                           "loss_first_5_batches": sum(hist[:5]) / 5, "loss_last_5_batches": sum(hist[-5:]) / 5,
                           "ler_bp_dc_held_out": ler}
    line["weighted_bp"] = {
        "config": f"BB[[144,12,12]] code capacity, product-sum, {WBP_T} unrolled iterations (= T_iter of the "
                  f"decode that uses them), weights 2 x {WBP_T} x {P6.E} (per edge, iteration and direction), "
                  f"Adam lr {WBP_LR}, {WBP_STEPS} batches of {WBP_BATCH} shots sampled at p=0.06, checkpoints "
                  "every 5 iterations; objectives: bce = mean BCE of every iteration's posteriors against the "
                  "sampled errors; coset = probability that each iteration's residual flips a logical operator "
                  "plus the probability of a missed syndrome bit, averaged over the iterations (a correction in "
                  "the error's coset scores 0)",
        "objectives": objectives, "held_out_shots": WBP_EVAL_SHOTS,
        "rule": "learned weights are used only where their BP+DC logical error rate is no worse than plain"}

    # ---- CPU baseline: the FP64 oracle on a bounded sample of the workload
    import oracle
    from bpdc_inputs.sampler import sample_shots
    oracle.build()
    opts = oracle.Options(alpha=ALPHA, max_iter=T_ITER)
    samples = []
    for b in batches:
        n = oracle_sample_plan(b["code"])
        _, s, _ = sample_shots(b["P"], SEED, b["shot_offset"], n)
        t = time.perf_counter()
        oracle.decode_batch(b["P"], s, b["shot_offset"], opts)
        samples.append((n, time.perf_counter() - t))
    cpu = extrapolate_cpu(samples, args.shots_per_point)
    cores = oracle.max_threads()
    # one core, on a sixteenth of the sample
    oracle.set_threads(1)
    samples1 = []
    for b in batches:
        n = max(1, oracle_sample_plan(b["code"]) // 16)
        _, s, _ = sample_shots(b["P"], SEED, b["shot_offset"], n)
        t = time.perf_counter()
        oracle.decode_batch(b["P"], s, b["shot_offset"], opts)
        samples1.append((n, time.perf_counter() - t))
    oracle.set_threads(cores)
    line["cpu_baseline"] = {"value": cpu, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"first {oracle_sample_plan('bb72')} (BB) / {oracle_sample_plan('hgp2500')} "
                                      "(HGP) shots of each (code, p) point, CPU sampler, extrapolated per point "
                                      f"to {args.shots_per_point} shots; {sum(t for _, t in samples):.1f} s of CPU",
                            "value_1_core": extrapolate_cpu(samples1, args.shots_per_point),
                            "sample_1_core": f"first {oracle_sample_plan('bb72') // 16} (BB) / "
                                             f"{oracle_sample_plan('hgp2500') // 16} (HGP) shots of each point, "
                                             f"{sum(t for _, t in samples1):.1f} s"}


if __name__ == "__main__":
    main()
