"""Kernel-variant autotuner.

The compiled decode kernels differ in threads per shot (G), the number of
checks and variables each thread owns, the row and column weights they are
specialised for, and their register budget (resident blocks per SM).  For a
graph the autotuner times every variant that accepts it on a sample of shots
(CUDA events on the current stream, after a warm-up launch) and keeps the
fastest; the graph's automatically chosen variant stays unless another is
more than ``margin`` faster, so that near-ties do not flip between runs.
Results are identical for every variant; only the speed differs.
"""
from __future__ import annotations


def choose(times: dict, incumbent: int, margin: float = 0.02) -> int:
    """The variant to keep given measured times: the fastest, unless the
    incumbent was timed and the fastest beats it by no more than ``margin``."""
    best = min(times, key=times.get)
    if incumbent in times and times[best] > (1.0 - margin) * times[incumbent]:
        return incumbent
    return best


def autotune(graph, syndromes, shot_offset: int = 0, reps: int = 2, persistent: bool = True,
             verbose: bool = False, margin: float = 0.02) -> dict:
    """Selects the fastest kernel variant for ``graph`` on ``syndromes``.

    Returns ``{"best": kernel_id, "ms": {kernel_id: ms per decode}}``.
    """
    import torch
    B = int(syndromes.shape[0])
    incumbent = graph.info["kernel_id"]
    times = {}
    for k in graph.kernels():
        graph.set_kernel(k)
        out = graph.alloc_outputs(B, iterations=False, logical=True)
        graph.decode(syndromes, shot_offset, out=out, persistent=persistent)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            graph.decode(syndromes, shot_offset, out=out, persistent=persistent)
        e1.record()
        torch.cuda.synchronize()
        times[k] = e0.elapsed_time(e1) / reps
        if verbose:
            print(f"kernel {k}: G={graph.info['threads_per_shot']} blocks/SM={graph.info['blocks_per_sm']} "
                  f"{times[k]:.3f} ms", flush=True)
    best = choose(times, incumbent, margin)
    graph.set_kernel(best)
    return {"best": best, "ms": times}
