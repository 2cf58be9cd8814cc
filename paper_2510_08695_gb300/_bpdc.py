"""ctypes binding of libbpdc.so (argument marshalling only).

Every decoding step runs in the CUDA library; this module converts torch
tensors to device pointers and the caller's current CUDA stream to a
``cudaStream_t``.  It raises if the library is missing or a call fails: there
is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)


class BpdcError(RuntimeError):
    """A libbpdc call returned an error status."""

    def __init__(self, code: int, message: str):
        super().__init__(f"libbpdc error {code}: {message}")
        self.code = code


ERR_INVALID_ARG, ERR_DIM_MISMATCH, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6
ERR_CHECK = -7


class _Csr(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("cols", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("row_ptr", _i32p), ("col_idx", _i32p)]


class _Opts(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("ms_scale", ctypes.c_float), ("max_iter", ctypes.c_int32),
                ("dc_enable", ctypes.c_int32), ("dc_prior", ctypes.c_int32), ("tie_rel", ctypes.c_float),
                ("tie_seed", ctypes.c_uint64)]


class _Info(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int32), ("N", ctypes.c_int32), ("K", ctypes.c_int32), ("Md", ctypes.c_int32),
                ("E", ctypes.c_int64), ("syndrome_words", ctypes.c_int32),
                ("correction_words", ctypes.c_int32), ("logical_words", ctypes.c_int32),
                ("threads_per_shot", ctypes.c_int32), ("shots_per_block", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("smem_per_block", ctypes.c_int32),
                ("kernel_id", ctypes.c_int32)]


class _Outputs(ctypes.Structure):
    _fields_ = [("corrections", ctypes.c_void_p), ("status", ctypes.c_void_p),
                ("logical_flips", ctypes.c_void_p), ("obs_true", ctypes.c_void_p),
                ("iterations", ctypes.c_void_p), ("posterior_llr", ctypes.c_void_p),
                ("counters", ctypes.c_void_p), ("cut_in", ctypes.c_void_p)]


class _Batch(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_void_p), ("B", ctypes.c_int64), ("syndromes", ctypes.c_void_p),
                ("shot_offset", ctypes.c_uint64), ("out", _Outputs)]


HEADER = os.path.join(_build.ROOT, "include", "bpdc.h")


def declared_symbols() -> list[str]:
    """Function names declared in include/bpdc.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*(bpdc_\w+)\s*\(", text, re.M)))


def library_path() -> str:
    """Path of the library load() uses (the checked build under BPDC_CHECKED=1)."""
    return _build.LIB_CHECKED if os.environ.get("BPDC_CHECKED") == "1" else _build.LIB


def load(build_if_missing: bool = True):
    """Loads libbpdc.so (building it first if needed); libbpdc_checked.so, the
    bounds-checked debugging build, when the environment sets BPDC_CHECKED=1."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if build_if_missing and _build.stale(path):
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libbpdc.so not built at {path}; run paper_2510_08695_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i64, u64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32
    sig = {
        "bpdc_opts_default": (None, [ctypes.POINTER(_Opts)]),
        "bpdc_graph_create": (ctypes.c_int, [ctypes.POINTER(_Csr)] * 3 +
                              [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_Opts), ctypes.c_int,
                               ctypes.POINTER(vp)]),
        "bpdc_graph_destroy": (ctypes.c_int, [vp]),
        "bpdc_graph_get_info": (ctypes.c_int, [vp, ctypes.POINTER(_Info)]),
        "bpdc_graph_set_plan": (ctypes.c_int, [vp, i32]),
        "bpdc_graph_set_kernel": (ctypes.c_int, [vp, i32]),
        "bpdc_kernel_count": (ctypes.c_int, []),
        "bpdc_graph_set_layout": (ctypes.c_int, [vp, i32]),
        "bpdc_layout_plan": (ctypes.c_int, [ctypes.POINTER(_Csr), i32, i32, _i32p, _i32p]),
        "bpdc_layout_plan_slots": (ctypes.c_int, [ctypes.POINTER(_Csr), i32, i32, i32, _i32p, _i32p, _i32p]),
        "bpdc_decode": (ctypes.c_int, [vp, i64, vp, u64, ctypes.POINTER(_Outputs), ctypes.c_int, vp]),
        "bpdc_decode_multi": (ctypes.c_int, [ctypes.POINTER(_Batch), i32, vp]),
        "bpdc_decode_multi_noalloc": (ctypes.c_int, [ctypes.POINTER(_Batch), i32, vp]),
        "bpdc_decode_host": (ctypes.c_int, [ctypes.POINTER(_Batch), i32, i64, vp]),
        "bpdc_cut_select": (ctypes.c_int, [vp, i64, vp, u64, vp, vp]),
        "bpdc_sample": (ctypes.c_int, [vp, i64, u64, u64, vp, vp, vp, vp]),
        "bpdc_graph_sync_status": (ctypes.c_int, [vp, vp]),
        "bpdc_check_status": (ctypes.c_int, [i32, _i32p, ctypes.POINTER(ctypes.c_int64)]),
        "bpdc_debug_fail_allocations": (ctypes.c_int, [i32, i32]),
        "bpdc_graph_set_weights": (ctypes.c_int, [vp, vp, i32, ctypes.c_float]),
        "bpdc_wbp_workspace_size": (ctypes.c_int, [vp, i64, i32, i32, ctypes.POINTER(ctypes.c_size_t)]),
        "bpdc_wbp_forward": (ctypes.c_int, [vp, i64, vp, vp, i32, ctypes.c_float, i32, vp, vp, ctypes.c_size_t,
                                            vp]),
        "bpdc_decode_backward": (ctypes.c_int, [vp, i64, vp, vp, i32, ctypes.c_float, i32, vp, vp, vp,
                                                ctypes.c_size_t, vp]),
        "bpdc_measure_smem_peak": (ctypes.c_int, [i32, i32, ctypes.POINTER(ctypes.c_double),
                                                  ctypes.POINTER(ctypes.c_int32)]),
        "bpdc_last_error": (ctypes.c_char_p, []),
        "bpdc_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        raise BpdcError(rc, _lib.bpdc_last_error().decode())


@dataclass
class Options:
    """Decoder options (see bpdc_opts in include/bpdc.h)."""
    ms_scale: float = 0.625
    max_iter: int = 50
    dc_enable: int = 1
    dc_prior: int = 0
    tie_rel: float = 1e-5
    tie_seed: int = 0x2510086950
    variant: int = 0

    def _c(self) -> _Opts:
        return _Opts(self.variant, self.ms_scale, self.max_iter, self.dc_enable, self.dc_prior,
                     self.tie_rel, self.tie_seed)


def _csr(m):
    m = m.tocsr()
    ptr = np.ascontiguousarray(m.indptr, dtype=np.int32)
    col = np.ascontiguousarray(m.indices, dtype=np.int32)
    c = _Csr(m.shape[0], m.shape[1], int(m.nnz), ptr.ctypes.data_as(_i32p), col.ctypes.data_as(_i32p))
    return c, (ptr, col)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Graph:
    """A device-resident decoding problem (H, L, D, priors)."""

    def __init__(self, H, L, D, priors, opts: Options | None = None, device: int = 0):
        lib = load()
        self.opts = opts or Options()
        h, keep_h = _csr(H)
        l, keep_l = _csr(L)
        d, keep_d = _csr(D)
        pr = np.ascontiguousarray(priors, dtype=np.float64)
        handle = ctypes.c_void_p()
        o = self.opts._c()
        _check(lib.bpdc_graph_create(ctypes.byref(h), ctypes.byref(l), ctypes.byref(d),
                                     pr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(o),
                                     int(device), ctypes.byref(handle)))
        self.handle = handle
        self.device = int(device)
        self._refresh()

    @classmethod
    def from_problem(cls, problem, opts: Options | None = None, device: int = 0) -> "Graph":
        return cls(problem.H, problem.L, problem.D, problem.priors, opts, device)

    def _refresh(self):
        info = _Info()
        _check(_lib.bpdc_graph_get_info(self.handle, ctypes.byref(info)))
        self.info = {f: getattr(info, f) for f, _ in _Info._fields_}
        self.M, self.N, self.K, self.Md, self.E = info.M, info.N, info.K, info.Md, info.E
        self.MW, self.NW, self.KW = info.syndrome_words, info.correction_words, info.logical_words

    def set_plan(self, threads_per_shot: int):
        _check(_lib.bpdc_graph_set_plan(self.handle, int(threads_per_shot)))
        self._refresh()

    def set_layout(self, mode: int):
        """1: bank-conflict-aware message layout (default); 0: identity layout."""
        _check(_lib.bpdc_graph_set_layout(self.handle, int(mode)))
        self._refresh()

    def set_kernel(self, kernel_id: int):
        _check(_lib.bpdc_graph_set_kernel(self.handle, int(kernel_id)))
        self._refresh()

    def kernels(self) -> list[int]:
        """Kernel variants that accept this graph."""
        cur = self.info["kernel_id"]
        ok = []
        for k in range(_lib.bpdc_kernel_count()):
            if _lib.bpdc_graph_set_kernel(self.handle, k) == 0:
                ok.append(k)
        _check(_lib.bpdc_graph_set_kernel(self.handle, cur))
        self._refresh()
        return ok

    def close(self):
        if getattr(self, "handle", None):
            _lib.bpdc_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- decoding -----------------------------------------------------------
    def alloc_outputs(self, B: int, iterations=True, logical=True, posterior=False):
        import torch
        dev = torch.device("cuda", self.device)
        out = dict(corrections=torch.empty((B, self.NW), dtype=torch.int32, device=dev),
                   status=torch.empty((B,), dtype=torch.uint8, device=dev))
        if logical:
            out["logical_flips"] = torch.empty((B, max(self.KW, 1)), dtype=torch.int32, device=dev)
        if iterations:
            out["iterations"] = torch.empty((B,), dtype=torch.int32, device=dev)
        if posterior:
            out["posterior_llr"] = torch.empty((B, self.N), dtype=torch.float32, device=dev)
        return out

    def alloc_host_outputs(self, B: int, iterations=True, logical=True):
        """Page-locked host outputs for decode_host (same shapes as alloc_outputs)."""
        import torch
        out = dict(corrections=torch.empty((B, self.NW), dtype=torch.int32, pin_memory=True),
                   status=torch.empty((B,), dtype=torch.uint8, pin_memory=True))
        if logical:
            out["logical_flips"] = torch.empty((B, max(self.KW, 1)), dtype=torch.int32, pin_memory=True)
        if iterations:
            out["iterations"] = torch.empty((B,), dtype=torch.int32, pin_memory=True)
        return out

    def _outputs(self, out, obs_true=None, counters=None, cut_in=None) -> _Outputs:
        return _Outputs(_ptr(out["corrections"]), _ptr(out["status"]), _ptr(out.get("logical_flips")),
                        _ptr(obs_true), _ptr(out.get("iterations")), _ptr(out.get("posterior_llr")),
                        _ptr(counters), _ptr(cut_in))

    def decode(self, syndromes, shot_offset: int = 0, *, obs_true=None, counters=None, cut_in=None,
               out=None, persistent: bool = True, iterations: bool = True, posterior: bool = False,
               stream=None):
        """Decodes ``syndromes`` (int32 [B, ceil(M/32)] on the graph's device).

        Returns a dict of device tensors: corrections [B, ceil(N/32)] int32 (bit
        words), status [B] uint8, logical_flips [B, ceil(K/32)], iterations [B]
        (first run in the low 16 bits, second run in the high 16 bits) and, with
        ``posterior=True``, posterior_llr [B, N] float32.
        """
        B = int(syndromes.shape[0])
        assert syndromes.shape[1] == self.MW and syndromes.is_cuda and syndromes.is_contiguous()
        if out is None:
            out = self.alloc_outputs(B, iterations=iterations, posterior=posterior)
        o = self._outputs(out, obs_true, counters, cut_in)
        _check(_lib.bpdc_decode(self.handle, B, _ptr(syndromes), ctypes.c_uint64(shot_offset),
                                ctypes.byref(o), int(bool(persistent)), _stream_ptr(stream)))
        return out

    def cut_select(self, posterior_llr, shot_offset: int = 0, stream=None):
        """Cut sets chosen from posterior LLRs (float32 [B, N] on device)."""
        import torch
        B = int(posterior_llr.shape[0])
        assert posterior_llr.dtype == torch.float32 and posterior_llr.shape[1] == self.N
        cut = torch.empty((B, self.NW), dtype=torch.int32, device=posterior_llr.device)
        _check(_lib.bpdc_cut_select(self.handle, B, _ptr(posterior_llr), ctypes.c_uint64(shot_offset),
                                    _ptr(cut), _stream_ptr(stream)))
        return cut

    def sample(self, B: int, seed: int, shot_offset: int = 0, errors: bool = False, stream=None):
        """GPU shot sampler: (syndromes, observables, errors or None) as int32 bit words."""
        import torch
        dev = torch.device("cuda", self.device)
        syn = torch.empty((B, self.MW), dtype=torch.int32, device=dev)
        obs = torch.empty((B, max(self.KW, 1)), dtype=torch.int32, device=dev)
        err = torch.empty((B, self.NW), dtype=torch.int32, device=dev) if errors else None
        _check(_lib.bpdc_sample(self.handle, int(B), ctypes.c_uint64(seed), ctypes.c_uint64(shot_offset),
                                _ptr(syn), _ptr(obs), _ptr(err), _stream_ptr(stream)))
        return syn, obs, err

    def set_weights(self, weights=None, clip: float = 20.0):
        """Learned weighted-BP weights [2, T, E] (CPU or CUDA tensor, or numpy)
        used by decode / decode_multi; None restores plain BP."""
        if weights is None:
            _check(_lib.bpdc_graph_set_weights(self.handle, None, 0, ctypes.c_float(0.0)))
            return
        w = np.ascontiguousarray(np.asarray(weights.detach().cpu() if hasattr(weights, "detach") else weights,
                                            dtype=np.float32))
        assert w.ndim == 3 and w.shape[0] == 2 and w.shape[2] == self.E, w.shape
        _check(_lib.bpdc_graph_set_weights(self.handle, w.ctypes.data_as(ctypes.c_void_p), int(w.shape[1]),
                                           ctypes.c_float(clip)))
        self._refresh()

    def sync_status(self, stream=None):
        _check(_lib.bpdc_graph_sync_status(self.handle, _stream_ptr(stream)))


def _batches(items):
    arr = (_Batch * len(items))()
    for i, it in enumerate(items):
        g = it["graph"]
        arr[i].graph = g.handle
        arr[i].B = int(it["syndromes"].shape[0])
        arr[i].syndromes = it["syndromes"].data_ptr()
        arr[i].shot_offset = int(it.get("shot_offset", 0))
        arr[i].out = g._outputs(it["out"], it.get("obs_true"), it.get("counters"), it.get("cut_in"))
    return arr


def debug_fail_allocations(skip: int, count: int):
    """bpdc_debug_fail_allocations: after ``skip`` allocations of the library,
    the next ``count`` fail as if memory were exhausted (0: off)."""
    _check(load().bpdc_debug_fail_allocations(int(skip), int(count)))


def check_status(device: int = 0):
    """bpdc_check_status (checked build only): None if no bounds check failed
    on ``device`` since the last call, else (site, index) of the first
    failure; the latch is cleared.  Raises BpdcError in the normal build."""
    site, index = ctypes.c_int32(), ctypes.c_int64()
    rc = load().bpdc_check_status(int(device), ctypes.byref(site), ctypes.byref(index))
    if rc == ERR_CHECK:
        return site.value, index.value
    _check(rc)
    return None


def decode_multi(items, stream=None):
    """Decodes several batches (possibly of different graphs) in persistent launches.

    ``items``: list of dicts with keys graph, syndromes, shot_offset, out and
    optionally obs_true, counters.
    """
    lib = load()
    _check(lib.bpdc_decode_multi(_batches(items), len(items), _stream_ptr(stream)))


def decode_host(items, chunk_shots: int = 0, stream=None):
    """bpdc_decode_host: the decode of ``decode_multi`` from and into HOST
    tensors (page-locked for copy / compute overlap), pipelined in pieces of
    at most ``chunk_shots`` shots (0: the library's default).  ``items`` as for
    decode_multi, with CPU tensors for syndromes, obs_true and every output;
    synchronous."""
    import torch
    for it in items:
        g, syn, out = it["graph"], it["syndromes"], it["out"]
        B = int(syn.shape[0])
        want = {"syndromes": (syn, (B, g.MW), torch.int32), "obs_true": (it.get("obs_true"), (B, max(g.KW, 1)), torch.int32),
                "corrections": (out["corrections"], (B, g.NW), torch.int32), "status": (out["status"], (B,), torch.uint8),
                "logical_flips": (out.get("logical_flips"), (B, max(g.KW, 1)), torch.int32),
                "iterations": (out.get("iterations"), (B,), torch.int32)}
        for name, (t, shape, dtype) in want.items():
            if t is None:
                continue
            if t.is_cuda or not t.is_contiguous() or tuple(t.shape) != shape or t.dtype != dtype:
                raise ValueError(f"decode_host: {name} must be a contiguous CPU {dtype} tensor of shape {shape}")
    lib = load()
    _check(lib.bpdc_decode_host(_batches(items), len(items), int(chunk_shots), _stream_ptr(stream)))


def decode_multi_noalloc(items, stream=None):
    """bpdc_decode_multi_noalloc: the same decode with the library's fixed
    device scratch (no allocation in the call); at most 16 batches, all on one
    kernel variant.  The output tensors in ``items`` must be allocated by the
    caller beforehand."""
    lib = load()
    _check(lib.bpdc_decode_multi_noalloc(_batches(items), len(items), _stream_ptr(stream)))


def wbp_workspace(graph: Graph, B: int, T: int, ckpt_every: int):
    """A device workspace (uint8 tensor) for bpdc_wbp_forward / bpdc_decode_backward."""
    import torch
    n = ctypes.c_size_t()
    _check(load().bpdc_wbp_workspace_size(graph.handle, int(B), int(T), int(ckpt_every), ctypes.byref(n)))
    return torch.empty(max(int(n.value), 1), dtype=torch.uint8, device=torch.device("cuda", graph.device))


def wbp_forward(graph: Graph, syndromes, weights, T: int, clip: float, ckpt_every: int, workspace,
                posteriors=None, stream=None):
    """bpdc_wbp_forward: posteriors [B, T, N] float32 of weighted BP."""
    import torch
    B = int(syndromes.shape[0])
    if posteriors is None:
        posteriors = torch.empty((B, T, graph.N), dtype=torch.float32, device=syndromes.device)
    _check(load().bpdc_wbp_forward(graph.handle, B, _ptr(syndromes), _ptr(weights), int(T), float(clip),
                                   int(ckpt_every), _ptr(posteriors), _ptr(workspace), workspace.numel(),
                                   _stream_ptr(stream)))
    return posteriors


def decode_backward(graph: Graph, syndromes, weights, T: int, clip: float, ckpt_every: int, grad_posteriors,
                    workspace, grad_weights=None, stream=None):
    """bpdc_decode_backward: dLoss/dW [2, T, E] from dLoss/dL [B, T, N]."""
    import torch
    B = int(syndromes.shape[0])
    if grad_weights is None:
        grad_weights = torch.empty_like(weights)
    _check(load().bpdc_decode_backward(graph.handle, B, _ptr(syndromes), _ptr(weights), int(T), float(clip),
                                       int(ckpt_every), _ptr(grad_posteriors), _ptr(grad_weights),
                                       _ptr(workspace), workspace.numel(), _stream_ptr(stream)))
    return grad_weights


def layout_plan(H, G: int, optimize: bool = True, pass_slots=None):
    """Host-only layout planner: (pos_of_var [N], edge_round [nnz] in H's CSR
    order); ``pass_slots`` (message slots of each variable pass) places the
    variables under a slot profile (bpdc_layout_plan_slots)."""
    lib = load()
    h, keep = _csr(H)
    pos = np.zeros(h.cols, np.int32)
    rnd = np.zeros(max(int(h.nnz), 1), np.int32)
    if pass_slots is None:
        _check(lib.bpdc_layout_plan(ctypes.byref(h), int(G), int(bool(optimize)), pos.ctypes.data_as(_i32p),
                                    rnd.ctypes.data_as(_i32p)))
    else:
        ps = np.ascontiguousarray(pass_slots, dtype=np.int32)
        _check(lib.bpdc_layout_plan_slots(ctypes.byref(h), int(G), int(bool(optimize)), int(ps.size),
                                          ps.ctypes.data_as(_i32p), pos.ctypes.data_as(_i32p),
                                          rnd.ctypes.data_as(_i32p)))
    return pos, rnd[:int(h.nnz)]


def measure_smem_peak(device: int = 0, reps: int = 40000) -> dict:
    """Shared-memory bandwidth microbenchmark (bpdc_measure_smem_peak)."""
    lib = load()
    bps = ctypes.c_double()
    sms = ctypes.c_int32()
    _check(lib.bpdc_measure_smem_peak(int(device), int(reps), ctypes.byref(bps), ctypes.byref(sms)))
    return dict(bytes_per_s=bps.value, num_sms=sms.value)


def version() -> str:
    return load().bpdc_version().decode()
