"""Python access to the FP64 CPU oracle of BP+DC (``bpdc_oracle.c``).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` import this package.  The
oracle is plain C compiled with gcc (``-O2 -fopenmp -ffp-contract=off``); it
shares no code with the CUDA decoder.

Parity status of the functions exported here (pins live in ``tests/``):
    bp()            pinned (exact marginals / min-energy on trees, invariants)
    dc_select()     pinned (invariants: one cut per row, windowed maxima,
                    row-order independence)
    decode_batch()  pinned (Algorithm 1 == Algorithm 2, invariants,
                    Table II first-BP failure rate as a soft statistical pin)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bpdc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)


class _Problem(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int32), ("N", ctypes.c_int32),
                ("h_row_ptr", _i32p), ("h_col", _i32p),
                ("Md", ctypes.c_int32), ("d_row_ptr", _i32p), ("d_col", _i32p),
                ("K", ctypes.c_int32), ("l_row_ptr", _i32p), ("l_col", _i32p),
                ("prior", _f64p)]


class _Opts(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("alpha", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("dc_enable", ctypes.c_int32),
                ("dc_prior", ctypes.c_int32), ("cut_form", ctypes.c_int32),
                ("tie_rel", ctypes.c_double), ("tie_seed", ctypes.c_uint64)]


@dataclass
class Options:
    """Decoder options (same meaning as the CUDA library's options)."""
    variant: int = 0          # 0 normalized min-sum, 1 product-sum
    alpha: float = 0.625      # min-sum scale
    max_iter: int = 50        # T_iter
    dc_enable: int = 1
    dc_prior: int = 0         # 0: second BP on priors p; 1: on first-run posterior
    cut_form: int = 0         # 0: DeleteColumns (Algorithm 1); 1: zero prior (Algorithm 2)
    tie_rel: float = 1e-5
    tie_seed: int = 0x2510086950

    def _c(self):
        return _Opts(self.variant, self.alpha, self.max_iter, self.dc_enable, self.dc_prior,
                     self.cut_form, self.tie_rel, self.tie_seed)


def compile_oracle(src: str, out: str) -> str:
    """gcc the oracle source ``src`` into the shared library ``out``."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
                           "-fno-fast-math", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (if stale)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_oracle(_SRC, _LIB)
    return _LIB


def _ptr(a, t):
    return None if a is None else a.ctypes.data_as(t)


class _Prob:
    """Keeps the numpy arrays of a problem alive next to its C view."""

    def __init__(self, problem):
        H, D, L = problem.H.tocsr(), problem.D.tocsr(), problem.L.tocsr()
        D = D.copy()
        D.sort_indices()
        self.arrs = [np.ascontiguousarray(x, dtype=np.int32) for x in
                     (H.indptr, H.indices, D.indptr, D.indices, L.indptr, L.indices)]
        self.prior = np.ascontiguousarray(problem.priors, dtype=np.float64)
        a = self.arrs
        self.c = _Problem(H.shape[0], H.shape[1], _ptr(a[0], _i32p), _ptr(a[1], _i32p),
                          D.shape[0], _ptr(a[2], _i32p), _ptr(a[3], _i32p),
                          L.shape[0], _ptr(a[4], _i32p), _ptr(a[5], _i32p),
                          _ptr(self.prior, _f64p))
        self.M, self.N, self.K, self.Md = H.shape[0], H.shape[1], L.shape[0], D.shape[0]


def prior_llr(p):
    p = np.asarray(p, dtype=np.float64)
    with np.errstate(divide="ignore"):
        return np.log((1.0 - p) / p)


class Oracle:
    """One loaded build of the oracle library."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        lib.oracle_hash.restype = ctypes.c_uint64
        lib.oracle_hash.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.oracle_bp.restype = ctypes.c_int
        lib.oracle_bp.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(_Opts), _u8p, _f64p,
                                  ctypes.c_int, _u8p, _f64p, _i32p]
        lib.oracle_dc_select.restype = None
        lib.oracle_dc_select.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(_Opts), _f64p,
                                         ctypes.c_uint64, _u8p]
        lib.oracle_decode_batch.restype = ctypes.c_int
        lib.oracle_decode_batch.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(_Opts),
                                            ctypes.c_int64, _u8p, ctypes.c_uint64, _u8p, _u8p,
                                            _i32p, _i32p, _f64p, _f64p, _u8p, _u8p, ctypes.c_int]
        lib.oracle_max_threads.restype = ctypes.c_int
        self.lib = lib
        self.Options = Options

    def hash64(self, key: int, ctr: int) -> int:
        return int(self.lib.oracle_hash(key, ctr))

    def bp(self, problem, syndrome, lam=None, opts: Options | None = None, early_stop: bool = True):
        """One BP_decode run.  Returns (converged, e_hat, posterior_llr, iterations)."""
        opts = opts or Options()
        pr = _Prob(problem)
        s = np.ascontiguousarray(syndrome, dtype=np.uint8)
        lam = prior_llr(problem.priors) if lam is None else np.ascontiguousarray(lam, dtype=np.float64)
        e = np.zeros(pr.N, np.uint8)
        post = np.zeros(pr.N, np.float64)
        it = np.zeros(1, np.int32)
        c_opts = opts._c()
        ok = self.lib.oracle_bp(ctypes.byref(pr.c), ctypes.byref(c_opts), _ptr(s, _u8p),
                                _ptr(lam, _f64p), int(early_stop), _ptr(e, _u8p),
                                _ptr(post, _f64p), _ptr(it, _i32p))
        return bool(ok), e, post, int(it[0])

    def dc_select(self, problem, posterior, shot: int, opts: Options | None = None):
        """Cut set (uint8 mask over columns) chosen from a posterior LLR vector."""
        opts = opts or Options()
        pr = _Prob(problem)
        post = np.ascontiguousarray(posterior, dtype=np.float64)
        cut = np.zeros(pr.N, np.uint8)
        c_opts = opts._c()
        self.lib.oracle_dc_select(ctypes.byref(pr.c), ctypes.byref(c_opts), _ptr(post, _f64p),
                                  ctypes.c_uint64(shot), _ptr(cut, _u8p))
        return cut

    def decode_batch(self, problem, syndromes, shot_offset: int = 0, opts: Options | None = None,
                     want_post: bool = False, want_post1: bool = False, want_cut: bool = False,
                     nthreads: int = 0):
        """Algorithm 1 on every shot.  ``syndromes`` is uint8 [B, M].

        Returns a dict with e_hat [B,N] u8, status [B] u8, iters1/iters2 [B] i32,
        obs_pred [B,K] u8 and, on request, post / post1 [B,N] f64 and cut [B,N] u8.
        """
        opts = opts or Options()
        pr = _Prob(problem)
        syn = np.ascontiguousarray(syndromes, dtype=np.uint8)
        B = syn.shape[0]
        assert syn.shape[1] == pr.M
        out = dict(e_hat=np.zeros((B, pr.N), np.uint8), status=np.zeros(B, np.uint8),
                   iters1=np.zeros(B, np.int32), iters2=np.zeros(B, np.int32),
                   obs_pred=np.zeros((B, pr.K), np.uint8))
        if want_post:
            out["post"] = np.zeros((B, pr.N), np.float64)
        if want_post1:
            out["post1"] = np.zeros((B, pr.N), np.float64)
        if want_cut:
            out["cut"] = np.zeros((B, pr.N), np.uint8)
        c_opts = opts._c()
        self.lib.oracle_decode_batch(
            ctypes.byref(pr.c), ctypes.byref(c_opts), B, _ptr(syn, _u8p),
            ctypes.c_uint64(shot_offset), _ptr(out["e_hat"], _u8p), _ptr(out["status"], _u8p),
            _ptr(out["iters1"], _i32p), _ptr(out["iters2"], _i32p), _ptr(out.get("post"), _f64p),
            _ptr(out.get("post1"), _f64p), _ptr(out.get("cut"), _u8p), _ptr(out["obs_pred"], _u8p),
            int(nthreads))
        return out

    def max_threads(self) -> int:
        return int(self.lib.oracle_max_threads())

    def set_threads(self, n: int) -> None:
        self.lib.oracle_set_threads(ctypes.c_int(int(n)))


def _load() -> Oracle:
    global _lib
    if _lib is None:
        _lib = Oracle(build())
    return _lib


def hash64(key: int, ctr: int) -> int:
    return _load().hash64(key, ctr)


def bp(*args, **kw):
    return _load().bp(*args, **kw)


def dc_select(*args, **kw):
    return _load().dc_select(*args, **kw)


def decode_batch(*args, **kw):
    return _load().decode_batch(*args, **kw)


def max_threads() -> int:
    return _load().max_threads()


def set_threads(n: int) -> None:
    """Threads of the oracle's loop over shots (timing of the CPU baseline)."""
    _load().set_threads(n)
