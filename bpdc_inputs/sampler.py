"""Counter-based seeded shot sampler (CPU).

The hash is the SplitMix64 output function (Steele, Lea & Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014): the ``c``-th
output of a SplitMix64 stream whose state starts at ``key`` is

    z  = key + (c + 1) * 0x9E3779B97F4A7C15        (mod 2^64)
    z  = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z  = (z ^ (z >> 27)) * 0x94D049BB133111EB
    out = z ^ (z >> 31)

Shot ``i`` (global index) and column ``j`` of a problem with ``N`` columns
draw ``e_ij = [ (h(seed, i*N + j) >> 32) < floor(p_j * 2^32) ]``.  The GPU
sampler implements the same definition and is checked bit for bit against
this one.
"""
from __future__ import annotations

import numpy as np

__all__ = ["splitmix64_hash", "bernoulli_threshold", "sample_errors", "syndromes",
           "observables", "pack_bits", "unpack_bits", "sample_shots"]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_hash(key, ctr):
    """Vectorised SplitMix64 output ``h(key, ctr)`` (uint64)."""
    with np.errstate(over="ignore"):
        k = np.asarray(key, dtype=np.uint64)
        c = np.asarray(ctr, dtype=np.uint64)
        z = k + (c + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def bernoulli_threshold(p) -> np.ndarray:
    """floor(p * 2^32) as uint64, with p in [0, 1)."""
    p = np.asarray(p, dtype=np.float64)
    return np.floor(p * 4294967296.0).astype(np.uint64)


def sample_errors(priors, seed: int, shot_offset: int, B: int, chunk: int = 1 << 22) -> np.ndarray:
    """uint8 [B, N] error vectors for global shots shot_offset .. shot_offset+B-1."""
    priors = np.asarray(priors, dtype=np.float64)
    N = priors.shape[0]
    thr = bernoulli_threshold(priors)
    out = np.empty((B, N), dtype=np.uint8)
    rows_per = max(1, chunk // max(N, 1))
    cols = np.arange(N, dtype=np.uint64)
    for b0 in range(0, B, rows_per):
        b1 = min(B, b0 + rows_per)
        shots = np.arange(shot_offset + b0, shot_offset + b1, dtype=np.uint64)
        ctr = shots[:, None] * np.uint64(N) + cols[None, :]
        h = splitmix64_hash(np.uint64(seed), ctr)
        out[b0:b1] = ((h >> np.uint64(32)) < thr[None, :]).astype(np.uint8)
    return out


def syndromes(errors: np.ndarray, H) -> np.ndarray:
    """uint8 [B, M]: s = e H^T mod 2."""
    prod = H @ errors.T.astype(np.int32) if hasattr(H, "tocsr") else np.asarray(H, np.int32) @ errors.T.astype(np.int32)
    return (np.asarray(prod).T % 2).astype(np.uint8)


def observables(errors: np.ndarray, L) -> np.ndarray:
    """uint8 [B, K]: e L^T mod 2."""
    return syndromes(errors, L)


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """uint8 [B, n] -> uint32 [B, ceil(n/32)], bit c%32 of word c//32."""
    bits = np.asarray(bits, dtype=np.uint8) & 1
    B, n = bits.shape
    w = (n + 31) // 32
    padded = np.zeros((B, w * 32), dtype=np.uint8)
    padded[:, :n] = bits
    x = padded.reshape(B, w, 32).astype(np.uint32)
    return np.bitwise_or.reduce(x << np.arange(32, dtype=np.uint32), axis=2).astype(np.uint32)


def unpack_bits(words: np.ndarray, n: int) -> np.ndarray:
    words = np.asarray(words, dtype=np.uint32)
    B, w = words.shape
    bits = (words[:, :, None] >> np.arange(32, dtype=np.uint32)) & np.uint32(1)
    return bits.reshape(B, w * 32)[:, :n].astype(np.uint8)


def sample_shots(problem, seed: int, shot_offset: int, B: int):
    """(errors, syndromes, observables) as uint8 arrays for a Problem."""
    e = sample_errors(problem.priors, seed, shot_offset, B)
    return e, syndromes(e, problem.H), observables(e, problem.L)
