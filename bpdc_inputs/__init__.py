"""Seeded input generators shared by the oracle tests and the GPU path.

Holds code constructions (BB, hypergraph-product, phenomenological detector
models), GF(2) helpers used to build them, and the counter-based shot
sampler.  No decoder arithmetic lives here.
"""
from . import gf2, codes, sampler  # noqa: F401
from .codes import Problem  # noqa: F401

import functools


@functools.lru_cache(maxsize=None)
def _bb(name):
    hx, hz = codes.bb_code(name)
    oz = codes.logical_basis(hx, hz)
    return hx, hz, oz


@functools.lru_cache(maxsize=None)
def _hgp(n=40, seed=2510):
    h = codes.gallager_regular(n, 3, 4, seed)
    hx, hz = codes.hgp_matrices(h, h)
    oz = codes.logical_basis(hx, hz)
    return h, hx, hz, oz


def bb_problem(name: str, p: float) -> Problem:
    """Code-capacity problem for a Table I BB code at bit-flip rate p."""
    hx, hz, oz = _bb(name)
    return codes.code_capacity_problem(hx, hz, p, f"{name}_p{p:g}", oz=oz)


@functools.lru_cache(maxsize=None)
def _surface(d):
    hx, hz = codes.rotated_surface_code(d)
    oz = codes.logical_basis(hx, hz)
    return hx, hz, oz


def surface_problem(d: int, p: float) -> Problem:
    """Code-capacity problem for the rotated surface code [[d^2, 1, d]]."""
    hx, hz, oz = _surface(d)
    return codes.code_capacity_problem(hx, hz, p, f"surface{d}_p{p:g}", oz=oz)


def hgp_problem(p: float, n: int = 40, seed: int = 2510) -> Problem:
    """Code-capacity problem for the hypergraph product of a seeded (3,4)-regular code."""
    _, hx, hz, oz = _hgp(n, seed)
    return codes.code_capacity_problem(hx, hz, p, f"hgp{hz.shape[1]}_p{p:g}", oz=oz)


def phenomenological_bb_problem(name: str, T: int, p: float, q: float | None = None) -> Problem:
    """Phenomenological problem for a Table I BB code with T noisy rounds + 1 perfect."""
    hx, hz, oz = _bb(name)
    return codes.phenomenological_problem(hx, hz, T, p, q, name=f"{name}_phen_T{T}_p{p:g}", oz=oz)
