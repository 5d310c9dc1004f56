"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds random-number generation only: no lattice constant, no
equilibrium, no part of the method's arithmetic.  Both sides of every parity
check receive the same arrays from here and build everything else with their
own code.

Generators:
  * SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
    generators", OOPSLA 2014): a counter-based stream, so element k of a draw
    depends only on (seed, k).  Used for the initial temperature noise of the
    cavity runs and for random population states.
  * numpy's PCG64 for the Ra / mesh-size draws of the batched sweep and the
    Gaussian weights of the warm-start network tests.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def splitmix64(count: int, seed: int = 0, offset: int = 0) -> np.ndarray:
    """Return `count` raw 64-bit SplitMix64 outputs for counters offset+1 .. offset+count."""
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(count: int, seed: int = 0, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(count, seed, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def temperature_noise(shape, amplitude: float = 1e-6, seed: int = 0) -> np.ndarray:
    """Uniform noise in [-amplitude, amplitude) over a grid, in row-major node order.

    `shape` is (Ny, Nx) or (Nz, Ny, Nx): x varies fastest.
    """
    n = int(np.prod(shape))
    return (amplitude * (2.0 * uniform01(n, seed) - 1.0)).reshape(shape)


def random_populations(q: int, shape, seed: int, spread: float = 0.05,
                       base: float | None = None) -> np.ndarray:
    """Positive random populations b * (1 + spread * r), r uniform in [-1, 1).

    Returns shape (q, *shape).  `base` defaults to 1/q, so the density of a node
    is about 1; no lattice weight is involved.
    """
    n = q * int(np.prod(shape))
    b = 1.0 / q if base is None else base
    r = 2.0 * uniform01(n, seed) - 1.0
    return (b * (1.0 + spread * r)).reshape((q,) + tuple(shape))


def random_signed(q: int, shape, seed: int, amplitude: float) -> np.ndarray:
    """Uniform values in [-amplitude, amplitude), shape (q, *shape)."""
    n = q * int(np.prod(shape))
    return (amplitude * (2.0 * uniform01(n, seed) - 1.0)).reshape((q,) + tuple(shape))


def smooth_field(shape, seed: int, amplitude: float, modes: int = 3) -> np.ndarray:
    """A smooth random field: a sum of a few low sine modes with seeded amplitudes.

    Used as a non-trivial but well-resolved initial velocity / temperature
    field (values vanish on the boundary of the unit box).
    """
    d = len(shape)
    coeff = 2.0 * uniform01(modes ** d, seed) - 1.0
    axes = [(np.arange(n) + 0.5) / n for n in shape]  # axis order as in `shape`
    grids = np.meshgrid(*axes, indexing="ij")
    out = np.zeros(shape)
    for flat in range(modes ** d):
        idx = np.unravel_index(flat, (modes,) * d)
        term = np.ones(shape)
        for g, k in zip(grids, idx):
            term = term * np.sin(np.pi * (k + 1) * g)
        out += coeff[flat] * term
    return amplitude * out / max(1.0, np.abs(out).max() / 1.0)


def ra_sweep(count: int, seed: int = 0, log10_lo: float = 6.0, log10_hi: float = 8.0,
             sizes=(128, 256, 384, 512)):
    """Ra log-uniform in [10^lo, 10^hi] and mesh sizes drawn uniformly from `sizes` (PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ra = 10.0 ** rng.uniform(log10_lo, log10_hi, size=count)
    n = rng.choice(np.asarray(sizes), size=count)
    return ra, n


def gaussian_arrays(shapes, seed: int, scales=None) -> dict:
    """Independent N(0, scale^2) float64 arrays, one per (name, shape) pair, in order.

    Used for the weights and inputs of the warm-start network's parity tests;
    scales maps a name to its standard deviation (default 1)."""
    rng = np.random.default_rng(seed)
    scales = scales or {}
    return {name: rng.standard_normal(shape) * scales.get(name, 1.0) for name, shape in shapes}
