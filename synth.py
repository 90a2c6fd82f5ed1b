"""Seeded synthetic point clouds for the simplex-domain workloads.

This module only draws random numbers. It holds none of the arithmetic of
the method (no maps, no distances, no energies), so both the CPU oracle
(``oracle/``) and the CUDA path (``paper_1610_07394_gb300``) can be fed the
same inputs without sharing any of the computation.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014). It is counter-based: draw ``i`` of stream
``seed`` is ``mix(seed + (i + 1) * GAMMA)``, so a whole array is produced in
one vectorised step and any element can be recomputed alone.

Recipes (the workloads the paper's problem classes describe, with sizes
chosen by the benchmark configurations):

* ``uniform_cube(n, d, side, seed)``: FP32 coordinates ``side * u`` with ``u``
  the top 24 bits of a draw times 2^-24 (exact in FP32; one rounding for the
  scale).
* ``normal(n, d, seed)``: Box-Muller in FP64 from two 53-bit uniforms, rounded
  to FP32.
* ``perturbed(x, sigma, seed)``: ``x + sigma * normal(seed)`` in FP64, rounded
  to FP32 (the reference configuration of a stress loss).
* ``sample_indices(count, n, seed)``: distinct indices by a SplitMix64-keyed
  permutation (used to pick sampled atoms and pairs for checks at full size).
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws ``offset .. offset+count-1`` of the SplitMix64 stream ``seed``."""
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + ctr * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform24(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform FP64 values in [0, 1) with 24 significant bits (exact in FP32)."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)


def uniform53(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform FP64 values in [0, 1) with 53 significant bits."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_cube(n: int, d: int, side: float, seed: int) -> np.ndarray:
    """``n`` points uniform in the cube [0, side)^d, FP32, row-major (n, d)."""
    u = uniform24(seed, n * d)
    return (u * float(side)).astype(np.float32).reshape(n, d)


def normal(n: int, d: int, seed: int) -> np.ndarray:
    """``n`` points with i.i.d. N(0, 1) coordinates, FP32, row-major (n, d)."""
    m = n * d
    half = (m + 1) // 2
    u = uniform53(seed, 2 * half)
    u1 = 1.0 - u[0::2]            # (0, 1]: log is finite
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * half, dtype=np.float64)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:m].astype(np.float32).reshape(n, d)


def perturbed(x: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """``x + sigma * N(0, 1)`` (FP64 sum, rounded to FP32)."""
    n, d = x.shape
    g = normal(n, d, seed).astype(np.float64)
    return (x.astype(np.float64) + float(sigma) * g).astype(np.float32)


def sample_indices(count: int, n: int, seed: int) -> np.ndarray:
    """``count`` distinct indices in [0, n): the first ``count`` of a random
    permutation whose sort keys are SplitMix64 draws of stream ``seed``."""
    keys = splitmix64(seed, n)
    perm = np.argsort(keys, kind="stable")
    return perm[: min(count, n)].astype(np.int64)


def sample_pairs(count: int, n: int, seed: int) -> np.ndarray:
    """``count`` index pairs (i, j) with 0 <= j <= i < n, as an int64 (count, 2)
    array, drawn from SplitMix64 stream ``seed`` (repeats are possible)."""
    z = splitmix64(seed, 2 * count)
    a = (z[0::2] % np.uint64(n)).astype(np.int64)
    b = (z[1::2] % np.uint64(n)).astype(np.int64)
    return np.stack([np.maximum(a, b), np.minimum(a, b)], axis=1)


# The benchmark workloads: name -> (kind, n, d, generator arguments).
WORKLOADS = {
    "edm_n1024_d3": dict(n=1024, d=3, gen="uniform", side=1.0, seed=0),
    "atm_n1024": dict(n=1024, d=3, gen="uniform", side=10.0, seed=1),
    "edm_n32768_d256": dict(n=32768, d=256, gen="normal", seed=2),
    "atm_n4096": dict(n=4096, d=3, gen="uniform", side=20.0, seed=3),
    "stress_n65536_d64": dict(n=65536, d=64, gen="normal", seed=4, y_seed=5, sigma=0.1),
    "atm_n16384": dict(n=16384, d=3, gen="uniform", side=20.0, seed=6),
}


def make_points(name: str) -> np.ndarray:
    """The point cloud of a named workload (see ``WORKLOADS``)."""
    w = WORKLOADS[name]
    if w["gen"] == "uniform":
        return uniform_cube(w["n"], w["d"], w["side"], w["seed"])
    return normal(w["n"], w["d"], w["seed"])
