"""Seeded synthetic inputs for the spectral Poisson workloads.

This module only draws random numbers and arranges them; it holds none of the
solver's arithmetic, so that both the GPU library's tests/benchmark and the CPU
oracle can take their inputs from here without sharing method code.

Random semantics (the paper fixes none): numpy's ``default_rng(seed)``,
``standard_normal`` in FP64, C order.
"""
from __future__ import annotations

import numpy as np


def gaussian(seed: int, shape) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(shape)


def decay_weights(n: int, power: int) -> np.ndarray:
    """w_j = 1/(1+j)^power, j = 0..n-1."""
    return 1.0 / (1.0 + np.arange(n, dtype=np.float64)) ** power


def square_rhs(n: int, seed: int, power: int = 2) -> np.ndarray:
    """F_jk = g_jk / ((1+j)^power (1+k)^power), g iid N(0,1) from ``seed``."""
    g = gaussian(seed, (n, n))
    w = decay_weights(n, power)
    return g * w[:, None] * w[None, :]


def cube_rhs(n: int, seed: int, power: int = 2) -> np.ndarray:
    """F_ijk = g_ijk / ((1+i)^p (1+j)^p (1+k)^p)."""
    g = gaussian(seed, (n, n, n))
    w = decay_weights(n, power)
    return g * w[:, None, None] * w[None, :, None] * w[None, None, :]


def poly_values(seed: int, deg: int = 10) -> np.ndarray:
    """N(0,1) coefficients of the (deg+1)(deg+2)/2 monomials x^a y^b, a+b <= deg,
    in the order: total degree t = 0..deg, then a descending."""
    return gaussian(seed, ((deg + 1) * (deg + 2) // 2,))


def batch_problems(seed: int = 5, count: int = 512, n_lo: int = 32, n_hi: int = 2048, nrhs: int = 4,
                   power: int = 2, draw_rhs: bool = True):
    """Batched workload: ``count`` squares with n drawn log-uniformly in
    [n_lo, n_hi], then (same generator) each problem's ``nrhs`` right-hand sides
    F_jk = g_jk / ((1+j)^p (1+k)^p).  Returns (ns, list of (nrhs, n, n) arrays)."""
    rng = np.random.default_rng(seed)
    ns = np.rint(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), size=count))).astype(np.int64)
    ns = np.clip(ns, n_lo, n_hi)
    if not draw_rhs:
        return ns, None
    rhs = []
    for n in ns:
        w = decay_weights(int(n), power)
        g = rng.standard_normal((nrhs, int(n), int(n)))
        rhs.append(g * w[None, :, None] * w[None, None, :])
    return ns, rhs


def unit_directions(seed: int, count: int, shape) -> np.ndarray:
    """``count`` random directions of unit Frobenius norm."""
    v = gaussian(seed, (count, *shape))
    norms = np.sqrt((v.reshape(count, -1) ** 2).sum(axis=1))
    return v / norms.reshape((count,) + (1,) * len(shape))
