"""Seeded synthetic double-double inputs (test and benchmark data only).

Both the CUDA path's tests and the oracle's tests draw their inputs here.
This module holds no arithmetic of the method: it only draws random FP64x2
matrices with the shapes and value distributions of the workloads.

Every generator uses numpy's PCG64 ``default_rng(seed)`` and draws, in order,
A_hi, A_lo, B_hi, B_lo (then any extra matrices).  A double-double value is
the exact real hi + lo.  The ``lo`` part is ``hi * 2**-53 * U[-1, 1]``, so
|lo| <= ulp(hi)/2: the uniform generator of the paper's accuracy section
(random FP64, then extra random low-order bits).
"""
from __future__ import annotations

import numpy as np

TWO_M53 = 2.0 ** -53


def _lo_from_hi(rng, hi):
    return hi * TWO_M53 * rng.uniform(-1.0, 1.0, size=hi.shape)


def uniform_hi(rng, shape):
    """hi ~ U[-1, 1]."""
    return rng.uniform(-1.0, 1.0, size=shape)


def wide_hi(rng, shape, spread=40.0):
    """hi = s * 2**u, u ~ U[-spread/2, spread/2], s = +-1 with equal odds
    (log-uniform magnitudes; spread = 40 gives 2^-20 .. 2^20)."""
    u = rng.uniform(-spread / 2.0, spread / 2.0, size=shape)
    s = np.where(rng.integers(0, 2, size=shape) == 0, -1.0, 1.0)
    return s * np.exp2(u)


def dd_matrix(rng, shape, kind="uniform", spread=40.0):
    """One FP64x2 matrix (hi, lo) drawn from the named distribution."""
    if kind == "uniform":
        hi = uniform_hi(rng, shape)
    elif kind == "wide":
        hi = wide_hi(rng, shape, spread)
    else:
        raise ValueError(f"unknown distribution {kind!r}")
    return hi, _lo_from_hi(rng, hi)


def gemm_inputs(m, n, k, kind="uniform", seed=0, spread=40.0):
    """A (m x k) and B (k x n) as row-major float64 (hi, lo) pairs.

    kind="uniform": hi ~ U[-1, 1] (the 256^3 small case).
    kind="wide":    hi log-uniform over 2^-spread/2 .. 2^spread/2 with random
                    signs (the 4096^3 and 8192x1024x4096 cases, spread 40)."""
    rng = np.random.default_rng(seed)
    a_hi = (uniform_hi(rng, (m, k)) if kind == "uniform" else wide_hi(rng, (m, k), spread))
    a_lo = _lo_from_hi(rng, a_hi)
    b_hi = (uniform_hi(rng, (k, n)) if kind == "uniform" else wide_hi(rng, (k, n), spread))
    b_lo = _lo_from_hi(rng, b_hi)
    return a_hi, a_lo, b_hi, b_lo


def integer_inputs(m, n, k, bits=10, seed=0):
    """Small-integer matrices (|entry| < 2**bits), lo = 0."""
    rng = np.random.default_rng(seed)
    lim = 2 ** bits
    a = rng.integers(-lim + 1, lim, size=(m, k)).astype(np.float64)
    b = rng.integers(-lim + 1, lim, size=(k, n)).astype(np.float64)
    return a, np.zeros_like(a), b, np.zeros_like(b)


def batched_shapes(count=512, lo=64, hi=1024, seed=0):
    """(m, n, k) triples, each drawn log-uniform from [lo, hi] independently."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(np.log(lo), np.log(hi + 1), size=(count, 3))
    return np.floor(np.exp(u)).astype(np.int64).clip(lo, hi)


def device_uniform_dd(shape, seed, device="cuda"):
    """A uniform FP64x2 matrix drawn on a CUDA device, for operands too large
    to draw on the host: hi ~ U[-1, 1], lo = hi * 2**-53 * U[-1, 1], from
    torch's seeded generator on that device (its own stream of values, not
    numpy's: tests gather the entries they check back to the host)."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    hi = torch.empty(shape, dtype=torch.float64, device=device).uniform_(-1.0, 1.0, generator=g)
    lo = torch.empty_like(hi).uniform_(-1.0, 1.0, generator=g)
    lo.mul_(hi).mul_(TWO_M53)
    return hi, lo
