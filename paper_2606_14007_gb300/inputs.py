"""Seeded synthetic inputs for plots: plot keys and plot-request mixes.

This module holds no arithmetic of the plotting method.  It is shared by the
CUDA path's callers (tests, benchmark, server driver) and by the oracle's
callers; neither the oracle nor the library imports it.

The paper does not say where plot keys come from (Sec. III-B only says the
key is 256 bits), so keys are drawn from a published generator: four
successive SplitMix64 outputs (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) from ``seed``, each stored
little-endian.
"""
from __future__ import annotations

import numpy as np

_M64 = (1 << 64) - 1


def splitmix64(seed: int, count: int) -> list[int]:
    """`count` successive SplitMix64 outputs starting from state `seed`."""
    state = seed & _M64
    out = []
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & _M64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        out.append(z ^ (z >> 31))
    return out


def plot_key(seed: int) -> bytes:
    """32-byte plot key of a seed: 4 SplitMix64 words, little-endian."""
    return b"".join(w.to_bytes(8, "little") for w in splitmix64(seed, 4))


def batch_mix(count: int = 64, k_lo: int = 20, k_hi: int = 26, rng_seed: int = 2026,
              key_seed0: int = 1000) -> list[tuple[int, bytes]]:
    """Mixed-K batch: K uniform in [k_lo, k_hi] from numpy's default_rng(rng_seed),
    key i from seed key_seed0 + i."""
    rng = np.random.default_rng(rng_seed)
    ks = rng.integers(k_lo, k_hi + 1, size=count)
    return [(int(k), plot_key(key_seed0 + i)) for i, k in enumerate(ks)]


def poisson_arrivals(rate_hz: float, duration_s: float, k_lo: int = 22, k_hi: int = 29,
                     rng_seed: int = 7) -> list[tuple[float, int, bytes]]:
    """Plot requests with exponential inter-arrival times: (t, K, key), key of
    request r from seed r."""
    rng = np.random.default_rng(rng_seed)
    t = 0.0
    out = []
    r = 0
    while True:
        t += float(rng.exponential(1.0 / rate_hz))
        if t >= duration_s:
            break
        out.append((t, int(rng.integers(k_lo, k_hi + 1)), plot_key(r)))
        r += 1
    return out
