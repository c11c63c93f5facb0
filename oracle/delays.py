"""Delay emulation (oracle; test infrastructure).

Two sources of delays. The communication-avoiding cycle of Section 6.3 (``caa_delay``):
every period of `sync_steps` + L steps starts with `sync_steps` steps that communicate and
synchronise (delay 0), followed by L steps without communication, whose faces use the levels
0, 1, ..., L-1 steps old. The random emulation of Section 6.1:
at each time step a uniform random number in [0, 1] is drawn at each PE
boundary and matched against L bins of sizes p_0 .. p_{L-1}; bin k gives the delay k.
The bins are [c_k, c_{k+1}) with c_k = p_0 + ... + p_{k-1} summed left to right in FP64.

The uniform numbers come from SplitMix64 (Steele, Lea and Flood, 2014; the generator in
Vigna's public reference implementation): the i-th output (i = 0, 1, ...) for a 64-bit
seed s is mix(s + (i+1) * 0x9E3779B97F4A7C15 mod 2^64). The draw for step n at PE face j
of a run with P PEs is output i = n * P + j, mapped to [0, 1) as (z >> 11) * 2^-53.
"""
from __future__ import annotations

import numpy as np

_MASK = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def splitmix64_output(seed: int, i: int) -> int:
    """The i-th SplitMix64 output for `seed` (plain Python integers, mod 2^64)."""
    z = (seed + (i + 1) * GAMMA) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def uniform01(seed: int, i: int) -> float:
    return float(splitmix64_output(seed, i) >> 11) * (2.0 ** -53)


def bin_edges(probs):
    """Upper bin edges c_1 .. c_L (c_{k+1} = p_0 + ... + p_k, summed in order in FP64)."""
    edges = []
    c = 0.0
    for pk in probs:
        c = c + float(pk)
        edges.append(c)
    return edges


def delay_from_uniform(u: float, edges) -> int:
    """Smallest k with u < c_{k+1}; draws beyond the last edge (rounding) map to L-1."""
    for k, c in enumerate(edges):
        if u < c:
            return k
    return len(edges) - 1


def delay_table(seed: int, P: int, steps: int, L: int, probs=None, first_step: int = 0):
    """uint8 table D[n - first_step][j] for steps first_step .. first_step+steps-1."""
    if probs is None:
        probs = [1.0 / L] * L
    if len(probs) != L:
        raise ValueError("len(probs) must equal L")
    edges = bin_edges(probs)
    out = np.zeros((steps, P), dtype=np.uint8)
    for r in range(steps):
        n = first_step + r
        for j in range(P):
            out[r, j] = delay_from_uniform(uniform01(seed, n * P + j), edges)
    return out


def caa_delay(n: int, sync_steps: int, L: int) -> int:
    """Delay of step n under the communication-avoiding cycle (Section 6.3): position
    m = n mod (sync_steps + L) in the period; 0 for m < sync_steps, else m - sync_steps."""
    m = n % (sync_steps + L)
    return 0 if m < sync_steps else m - sync_steps


def caa_communicates(n: int, sync_steps: int, L: int) -> bool:
    """Whether step n of the cycle exchanges PE-face data (its synchronised steps only)."""
    return n % (sync_steps + L) < sync_steps


def caa_table(P: int, steps: int, sync_steps: int, L: int, first_step: int = 0):
    """uint8 table D[n - first_step][j] of the cycle (the same delay at every PE face)."""
    out = np.zeros((steps, P), dtype=np.uint8)
    for r in range(steps):
        out[r, :] = caa_delay(first_step + r, sync_steps, L)
    return out
