"""Asynchrony-tolerant flux coefficients (oracle; test infrastructure).

Section 5, Eq. at-flux-gen: the AT flux for the update n -> n+1 at a PE boundary node is a
combination sum_{l=L1}^{L2} c^l f^{n-l} of fluxes from delayed levels. Eq. at-flux-constraints
fixes the coefficients: sum_l c^l (-l dt)^zeta / zeta! = 1 for zeta = 0 and 0 for
0 < zeta < order, with L1 = k (the delay) and L2 = k + order - 1. The system is solved here
in exact rational arithmetic (dt cancels row by row), by plain Gaussian elimination.
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial


def constraint_system(k: int, order: int):
    """Rows zeta = 0..order-1 of Eq. at-flux-constraints over levels l = k..k+order-1,
    with dt = 1 (each row scales by dt^zeta, which leaves the solution unchanged)."""
    levels = [k + m for m in range(order)]
    A = [[Fraction((-l) ** zeta, factorial(zeta)) for l in levels] for zeta in range(order)]
    b = [Fraction(1 if zeta == 0 else 0) for zeta in range(order)]
    return A, b


def solve_exact(A, b):
    n = len(b)
    M = [row[:] + [b[i]] for i, row in enumerate(A)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return [M[i][n] / M[i][i] for i in range(n)]


def at_coefficients(k: int, order: int):
    """Exact coefficients [c^k, c^{k+1}, ..., c^{k+order-1}] for delay k."""
    if order < 1 or k < 0:
        raise ValueError("order >= 1 and k >= 0")
    A, b = constraint_system(k, order)
    return solve_exact(A, b)


def at_coefficients_f64(k: int, order: int):
    return [float(c) for c in at_coefficients(k, order)]
