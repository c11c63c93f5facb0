"""Pins of the oracle's reference-element operators (Section 2, Eq. matrices-reference)."""
import math
import os

import numpy as np
import pytest

from oracle.operators import ref_ops, lgl_nodes_weights

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _lgl_table():
    rows = {}
    for line in open(os.path.join(GOLD, "lgl_nodes.txt")):
        if line.startswith("#") or not line.strip():
            continue
        p, xe, we = line.split()
        env = {"sqrt": math.sqrt}
        rows.setdefault(int(p), []).append((eval(xe, env), eval(we, env)))
    return rows


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lgl_closed_form(p):
    x, w = lgl_nodes_weights(p)
    ref = _lgl_table()[p]
    assert np.allclose(x, [r[0] for r in ref], atol=1e-15, rtol=0)
    assert np.allclose(w, [r[1] for r in ref], atol=1e-15, rtol=0)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_derivative_exact_on_polynomials(p):
    ops = ref_ops(p)
    x = ops.nodes
    assert np.max(np.abs(ops.D @ np.ones_like(x))) < 1e-13
    for m in range(1, p + 1):
        assert np.allclose(ops.D @ x ** m, m * x ** (m - 1), atol=1e-13, rtol=0)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_mass_and_stiffness_identities(p):
    ops = ref_ops(p)
    # M 1 = w: the LGL rule integrates each basis function exactly (degree p <= 2p-1).
    assert np.allclose(ops.M @ np.ones(p + 1), ops.weights, atol=1e-15)
    assert np.allclose(ops.M, ops.M.T, atol=0)
    assert np.all(np.linalg.eigvalsh(ops.M) > 0)
    # Summation by parts: S + S^T = e_p e_p^T - e_0 e_0^T (integral of (l_i l_j)').
    SBP = np.outer(ops.ep, ops.ep) - np.outer(ops.e0, ops.e0)
    assert np.allclose(ops.S + ops.S.T, SBP, atol=1e-14)
    # Paper's S relates to the nodal derivative by S = D^T M.
    assert np.allclose(ops.S, ops.D.T @ ops.M, atol=1e-13)
    # Lift columns integrate to one: w^T M^{-1} e_0 = 1^T e_0 = 1.
    assert abs(ops.weights @ ops.Minv @ ops.e0 - 1.0) < 1e-13
    assert abs(ops.weights @ ops.Minv @ ops.ep - 1.0) < 1e-13


def test_p1_mass_matrix_textbook():
    ops = ref_ops(1)
    assert np.allclose(ops.M, [[2 / 3, 1 / 3], [1 / 3, 2 / 3]], atol=1e-15)
    assert np.allclose(ops.D, [[-0.5, 0.5], [-0.5, 0.5]], atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lift_diagonal_is_trace_constant(p):
    # (M^{-1})_{pp} = (p+1)^2 / 2 for the LGL nodal basis (the trace inverse constant).
    ops = ref_ops(p)
    assert abs(ops.Minv[p, p] - (p + 1) ** 2 / 2) < 1e-11


def test_flux_matrices_upwind():
    ops = ref_ops(2)
    Km, Kl, Kr, Kp = ops.flux_matrices(1.0, 0.0)
    assert Km[0, 2] == 1.0 and np.count_nonzero(Km) == 1
    assert Kr[2, 2] == -1.0 and np.count_nonzero(Kr) == 1
    assert np.count_nonzero(Kl) == 0 and np.count_nonzero(Kp) == 0
