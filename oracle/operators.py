"""Reference-element operators of nodal DG on [-1, 1] (oracle; test infrastructure).

Section 2: Lagrange basis functions phi_j on the reference element [-1, 1] whose j-th DoF
is the value at the j-th node; the paper does not name the node set, the nodal
Legendre-Gauss-Lobatto (LGL) set is used (so phi_j(-1) = delta_{j0}, phi_j(1) = delta_{jp}).

Eq. matrices-reference:
    M_ij  = int phi_j phi_i dxi,       S_ij  = int phi_j dphi_i/dxi dxi,
    K-_ij = B+ phi_j(1) phi_i(-1),     K+_ij = -B- phi_j(-1) phi_i(1),
    K_l_ij = B- phi_j(-1) phi_i(-1),   K_r_ij = -B+ phi_j(1) phi_i(1).
Integrals are exact (Gauss-Legendre quadrature with p+2 points, exact to degree 2p+3).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from numpy.polynomial import legendre as npleg
from numpy.polynomial import Polynomial


def lgl_nodes_weights(p: int):
    """LGL nodes (endpoints and the roots of P_p') and weights 2 / (p (p+1) P_p(x)^2)."""
    if p < 1:
        raise ValueError("p >= 1")
    cp = np.zeros(p + 1)
    cp[p] = 1.0
    dcp = npleg.legder(cp)
    interior = np.zeros(0)
    if p > 1:
        r = npleg.legroots(dcp)
        assert np.max(np.abs(np.imag(r))) < 1e-12
        interior = np.sort(np.real(r))
        d2cp = npleg.legder(dcp)
        for _ in range(3):      # Newton polish of the roots of P_p'
            interior = interior - npleg.legval(interior, dcp) / npleg.legval(interior, d2cp)
        interior = 0.5 * (interior - interior[::-1])   # the LGL set is symmetric about 0
    x = np.concatenate([[-1.0], interior, [1.0]])
    w = 2.0 / (p * (p + 1) * npleg.legval(x, cp) ** 2)
    return x, w


def lagrange_basis(nodes):
    """Lagrange polynomials l_j with l_j(nodes[i]) = delta_ij, as numpy Polynomials."""
    out = []
    for j, xj in enumerate(nodes):
        others = np.delete(nodes, j)
        out.append(Polynomial.fromroots(others) / np.prod(xj - others))
    return out


@dataclass
class RefOps:
    p: int
    nodes: np.ndarray
    weights: np.ndarray
    D: np.ndarray      # D_ij = l_j'(xi_i)
    M: np.ndarray
    Minv: np.ndarray
    S: np.ndarray      # paper's stiffness: S_ij = int l_j l_i'
    e0: np.ndarray     # phi_i(-1)
    ep: np.ndarray     # phi_i(+1)

    @property
    def Np(self) -> int:
        return self.p + 1

    def flux_matrices(self, Bp: float, Bm: float):
        """(K-, K_l, K_r, K+) of Eq. matrices-reference for flux weights B+, B-."""
        e0, ep = self.e0, self.ep
        Km = Bp * np.outer(e0, ep)      # [K-]_ij = B+ phi_j(1) phi_i(-1)
        Kp = -Bm * np.outer(ep, e0)     # [K+]_ij = -B- phi_j(-1) phi_i(1)
        Kl = Bm * np.outer(e0, e0)      # [K_l]_ij = B- phi_j(-1) phi_i(-1)
        Kr = -Bp * np.outer(ep, ep)     # [K_r]_ij = -B+ phi_j(1) phi_i(1)
        return Km, Kl, Kr, Kp


def ref_ops(p: int) -> RefOps:
    x, w = lgl_nodes_weights(p)
    ell = lagrange_basis(x)
    dell = [l.deriv() for l in ell]
    Np = p + 1
    D = np.array([[dell[j](x[i]) for j in range(Np)] for i in range(Np)])
    gx, gw = npleg.leggauss(p + 2)
    L = np.array([l(gx) for l in ell])        # (Np, nq)
    dL = np.array([d(gx) for d in dell])
    M = (L * gw) @ L.T                        # M_ij = int l_i l_j
    S = (dL * gw) @ L.T                       # S_ij = int l_i' l_j
    e0 = np.array([l(-1.0) for l in ell])
    ep = np.array([l(1.0) for l in ell])
    return RefOps(p=p, nodes=x, weights=w, D=D, M=M, Minv=np.linalg.inv(M), S=S, e0=e0, ep=ep)
