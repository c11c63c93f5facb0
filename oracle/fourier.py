"""Fourier-mode analysis of the synchronous and asynchronous DG-RK schemes (oracle).

Section 4.2: with u^e = mu exp(i kappa x_e) and theta = kappa dx, one RK stage increment
k = dt L(u) has the symbol
    Lhat(theta) = 2 sigma M^{-1} ( e^{-i theta} K- + K_l + S + K_r + e^{i theta} K+ ),
(Eq. dg2-rk2-updates), and one step of a synchronous scheme is u^{n+1} = G^s u^n.
Eigenvalues lambda of G give Omega = i ln(lambda) / (sigma (Np+1)); Im(Omega) <= 0, i.e.
|lambda| <= 1, for every wavenumber is the stability condition.

``G_paper_adg1_rk2_L2`` builds the asynchronous ADG(1)-RK2-L2 matrices exactly as printed in
Eq. async-dg2-rk2-l2 (left face one level late) and the block-companion amplification
matrix of Eq. one-step-async-l2; ``companion`` the general delay-k block companion.

``delayed_recurrence`` advances a single Fourier mode through the stage-consistent
delayed scheme with every face a PE face (P = K) and a constant delay: the stage-s
input of step n uses, at both faces, the stage-s inputs of levels n-k-i combined with the
AT coefficients. It is an independent restatement (in Fourier space, on amplitudes) of
what ``oracle.dg.Solver`` does element by element in physical space.
"""
from __future__ import annotations

import numpy as np

from .atflux import at_coefficients_f64
from .dg import TABLEAUX
from .operators import ref_ops


def symbols(p: int, theta: float, sigma: float, Bp: float = 1.0, Bm: float = 0.0):
    """(C S, C (e^{-i theta} K- + K_l), C (K_r + e^{i theta} K+)) with C = 2 sigma M^{-1}."""
    ops = ref_ops(p)
    Km, Kl, Kr, Kp = ops.flux_matrices(Bp, Bm)
    C = 2.0 * sigma * ops.Minv
    z = np.exp(1j * theta)
    return C @ ops.S, C @ (Km / z + Kl), C @ (Kr + z * Kp)


def G_sync(p: int, theta: float, sigma: float, rk: str = "rk2", Bp=1.0, Bm=0.0):
    """Amplification matrix of the synchronous DG(p)-RK scheme: stage increments
    K_s = Lhat (I + sum_j a_sj K_j), G = I + sum_s b_s K_s."""
    Lv, Ll, Lr = symbols(p, theta, sigma, Bp, Bm)
    Lhat = Lv + Ll + Lr
    a, b = TABLEAUX[rk]
    I = np.eye(p + 1, dtype=complex)
    Ks = []
    for s in range(len(b)):
        Y = I.copy()
        for j in range(s):
            Y = Y + a[s][j] * Ks[j]
        Ks.append(Lhat @ Y)
    G = I.copy()
    for s in range(len(b)):
        G = G + b[s] * Ks[s]
    return G


def G_paper_adg1_rk2_L2(p: int, theta: float, sigma: float, Bp=1.0, Bm=0.0):
    """Block amplification matrix [[G^{as,n}, G^{as,n-1}], [I, 0]] of the ADG-RK2-L2 scheme
    with the matrices of Eq. async-dg2-rk2-l2 taken as printed."""
    ops = ref_ops(p)
    Km, Kl, Kr, Kp = ops.flux_matrices(Bp, Bm)
    S = ops.S
    C = 2.0 * sigma * ops.Minv
    z = np.exp(1j * theta)
    I = np.eye(p + 1, dtype=complex)
    Kall = Kl + S + Kr
    K10_e = C @ ((S + Kr) + z * Kp)
    K11_e = C @ (Km / z + Kl)
    K11_em1 = C @ (Km / z ** 2 + Kall / z + Kp)
    K10_ep1 = C @ (Km + z * Kall + z ** 2 * Kp)
    K20_e = C @ (Kl @ K10_e + (S + Kr) @ (I + K10_e) + Kp @ (z * I + K10_ep1))
    K21_e = C @ (Km @ (I / z + K11_em1) + Kl @ (I + K11_e) + (S + Kr) @ K11_e)
    Gn = I + 0.5 * (K10_e + K20_e)
    Gn1 = 0.5 * (K11_e + K21_e)
    return companion(Gn, Gn1, 1)


def companion(Gn, Gnk, k: int):
    """(k+1)(Np+1) block companion for u^{n+1} = G^{as,n} u^n + G^{as,n-k} u^{n-k}."""
    Np = Gn.shape[0]
    N = (k + 1) * Np
    G = np.zeros((N, N), dtype=complex)
    G[:Np, :Np] = Gn
    G[:Np, k * Np:] = Gnk
    for r in range(1, k + 1):
        G[r * Np:(r + 1) * Np, (r - 1) * Np:r * Np] = np.eye(Np)
    return G


def omega(G, sigma: float, Np: int):
    """Omega = i ln(lambda) / (sigma Np) for each eigenvalue (Section 4.2.1); Np = p+1."""
    lam = np.linalg.eigvals(G)
    return 1j * np.log(lam.astype(complex)) / (sigma * Np)


def max_growth(builder, p: int, sigma: float, n_theta: int = 721, **kw) -> float:
    """max over theta in [-pi, pi] of the spectral radius of builder(p, theta, sigma)."""
    worst = 0.0
    for th in np.linspace(-np.pi, np.pi, n_theta):
        worst = max(worst, float(np.max(np.abs(np.linalg.eigvals(builder(p, th, sigma, **kw))))))
    return worst


def delayed_recurrence(p: int, theta: float, sigma: float, rk: str, k: int, q: int,
                       mu0: np.ndarray, nsteps: int, Bp=1.0, Bm=0.0):
    """Amplitude u^N of a single mode under the stage-consistent delayed scheme with all
    faces delayed by the constant k (clamped to k <= n), AT order q (q = 1: standard)."""
    Lv, Ll, Lr = symbols(p, theta, sigma, Bp, Bm)
    Lf = Ll + Lr
    a, b = TABLEAUX[rk]
    u = np.asarray(mu0, dtype=complex)
    hist = {}
    for n in range(nsteps):
        Ks = []
        for s in range(len(b)):
            Y = u.copy()
            for j in range(s):
                if a[s][j] != 0.0:
                    Y = Y + a[s][j] * Ks[j]
            hist[(n, s)] = Y
            kk = min(k, n)
            qe = min(q, n - kk + 1)
            c = at_coefficients_f64(kk, qe)
            face = sum(c[i] * hist[(n - kk - i, s)] for i in range(qe))
            Ks.append(Lv @ Y + Lf @ face)
        for s in range(len(b)):
            u = u + b[s] * Ks[s]
    return u
