"""Pins of the Fourier-mode analysis (Section 4.2) against the paper's printed results."""
import numpy as np
import pytest

from oracle import fourier


def test_dg1_rk2_upwind_stability_limit():
    # Section 4.2.1: DG(1)-RK2 with the upwind flux is stable only for sigma <= 0.333.
    assert fourier.max_growth(fourier.G_sync, 1, 0.333, rk="rk2") <= 1.0 + 1e-12
    assert fourier.max_growth(fourier.G_sync, 1, 0.25, rk="rk2") <= 1.0 + 1e-12
    assert fourier.max_growth(fourier.G_sync, 1, 0.34, rk="rk2") > 1.01


def _max_omega_i(builder, p, sigma, n=721):
    worst = -np.inf
    for th in np.linspace(-np.pi, np.pi, n):
        om = fourier.omega(builder(p, th, sigma), sigma, p + 1)
        worst = max(worst, float(np.max(om.imag)))
    return worst


def test_adg1_rk2_L2_stability_as_printed():
    # Section 4.2.2, Fig. 4: with the matrices of Eq. async-dg2-rk2-l2 the scheme is
    # unstable at sigma = 0.333 and stable (to plot resolution) at 0.1 and 0.05; the
    # largest Im(Omega) falls with sigma. The printed matrices give 7e-4 at 0.1 and 5e-5
    # at 0.05 (recorded as a reading), against 4.9e-2 at 0.333.
    b = fourier.G_paper_adg1_rk2_L2
    w333 = _max_omega_i(b, 1, 0.333)
    w10 = _max_omega_i(b, 1, 0.1)
    w05 = _max_omega_i(b, 1, 0.05)
    assert w333 > 1e-2
    assert w10 < 1e-3 and w05 < 1e-4
    assert w333 > 50 * w10 > 50 * w05 / 14


@pytest.mark.parametrize("rk", ["rk2", "ssprk3", "rk4", "lsrk3", "lsrk4"])
def test_physical_mode_dispersion(rk):
    # The physical mode satisfies Omega_r = K (K = theta/(Np)) for small wavenumbers.
    p, sigma = 2, 0.1
    for th in (0.05, 0.1, 0.2):
        om = fourier.omega(fourier.G_sync(p, th, sigma, rk), sigma, p + 1)
        Kw = th / (p + 1)
        best = om[np.argmin(np.abs(om.real - Kw))]
        assert abs(best.real - Kw) < 1e-4 and abs(best.imag) < 1e-4


def test_companion_structure():
    Gn = np.eye(2) * 2
    Gk = np.eye(2) * 3
    G = fourier.companion(Gn, Gk, 2)
    assert G.shape == (6, 6)
    assert np.array_equal(G[2:4, 0:2], np.eye(2)) and np.array_equal(G[4:6, 2:4], np.eye(2))
    assert np.array_equal(G[0:2, 4:6], Gk)
