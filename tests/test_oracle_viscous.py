"""Pins of the oracle's viscous Burgers operator (Eq. burgers by the local DG method of
Section 6, alternating fluxes for the viscous term): exactness of the LDG derivative for
polynomial data, convergence to the Cole-Hopf exact solution, conservation, and the zero-delay
reduction of the asynchronous scheme."""
import math

import numpy as np
import pytest
import torch

from oracle import delays, dg

TWO_PI = 2 * math.pi


def _cole_hopf(x, t, nu, a):
    """Exact periodic solution u = -2 nu phi_x / phi of u_t + u u_x = nu u_xx with
    phi = a_0 + sum_k a_k exp(-nu k^2 t) cos(k x) > 0 (the heat equation's solution)."""
    phi = np.full_like(x, a[0])
    dphi = np.zeros_like(x)
    for k in range(1, len(a)):
        g = a[k] * math.exp(-nu * k * k * t)
        phi = phi + g * np.cos(k * x)
        dphi = dphi - g * k * np.sin(k * x)
    return -2.0 * nu * dphi / phi


@pytest.mark.parametrize("p", [2, 3])
def test_ldg_derivative_is_exact_for_polynomials(p):
    # With uhat = u^- and u continuous, q = u_x exactly for u of degree <= p (integration by
    # parts); the periodic wrap face breaks continuity, so only elements away from it count.
    K = 12
    x = dg.node_coordinates(K, p, 0.0, TWO_PI)
    u = torch.tensor(0.3 * x ** 2 - 1.1 * x + 0.7)
    s = dg.Solver(dg.Problem(pde="burgers", K=K, p=p, P=1, dt=1e-3, nu=0.1), u)
    uL, _ = s.traces(u)
    q = s.ldg_q(u, uL, 0, 0).numpy()
    assert np.max(np.abs(q[1:-1] - (0.6 * x[1:-1] - 1.1))) < 1e-12


@pytest.mark.parametrize("mode,rk,fac,t_end", [("sync", "lsrk4", 0.1, 0.4), ("adg", "rk2", 0.01, 0.1)])
def test_viscous_burgers_converges_to_cole_hopf(mode, rk, fac, t_end):
    # LDG(2) against the exact solution (nu = 0.1, dt = fac dx^2, so the time error stays below
    # the space error): third order, as Fig. burgers-solution shows for LDG(2)-RK2 and
    # ALDG(2)-AT2-RK2 (P = 4, L = 3, probabilities 0.3, 0.4, 0.3). The asynchronous AT2 scheme
    # needs the smaller step (Section 6 runs it at sigma = 0.0005): at dt = 0.1 dx^2 it grows.
    nu, a, p = 0.1, [2.0, 1.0, 0.5], 2
    errs = []
    for K in (16, 32, 64):
        dx = TWO_PI / K
        n = int(math.ceil(t_end / (fac * dx * dx)))
        dt = t_end / n
        x = dg.node_coordinates(K, p, 0.0, TWO_PI)
        tbl = delays.delay_table(5, 4, n, 3, [0.3, 0.4, 0.3]) if mode == "adg" else None
        prob = dg.Problem(pde="burgers", K=K, p=p, P=4, dt=dt, nu=nu, rk=rk, mode=mode, q=2,
                          delays=tbl)
        uN = dg.run(prob, _cole_hopf(x, 0.0, nu, a), n).numpy()
        errs.append(np.mean(np.abs(uN - _cole_hopf(x, t_end, nu, a))))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(slopes) > 2.6, (errs, slopes)


def test_viscous_burgers_conserves_under_delays():
    # Single-valued face values (the common delayed level) keep sum_e (dx/2) w . u^e constant.
    K, p, P = 48, 2, 6
    x = dg.node_coordinates(K, p, 0.0, TWO_PI)
    u0 = 0.5 + np.sin(x) + 0.3 * np.cos(3 * x)
    tbl = delays.delay_table(3, P, 60, 3)
    prob = dg.Problem(pde="burgers", K=K, p=p, P=P, dt=2e-4, nu=0.05, mode="adg", q=2,
                      delays=tbl)
    s = dg.Solver(prob, u0)
    m0 = s.integral()
    s.run(60)
    assert abs(s.integral() - m0) < 1e-13 * abs(m0)


def test_viscous_zero_delay_is_sync():
    # k = 0 at every face: every AT sum is the current face value itself.
    K, p, P = 32, 2, 4
    x = dg.node_coordinates(K, p, 0.0, TWO_PI)
    u0 = 0.5 + np.sin(x)
    common = dict(pde="burgers", K=K, p=p, P=P, dt=2e-3, nu=0.1, q=2)
    a = dg.run(dg.Problem(mode="sync", **common), u0, 30).numpy()
    b = dg.run(dg.Problem(mode="adg", delays=np.zeros((1, P), np.uint8), **common), u0, 30).numpy()
    assert np.array_equal(a, b)
