"""Pins of the oracle's one-dimensional Euler solver (Section 6, Sod's shock tube): the exact
Riemann solution against the jump conditions it must satisfy, free-stream preservation,
conservation, convergence on a smooth wave, and the Sod solution of DG(1)-RK2 and
ADG(1)-AT2-RK2 with the limiter against the exact one."""
import math

import numpy as np
import pytest
import torch

from oracle import delays, dg, euler

G = euler.GAMMA


def test_exact_riemann_solution_meets_the_jump_conditions():
    left, right = euler.SOD_LEFT, euler.SOD_RIGHT
    ps, us = euler.star_state(left, right)
    # right shock: mass, momentum and energy fluxes continuous in the shock frame
    rr, ur, pr = right
    rs = euler.sample(left, right, us + 1e-9)[0]
    S = (rs * us - rr * ur) / (rs - rr)
    Er = pr / (G - 1) + 0.5 * rr * ur ** 2
    Es = ps / (G - 1) + 0.5 * rs * us ** 2
    assert abs(rr * (ur - S) - rs * (us - S)) < 1e-12
    assert abs(rr * ur * (ur - S) + pr - (rs * us * (us - S) + ps)) < 1e-12
    assert abs((Er + pr) * ur - S * Er - ((Es + ps) * us - S * Es)) < 1e-12
    # left rarefaction: isentropic, and u + 2c/(gamma-1) constant through the fan and across
    rl, ul, pl = left
    cl = math.sqrt(G * pl / rl)
    inv = ul + 2 * cl / (G - 1)
    for s in np.linspace(-cl, us - 1e-9, 7):
        rho, u, p = euler.sample(left, right, s)
        assert abs(p / rho ** G - pl / rl ** G) < 1e-12
        assert abs(u + 2 * math.sqrt(G * p / rho) / (G - 1) - inv) < 1e-12
    # contact: pressure and velocity continuous, density jumps
    a, b = euler.sample(left, right, us - 1e-9), euler.sample(left, right, us + 1e-9)
    assert abs(a[2] - b[2]) < 1e-12 and abs(a[1] - b[1]) < 1e-12 and a[0] > b[0]


def _state(x, rho, u, p):
    return torch.tensor(euler.conserved(rho, u, p))


@pytest.mark.parametrize("mode", ["sync", "adg"])
def test_free_stream_is_preserved_and_integrals_conserved(mode):
    K, p, P = 64, 1, 4
    x = dg.node_coordinates(K, p, 0.0, 0.02)
    tbl = delays.delay_table(4, P, 50, 3, [0.3, 0.4, 0.3]) if mode == "adg" else None
    prob = euler.EulerProblem(K=K, p=p, P=P, dt=2e-6, mode=mode, q=2, delays=tbl)
    U0 = _state(x, 1.0 + 0 * x, 0.7 + 0 * x, 2.0 + 0 * x)
    U = euler.run(prob, U0, 20)
    assert torch.max(torch.abs(U - U0)) < 1e-14 * torch.max(torch.abs(U0))
    rough = _state(x, 1.0 + 0.5 * np.sin(2 * math.pi * x / 0.02) ** 3, 0.3 + 0 * x,
                   1.0 + 0.4 * np.cos(6 * math.pi * x / 0.02))
    s = euler.EulerSolver(prob, rough)
    I0 = s.integrals()
    s.run(40)
    assert torch.max(torch.abs(s.integrals() - I0) / torch.abs(I0)) < 1e-13


@pytest.mark.parametrize("p", [1, 2])
def test_smooth_density_wave_converges(p):
    # rho = 1 + 0.2 sin(2 pi x / l), u = 1, p = 1 is carried at speed 1 unchanged; without the
    # limiter DG(p)-SSP-RK3 converges at order p + 1.
    errs = []
    for K in (16, 32, 64):
        x = dg.node_coordinates(K, p, 0.0, 0.02)
        dt = 0.05 * 0.02 / K / 2.5
        n = int(round(0.004 / dt))
        dt = 0.004 / n
        prob = euler.EulerProblem(K=K, p=p, P=1, dt=dt, rk="ssprk3", limiter=False)
        U = euler.run(prob, _state(x, 1 + 0.2 * np.sin(2 * math.pi * x / 0.02), 1 + 0 * x, 1 + 0 * x), n)
        exact = 1 + 0.2 * np.sin(2 * math.pi * (x - 0.004) / 0.02)
        errs.append(float(np.mean(np.abs(U[0].numpy() - exact))))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(slopes) > p + 1 - 0.3, (errs, slopes)


def _sod(K, mode, P=8):
    x = dg.node_coordinates(K, 1, 0.0, 0.02)
    rho, u, p = euler.sod_periodic(x, 0.0)
    dt = 0.1 * (0.02 / K)
    n = int(round(0.002 / dt))
    tbl = delays.delay_table(9, P, n, 3, [0.3, 0.4, 0.3]) if mode == "adg" else None
    prob = euler.EulerProblem(K=K, p=1, P=P, dt=0.002 / n, rk="rk2", mode=mode, q=2, delays=tbl)
    U = euler.run(prob, torch.tensor(euler.conserved(rho, u, p)), n).numpy()
    exact = euler.sod_periodic(x, 0.002)[0]
    return U[0], exact


def test_sod_with_limiter_converges_and_adg_at2_agrees():
    # Section 6: DG(1)-RK2 with the MUSCL limiter and ADG(1)-AT2-RK2 (L = 3, probabilities
    # 0.3 / 0.4 / 0.3) capture Sod's shock tube and agree with each other; the mean density
    # error against the exact solution at t = 0.002 falls with resolution.
    e = []
    for K in (256, 512):
        rho, exact = _sod(K, "sync")
        assert np.all(np.isfinite(rho)) and rho.min() > 0.1 and rho.max() < 1.02
        e.append(float(np.mean(np.abs(rho - exact))))
    assert e[1] < 0.75 * e[0] and e[1] < 0.01, e
    rho_a, _ = _sod(512, "adg")
    rho_s, exact = _sod(512, "sync")
    assert float(np.mean(np.abs(rho_a - exact))) < 1.2 * e[1]
    assert float(np.mean(np.abs(rho_a - rho_s))) < 0.5 * e[1]


def test_euler_zero_delay_is_sync():
    K = 64
    x = dg.node_coordinates(K, 1, 0.0, 0.02)
    U0 = torch.tensor(euler.conserved(*euler.sod_periodic(x, 0.0)))
    a = euler.run(euler.EulerProblem(K=K, p=1, P=4, dt=2e-6, q=2), U0, 25)
    b = euler.run(euler.EulerProblem(K=K, p=1, P=4, dt=2e-6, q=2, mode="adg",
                                     delays=np.zeros((1, 4), np.uint8)), U0, 25)
    assert torch.equal(a, b)


@pytest.mark.parametrize("left,right", [(euler.SOD_LEFT, euler.SOD_RIGHT),
                                        ((1.0, 0.75, 1.0), (0.125, 0.0, 0.1)),
                                        ((1.0, -2.0, 0.4), (1.0, 2.0, 0.4))])
def test_exact_riemann_solution_is_mirror_symmetric(left, right):
    # x -> -x swaps the states and negates the velocities: the mirrored problem's solution at
    # s is the original one at -s with u negated. Sod's problem (left rarefaction, right shock)
    # thus pins the left-shock and right-rarefaction branches too; the last pair has two
    # rarefactions.
    mirror = lambda st: (st[0], -st[1], st[2])
    for s in np.linspace(-2.5, 2.5, 41):
        a = euler.sample(left, right, s)
        b = euler.sample(mirror(right), mirror(left), -s)
        assert abs(a[0] - b[0]) < 1e-12 and abs(a[1] + b[1]) < 1e-12 and abs(a[2] - b[2]) < 1e-12
