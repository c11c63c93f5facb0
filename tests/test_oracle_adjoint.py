"""Pins of the oracle's discrete gradient (reverse-mode autodiff of the forward oracle)
against central finite differences and, for the linear case, the dot-product identity."""
import math

import numpy as np
import pytest
import torch

from oracle import dg, delays
from workloads import HALF_PLUS_SIN, random_nodal

TWO_PI = 2 * math.pi


def _burgers_problem(K=32, p=3, P=4, steps=40):
    u0 = dg.modes_initial(HALF_PLUS_SIN, K, p)
    dt = dg.dt_from_cfl("burgers", 0.01, TWO_PI / K, 1.0, u0)
    tbl = delays.delay_table(3, P, steps, 4)
    return dg.Problem(pde="burgers", K=K, p=p, P=P, dt=dt, mode="adg", q=2, delays=tbl), u0


def test_burgers_gradient_matches_central_differences():
    prob, u0 = _burgers_problem()
    steps = 40
    g = u0 + 0.05 * random_nodal(prob.K, prob.p, 5)
    J, grad = dg.gradient(prob, u0, g, steps)
    rng = np.random.default_rng(6)
    for _ in range(4):
        v = rng.normal(size=u0.shape)
        v /= np.linalg.norm(v)
        eps = 1e-5
        Jp = float(dg.misfit(prob, dg.run(prob, u0 + eps * v, steps), torch.tensor(g)))
        Jm = float(dg.misfit(prob, dg.run(prob, u0 - eps * v, steps), torch.tensor(g)))
        fd = (Jp - Jm) / (2 * eps)
        ad = float(np.sum(grad * v))
        assert abs(fd - ad) <= 1e-6 * max(abs(fd), 1e-8)


def test_linear_adjoint_dot_product_identity():
    # For linear advection the final field is A u0 (A linear, delays fixed). With
    # J = 1/2 <A u0 - g, A u0 - g>_M the gradient is A^T M_h (A u0 - g), so
    # <grad(u0 = v, g = 0), w> = <A v, A w>_M must be symmetric in v and w.
    K, p, P, N = 24, 2, 4, 30
    tbl = delays.delay_table(8, P, N, 4)
    prob = dg.Problem(pde="advection", K=K, p=p, P=P, dt=0.02 * TWO_PI / K, mode="adg",
                      q=3, delays=tbl)
    v = random_nodal(K, p, 1)
    w = random_nodal(K, p, 2)
    z = np.zeros_like(v)
    _, gv = dg.gradient(prob, v, z, N)
    _, gw = dg.gradient(prob, w, z, N)
    a, b = float(np.sum(gv * w)), float(np.sum(gw * v))
    assert abs(a - b) <= 1e-13 * max(abs(a), abs(b))
