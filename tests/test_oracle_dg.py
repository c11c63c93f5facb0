"""Pins of the oracle's DG / ADG / ADG-AT solver against what the paper and the
mathematics fix: Eq. DGscheme assembly, Fourier symbols, conservation (Section 4.1),
the k = 0 reduction, translation invariance, exact transport, convergence orders
(Section 6.2) and the exact Burgers solution before the shock."""
import math

import numpy as np
import pytest
import torch

from oracle import dg, delays, fourier
from oracle.operators import ref_ops
from workloads import PAPER_FIG6, SIN, HALF_PLUS_SIN, constant_table

TWO_PI = 2 * math.pi


def _prob(**kw):
    base = dict(pde="advection", K=32, p=2, P=8, dt=0.1 * TWO_PI / 32, mode="sync", q=1)
    base.update(kw)
    return dg.Problem(**base)


@pytest.mark.parametrize("a", [1.0, -0.7])
def test_rhs_matches_paper_K_matrix_assembly(a):
    # Eq. DGscheme: M du/dt = (2a/dx)(K- u^{e-1} + (K_l+S+K_r) u^e + K+ u^{e+1}),
    # with upwind weights B+ = 1, B- = 0 for a >= 0 and B+ = 0, B- = 1 for a < 0.
    K, p = 16, 3
    prob = _prob(K=K, p=p, P=1, a=a)
    u = np.random.default_rng(1).normal(size=(K, p + 1))
    s = dg.Solver(prob, u)
    got = s.L(torch.tensor(u), 0, 0).numpy()
    ops = ref_ops(p)
    Bp, Bm = (1.0, 0.0) if a >= 0 else (0.0, 1.0)
    Km, Kl, Kr, Kp = ops.flux_matrices(Bp, Bm)
    dx = TWO_PI / K
    ref = np.zeros_like(u)
    for e in range(K):
        body = Km @ u[e - 1] + (Kl + ops.S + Kr) @ u[e] + Kp @ u[(e + 1) % K]
        ref[e] = (2 * a / dx) * ops.Minv @ body
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def _order_residuals(a, b):
    """Residuals of the Runge-Kutta order conditions up to order four (c_i = sum_j a_ij)."""
    S = len(b)
    c = [sum(a[i]) for i in range(S)]
    Ac = [sum(a[i][j] * c[j] for j in range(S)) for i in range(S)]
    Ac2 = [sum(a[i][j] * c[j] ** 2 for j in range(S)) for i in range(S)]
    AAc = [sum(a[i][j] * Ac[j] for j in range(S)) for i in range(S)]
    from fractions import Fraction as Fr
    return [sum(b) - 1,
            sum(b[i] * c[i] for i in range(S)) - Fr(1, 2),
            sum(b[i] * c[i] ** 2 for i in range(S)) - Fr(1, 3),
            sum(b[i] * Ac[i] for i in range(S)) - Fr(1, 6),
            sum(b[i] * c[i] ** 3 for i in range(S)) - Fr(1, 4),
            sum(b[i] * c[i] * Ac[i] for i in range(S)) - Fr(1, 8),
            sum(b[i] * Ac2[i] for i in range(S)) - Fr(1, 12),
            sum(b[i] * AAc[i] for i in range(S)) - Fr(1, 24)]


def test_two_register_form_of_the_paper_rk2():
    # Eq. dg2-rk2 written as a 2N scheme: dU1 = dt L(u), U1 = u + dU1, dU2 = -dU1 + dt L(U1),
    # u+ = U1 + dU2 / 2; its Butcher form is the two-stage tableau of the equation.
    from fractions import Fraction as Fr
    a, b = dg.two_register_tableau([Fr(0), Fr(-1)], [Fr(1), Fr(1, 2)])
    assert (a, b) == ([[0, 0], [1, 0]], [Fr(1, 2), Fr(1, 2)])
    assert dg.TABLEAUX["rk2"] == ([[0.0, 0.0], [1.0, 0.0]], [0.5, 0.5])


def test_two_register_schemes_meet_their_order_conditions():
    # Williamson's scheme: third order exactly (rational arithmetic), nodes c = (0, 1/3, 3/4),
    # and not fourth order; Carpenter and Kennedy's: the eight conditions up to fourth order.
    from fractions import Fraction as Fr
    a, b = dg.two_register_tableau(*dg.TWO_REGISTER["lsrk3"])
    r = _order_residuals(a, b)
    assert [sum(row) for row in a] == [0, Fr(1, 3), Fr(3, 4)]
    assert all(x == 0 for x in r[:4]) and any(x != 0 for x in r[4:])
    a, b = dg.two_register_tableau(*dg.TWO_REGISTER["lsrk4"])
    assert max(abs(float(x)) for x in _order_residuals(a, b)) < 1e-20


@pytest.mark.parametrize("rk", ["rk1", "rk2", "ssprk3", "rk4", "lsrk3", "lsrk4"])
@pytest.mark.parametrize("p", [1, 3])
def test_sync_step_equals_amplification_matrix(rk, p):
    K, kap, sigma = 24, 5, 0.1
    dx = TWO_PI / K
    theta = kap * dx
    mu = np.random.default_rng(2).normal(size=p + 1) + 1j * np.random.default_rng(3).normal(size=p + 1)
    phase = np.exp(1j * theta * np.arange(K))[:, None]
    u0 = np.real(mu[None, :] * phase)
    uN = dg.run(_prob(K=K, p=p, P=1, dt=sigma * dx, rk=rk), u0, 1).numpy()
    G = fourier.G_sync(p, theta, sigma, rk)
    ref = np.real((G @ mu)[None, :] * phase)
    assert np.max(np.abs(uN - ref)) < 1e-13


@pytest.mark.parametrize("rk,k,q", [("rk1", 2, 1), ("rk2", 1, 2), ("ssprk3", 0, 3),
                                    ("ssprk3", 2, 1), ("ssprk3", 1, 2), ("rk4", 1, 3),
                                    ("lsrk3", 2, 2), ("lsrk4", 1, 3)])
def test_delayed_scheme_equals_fourier_recurrence(rk, k, q):
    # P = K: every face is a PE face; a constant delay k turns the scheme into a linear
    # recurrence on the amplitudes of one Fourier mode (block companion, Section 4.2.2).
    K, p, kap, sigma, N = 32, 2, 3, 0.02, 12
    dx = TWO_PI / K
    theta = kap * dx
    rng = np.random.default_rng(4)
    mu = rng.normal(size=p + 1) + 1j * rng.normal(size=p + 1)
    phase = np.exp(1j * theta * np.arange(K))[:, None]
    u0 = np.real(mu[None, :] * phase)
    prob = _prob(K=K, p=p, P=K, dt=sigma * dx, rk=rk, mode="adg", q=q,
                 delays=constant_table(1, K, k))
    uN = dg.run(prob, u0, N).numpy()
    uh = fourier.delayed_recurrence(p, theta, sigma, rk, k, q, mu, N)
    ref = np.real(uh[None, :] * phase)
    assert np.max(np.abs(uN - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def _integral_drift(mode, q, naive=False, steps=200):
    K, p, P = 64, 2, 8
    dx = TWO_PI / K
    tbl = delays.delay_table(5, P, steps, 3, [0.3, 0.4, 0.3])
    tblm = delays.delay_table(6, P, steps, 3, [0.3, 0.4, 0.3]) if naive else None
    prob = _prob(K=K, p=p, P=P, dt=0.02 * dx, mode=mode, q=q, delays=tbl, delays_minus=tblm)
    u0 = dg.modes_initial(PAPER_FIG6, K, p) + 1.0
    s = dg.Solver(prob, u0)
    I0 = float(s.integral())
    s.run(steps)
    return abs(float(s.integral()) - I0), I0


@pytest.mark.parametrize("mode,q", [("sync", 1), ("adg", 1), ("adg", 2), ("adg", 3)])
def test_conservation_to_roundoff(mode, q):
    drift, I0 = _integral_drift(mode, q)
    assert drift < 1e-12 * abs(I0)


def test_naive_delays_break_conservation():
    drift, I0 = _integral_drift("naive", 1, naive=True)
    assert drift > 1e-6 * abs(I0)


@pytest.mark.parametrize("pde,q", [("advection", 1), ("advection", 3), ("burgers", 2)])
def test_zero_delay_is_bitwise_sync(pde, q):
    K, p, P = 32, 3, 4
    u0 = dg.modes_initial(HALF_PLUS_SIN if pde == "burgers" else PAPER_FIG6, K, p)
    dt = dg.dt_from_cfl(pde, 0.05, TWO_PI / K, 1.0, u0)
    a = dg.run(_prob(pde=pde, K=K, p=p, P=P, dt=dt), u0, 30)
    b = dg.run(_prob(pde=pde, K=K, p=p, P=P, dt=dt, mode="adg", q=q,
                     delays=constant_table(30, P, 0)), u0, 30)
    assert torch.equal(a, b)


def test_translation_invariance_bitwise():
    K, p, P = 32, 2, 4
    u0 = np.random.default_rng(7).normal(size=(K, p + 1))
    a = dg.run(_prob(K=K, p=p, P=1), u0, 10).numpy()
    b = dg.run(_prob(K=K, p=p, P=1), np.roll(u0, 1, axis=0), 10).numpy()
    assert np.array_equal(np.roll(a, 1, axis=0), b)
    # ADG: shift by one PE and rotate the delay table columns with it.
    Kpe = K // P
    tbl = delays.delay_table(3, P, 10, 3)
    a = dg.run(_prob(K=K, p=p, P=P, mode="adg", q=2, delays=tbl), u0, 10).numpy()
    b = dg.run(_prob(K=K, p=p, P=P, mode="adg", q=2, delays=np.roll(tbl, 1, axis=1)),
               np.roll(u0, Kpe, axis=0), 10).numpy()
    assert np.array_equal(np.roll(a, Kpe, axis=0), b)


def _advection_error(p, rk, sigma, K, mode, q, tbl_fn=None, t_end=1.0, P=8, modes=PAPER_FIG6):
    dx = TWO_PI / K
    n = math.ceil(t_end / (sigma * dx))
    dt = t_end / n
    prob = _prob(K=K, p=p, P=P, dt=dt, rk=rk, mode=mode, q=q,
                 delays=tbl_fn(n, P) if tbl_fn else None)
    uN = dg.run(prob, dg.modes_initial(modes, K, p), n).numpy()
    x = dg.node_coordinates(K, p, 0.0, TWO_PI)
    ex = sum(A * np.sin(k * (x - t_end) + ph) for A, k, ph in zip(modes.amp, modes.kappa, modes.phase))
    return uN, ex


def _slopes(errs):
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


def test_exact_period_translation():
    # a = 1 on [0, 2 pi]: after t = 2 pi the exact solution is u0 again.
    K, p = 32, 3
    dx = TWO_PI / K
    n = math.ceil(TWO_PI / (0.1 * dx))
    uN = dg.run(_prob(K=K, p=p, P=1, dt=TWO_PI / n), dg.modes_initial(SIN, K, p), n).numpy()
    assert np.max(np.abs(uN - dg.modes_initial(SIN, K, p))) < 1e-5


@pytest.mark.parametrize("p,rk,sigma", [(1, "rk2", 0.1), (2, "ssprk3", 0.04), (3, "rk4", 0.02),
                                        (2, "lsrk3", 0.04), (3, "lsrk4", 0.02)])
def test_sync_convergence_order(p, rk, sigma):
    # Section 4.3 / Fig. 7: the synchronous DG(p)-RK error falls as dx^{p+1}.
    Ks = (16, 32, 64)
    errs = [np.mean(np.abs(np.subtract(*_advection_error(p, rk, sigma, K, "sync", 1, t_end=0.5))))
            for K in Ks]
    assert min(_slopes(errs)) > p + 1 - 0.3


def test_adg_standard_flux_first_order_and_at_recovery():
    # Section 4.3 / Fig. 7: with delayed standard fluxes the asynchrony error is first
    # order (it lives in the PE-boundary elements: max norm). AT2 restores second order.
    tb = lambda n, P: delays.delay_table(11, P, n, 3, [0.3, 0.4, 0.3])
    e_std, e_at = [], []
    for K in (64, 128, 256):
        s, _ = _advection_error(1, "rk2", 0.1, K, "sync", 1, t_end=1.0)
        a, _ = _advection_error(1, "rk2", 0.1, K, "adg", 1, tb, t_end=1.0)
        b, _ = _advection_error(1, "rk2", 0.1, K, "adg", 2, tb, t_end=1.0)
        e_std.append(np.max(np.abs(a - s)))
        e_at.append(np.max(np.abs(b - s)))
    sl = _slopes(e_std)
    assert 0.5 < np.mean(sl) < 1.5
    assert np.mean(_slopes(e_at)) > 1.6
    assert e_at[-1] < 0.1 * e_std[-1]


def test_naive_delays_first_order_in_mean():
    tb = lambda n, P: delays.delay_table(12, P, n, 3, [0.3, 0.4, 0.3])
    errs = []
    for K in (64, 128, 256):
        dx = TWO_PI / K
        n = math.ceil(1.0 / (0.1 * dx))
        prob = _prob(K=K, p=1, P=8, dt=1.0 / n, rk="rk2", mode="naive", delays=tb(n, 8),
                     delays_minus=delays.delay_table(13, 8, n, 3, [0.3, 0.4, 0.3]))
        u0 = dg.modes_initial(PAPER_FIG6, K, 1)
        s = dg.run(_prob(K=K, p=1, P=8, dt=1.0 / n, rk="rk2"), u0, n).numpy()
        errs.append(np.mean(np.abs(dg.run(prob, u0, n).numpy() - s)))
    assert 0.7 < np.mean(_slopes(errs)) < 1.3


def test_at3_recovers_third_order_inside_stability_bound():
    # Fig. 8(b): ADG(2)-AT3-RK3. At sigma = 0.01 the delayed self-feedback of the
    # upwind-side element stays inside its stability bound (see the next test).
    tb = lambda n, P: delays.delay_table(14, P, n, 3, [0.3, 0.4, 0.3])
    errs = []
    for K in (16, 32, 64):
        u, ex = _advection_error(2, "ssprk3", 0.01, K, "adg", 3, tb, t_end=0.25)
        errs.append(np.mean(np.abs(u - ex)))
    assert min(_slopes(errs)) > 2.7


def test_delayed_self_feedback_instability():
    # With the common delayed level (Eq. asyncEulerDGconserved) the upwind-side element
    # sees its own trace k steps late through the lift term: gain 2 sigma (p+1)^2/2 per
    # step. A delay with gain * k > 1 grows; far inside the bound the run stays bounded.
    K, p, P, N = 64, 2, 8, 400
    dx = TWO_PI / K
    u0 = dg.modes_initial(SIN, K, p)
    grow = dg.run(_prob(K=K, p=p, P=P, dt=0.1 * dx, mode="adg", q=1,
                        delays=constant_table(1, P, 3)), u0, N)
    calm = dg.run(_prob(K=K, p=p, P=P, dt=0.01 * dx, mode="adg", q=1,
                        delays=constant_table(1, P, 3)), u0, N)
    assert float(grow.abs().max()) > 1e3
    assert float(calm.abs().max()) < 1.01


def _burgers_exact(x, t, offset=0.5):
    # u = u0(x - u t) solved by Newton from u0(x); smooth for t < 1 (u0 = 0.5 + sin x).
    u = offset + np.sin(x)
    for _ in range(60):
        g = u - offset - np.sin(x - u * t)
        dg_ = 1 + t * np.cos(x - u * t)
        u = u - g / dg_
    return u


def test_burgers_sync_matches_characteristics():
    errs = []
    for K in (32, 64, 128):
        p = 2
        u0 = dg.modes_initial(HALF_PLUS_SIN, K, p)
        dx = TWO_PI / K
        t_end = 0.3
        n = math.ceil(t_end / dg.dt_from_cfl("burgers", 0.05, dx, 1.0, u0))
        uN = dg.run(_prob(pde="burgers", K=K, p=p, P=1, dt=t_end / n), u0, n).numpy()
        ex = _burgers_exact(dg.node_coordinates(K, p, 0.0, TWO_PI), t_end)
        errs.append(np.mean(np.abs(uN - ex)))
    assert errs[-1] < 1e-5
    assert min(_slopes(errs)) > 2.3


def test_window_solver_matches_full_mesh_at_centre():
    K, p, P, N = 64, 2, 8, 4
    u0 = np.random.default_rng(9).normal(size=(K, p + 1))
    tbl = delays.delay_table(21, P, N, 4)
    for pde in ("advection", "burgers"):
        dt = 0.01 * TWO_PI / K
        full = dg.run(_prob(pde=pde, K=K, p=p, P=P, dt=dt, mode="adg", q=2, delays=tbl), u0, N).numpy()
        lo, W = 10, 40
        win = dg.run(_prob(pde=pde, K=W, p=p, P=P, dt=dt, mode="adg", q=2, delays=tbl,
                           window_lo=lo, K_global=K), u0[lo:lo + W], N).numpy()
        r = 3 * N
        assert np.array_equal(win[r:W - r], full[lo + r:lo + W - r])
