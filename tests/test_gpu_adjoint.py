"""GPU parity of the discrete adjoint (adg_grad): against the oracle's gradient (reverse-mode
autodiff of the forward oracle), against central finite differences of the GPU forward
map at the full adjoint workload size, and the dot-product identity for linear advection."""
import math

import numpy as np
import pytest
import torch

import paper_2404_03399_gb300 as adg
from oracle import dg, delays as odelays
from workloads import ADJOINT_64K, HALF_PLUS_SIN, PAPER_FIG6, constant_table, random_nodal

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_03399_gb300 import build
    build.build()


def _pair(cfg, u0, g, steps, ckpt):
    s = adg.Solver(cfg, torch.tensor(u0, device="cuda"))
    dt = s.dt
    J, grad = s.grad(torch.tensor(g, device="cuda"), steps, ckpt)
    after = s.state().cpu().numpy()
    n_after = s.n
    s.close()
    assert n_after == 0 and np.array_equal(after, u0), "adg_grad must leave the state unchanged"
    q = cfg.q if cfg.mode == "at" else 1
    tbl = None
    if cfg.mode != "sync" and cfg.P > 1:
        tbl = cfg.table if cfg.table is not None else odelays.delay_table(cfg.seed, cfg.P, steps, cfg.L)
    prob = dg.Problem(pde=cfg.pde, K=cfg.K, p=cfg.p, P=cfg.P, dt=dt, a=cfg.a,
                      mode="adg" if tbl is not None else "sync", q=q, delays=tbl)
    Jo, go = dg.gradient(prob, u0, g, steps)
    return J, grad.cpu().numpy(), Jo, go


@pytest.mark.parametrize("case", [
    dict(pde="burgers", K=64, p=3, P=4, L=4, q=2, mode="at", steps=40, ckpt=16),
    dict(pde="burgers", K=48, p=2, P=48, L=3, q=2, mode="at", steps=25, ckpt=7),
    dict(pde="burgers", K=80, p=4, P=8, L=3, q=1, mode="async", steps=30, ckpt=50),
    dict(pde="burgers", K=64, p=1, P=4, L=1, q=0, mode="sync", steps=20, ckpt=4),
    dict(pde="advection", K=96, p=2, P=8, L=3, q=3, mode="at", steps=45, ckpt=10, a=1.3),
    dict(pde="advection", K=96, p=3, P=6, L=4, q=2, mode="at", steps=33, ckpt=8, a=-0.7),
    dict(pde="advection", K=40, p=2, P=40, L=2, q=2, mode="at", steps=20, ckpt=5, a=1.0),
])
def test_gradient_matches_oracle(case):
    c = dict(case)
    steps, ckpt = c.pop("steps"), c.pop("ckpt")
    cfg = adg.Config(cfl=0.01, seed=9, **c)
    if cfg.pde == "burgers":
        u0 = dg.modes_initial(HALF_PLUS_SIN, cfg.K, cfg.p)
    else:
        u0 = dg.modes_initial(PAPER_FIG6, cfg.K, cfg.p)
    g = u0 + 0.05 * random_nodal(cfg.K, cfg.p, 3)
    J, grad, Jo, go = _pair(cfg, u0, g, steps, ckpt)
    assert abs(J - Jo) <= TOL * abs(Jo)
    assert np.max(np.abs(grad - go)) <= TOL * np.max(np.abs(go))


def test_caller_table_gradient():
    cfg = adg.Config(pde="burgers", K=64, p=2, P=8, L=3, q=2, mode="at", cfl=0.01,
                     table=constant_table(1, 8, 2))
    u0 = dg.modes_initial(HALF_PLUS_SIN, 64, 2)
    g = u0 + 0.05 * random_nodal(64, 2, 4)
    J, grad, Jo, go = _pair(cfg, u0, g, 30, 9)
    assert np.max(np.abs(grad - go)) <= TOL * np.max(np.abs(go))


def test_linear_dot_product_identity():
    # J(u0) = 1/2 <A u0, A u0>_M with g = 0, so grad(v) = A^T M A v and
    # <grad(v), w> = <grad(w), v>.
    cfg = adg.Config(pde="advection", K=512, p=3, P=16, L=5, q=3, mode="at", cfl=0.005, seed=2)
    v = random_nodal(512, 3, 10)
    w = random_nodal(512, 3, 11)
    z = torch.zeros((512, 4), dtype=torch.float64, device="cuda")
    grads = []
    for x in (v, w):
        s = adg.Solver(cfg, torch.tensor(x, device="cuda"))
        grads.append(s.grad(z, 150, 40)[1].cpu().numpy())
        s.close()
    a, b = float(np.sum(grads[0] * w)), float(np.sum(grads[1] * v))
    assert abs(a - b) <= 1e-13 * max(abs(a), abs(b))


def test_autograd_function():
    cfg = adg.Config(pde="burgers", K=64, p=3, P=4, L=4, q=2, mode="at", cfl=0.01, seed=5)
    u0 = torch.tensor(dg.modes_initial(HALF_PLUS_SIN, 64, 3), device="cuda", requires_grad=True)
    g = (u0.detach() + 0.01).contiguous()
    J = adg.ADGFunction.apply(u0, cfg, g, 30, 8)
    J.backward()
    s = adg.Solver(cfg, u0.detach())
    J2, grad = s.grad(g, 30, 8)
    s.close()
    assert abs(float(J.detach()) - J2) == 0.0
    assert torch.equal(u0.grad, grad)


def test_full_size_finite_differences():
    # The adjoint workload: Burgers, K = 65536, p = 3, 1024 PEs, delays uniform in {0..3},
    # AT order 2, 2000 SSP-RK3 steps, checkpoints every 50. The gradient along 32 seeded
    # unit directions agrees with central differences of the GPU forward map.
    w = ADJOINT_64K
    cfg = adg.Config(pde="burgers", K=w.K, p=w.p, P=w.P, L=w.L, q=w.q, mode="at", cfl=w.cfl, seed=w.seed)
    u0 = adg.eval_modes(cfg, w.modes.amp, w.modes.kappa, w.modes.phase, w.modes.offset)
    rng = np.random.default_rng(7)
    amp = rng.uniform(0.25, 1.0, 4)
    kap = rng.integers(1, 17, 4).astype(float)
    ph = rng.uniform(0, 2 * math.pi, 4)
    shifted = adg.eval_modes(cfg, [1.0], [1.0], [-0.003], 0.5)
    g = shifted + 0.01 * adg.eval_modes(cfg, amp, kap, ph, 0.0)
    s = adg.Solver(cfg, u0)
    dt = s.dt
    J, grad = s.grad(g, w.steps, 50)
    s.close()
    fixed = adg.Config(pde="burgers", K=w.K, p=w.p, P=w.P, L=w.L, q=w.q, mode="at", dt=dt, seed=w.seed)

    def Jof(x):
        t = adg.Solver(fixed, x)
        t.step(w.steps)
        val = t.misfit(g)
        t.close()
        return val

    gen = torch.Generator(device="cpu").manual_seed(123)
    worst = 0.0
    eps = 1e-4
    for _ in range(32):
        d = torch.randn(u0.shape, generator=gen, dtype=torch.float64).cuda()
        d /= torch.linalg.norm(d)
        fd = (Jof(u0 + eps * d) - Jof(u0 - eps * d)) / (2 * eps)
        ad = float(torch.sum(grad * d))
        worst = max(worst, abs(fd - ad) / max(abs(ad), 1e-30))
    assert worst <= 1e-6, worst


@pytest.mark.parametrize("mode,P,L,q", [("at", 8, 4, 2), ("sync", 1, 1, 0)])
def test_gradient_independent_of_checkpoint_interval(mode, P, L, q):
    # Recomputation replays the forward bit for bit, so the gradient does not depend on the
    # checkpoint interval: C = 7 and 40 recompute on a second stream while the adjoint of the
    # next segment runs; C = 300 (2C larger than the 512-row delay window) runs segments one
    # after the other; C = 320 keeps the whole run in one recorded segment.
    cfg = adg.Config(pde="burgers", K=96, p=3, P=P, L=L, q=q, mode=mode, cfl=0.01, seed=3)
    u0 = dg.modes_initial(HALF_PLUS_SIN, 96, 3)
    g = torch.tensor(u0 + 0.05 * random_nodal(96, 3, 5), device="cuda")
    out = []
    for ckpt in (7, 40, 300, 320):
        s = adg.Solver(cfg, torch.tensor(u0, device="cuda"))
        J, grad = s.grad(g, 310, ckpt)
        s.close()
        out.append((J, grad.cpu().numpy()))
    for J, grad in out[1:]:
        assert J == out[0][0]
        assert np.array_equal(grad, out[0][1])
