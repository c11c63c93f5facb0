"""The host-buffer entry points (adg_init_host, adg_get_state_host) against the device-buffer
ones and the oracle: the initial field read from pinned host memory in place (over the host
link) or staged from pageable memory, the state written to pinned or pageable host memory.
Same arithmetic as the device path, so the results are compared bit for bit; one case per
path against the oracle at the FP64 tolerance of the parity tests."""
import ctypes as C
import math

import numpy as np
import pytest
import torch

import paper_2404_03399_gb300 as adg
from paper_2404_03399_gb300 import _abi
from oracle import dg, delays as odelays, euler as oeuler

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_03399_gb300 import build
    build.build()


def _host(x: np.ndarray, pinned: bool) -> torch.Tensor:
    t = torch.tensor(x, dtype=torch.float64)
    return t.pin_memory() if pinned else t


def _run(cfg, u0, steps, host_in, pinned_in, host_out, pinned_out):
    src = _host(u0, pinned_in) if host_in else torch.tensor(u0, device="cuda")
    s = adg.Solver(cfg, src)
    s.step(steps)
    if host_out:
        out = torch.empty(tuple(u0.shape), dtype=torch.float64)
        if pinned_out:
            out = out.pin_memory()
        s.state(out=out)
        got = out.numpy().copy()
    else:
        got = s.state().cpu().numpy()
    dt = s.dt
    s.close()
    return got, dt


CASES = {
    # fixed-point composed step (state kept in int64 block coordinates between the calls); at
    # this Courant number the delayed AT3 flux is inside its stability bound (at 0.05 the
    # field grows 7e4-fold in 40 steps and a 1e-15 perturbation of u0 grows to 3e-12)
    "advection_fixed": dict(pde="advection", K=1024, p=3, P=64, cfl=0.01, mode="at", L=4, q=3,
                            variant="fixed"),
    # staged FP64 stages, ragged K
    "burgers_staged": dict(pde="burgers", K=333, p=2, P=9, cfl=0.05, mode="at", L=3, q=2),
}


def _u0(cfg):
    x = dg.node_coordinates(cfg.K, cfg.p, cfg.x0, cfg.x1)
    return 0.5 + np.sin(x) + 0.25 * np.cos(3 * x)


@pytest.mark.parametrize("case", sorted(CASES))
def test_host_paths_equal_device_path_bitwise(case):
    cfg = adg.Config(seed=5, **CASES[case])
    u0 = _u0(cfg)
    steps = 37
    ref, _ = _run(cfg, u0, steps, False, False, False, False)
    for host_in, pinned_in, host_out, pinned_out in [
            (True, True, False, False), (True, False, False, False),
            (False, False, True, True), (False, False, True, False),
            (True, True, True, True), (True, False, True, False)]:
        got, _ = _run(cfg, u0, steps, host_in, pinned_in, host_out, pinned_out)
        assert np.array_equal(got, ref), (case, host_in, pinned_in, host_out, pinned_out)


def test_host_path_matches_oracle():
    cfg = adg.Config(seed=5, **CASES["advection_fixed"])
    u0 = _u0(cfg)
    steps = 40
    got, dt = _run(cfg, u0, steps, True, True, True, True)
    tbl = odelays.delay_table(cfg.seed, cfg.P, steps, cfg.L)
    prob = dg.Problem(pde="advection", K=cfg.K, p=cfg.p, P=cfg.P, dt=dt, mode="adg", q=cfg.q,
                      delays=tbl)
    ref = dg.run(prob, u0, steps).numpy()
    err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    assert err < TOL, err


def test_euler_three_fields_through_host_buffers():
    K, p, P, L, steps = 96, 2, 8, 3, 30
    x = dg.node_coordinates(K, p, 0.0, 0.02)
    U0 = oeuler.conserved(1 + 0.2 * np.sin(2 * math.pi * x / 0.02), 1 + 0 * x, 1 + 0 * x)
    cfg = adg.Config(pde="euler", K=K, p=p, P=P, x0=0.0, x1=0.02, dt=0.05 * 0.02 / K,
                     rk="ssprk3", mode="at", L=L, q=2, probs=[0.3, 0.4, 0.3], seed=17)
    ref, _ = _run(cfg, U0, steps, False, False, False, False)
    for pinned in (True, False):
        got, _ = _run(cfg, U0, steps, True, pinned, True, pinned)
        assert np.array_equal(got, ref), pinned


def test_batch_state_into_host_memory():
    cfgs = [adg.Config(pde="advection", K=K, p=p, P=K // 16, cfl=0.05, mode="at", L=3, q=2,
                       seed=11 + K) for K, p in ((256, 1), (320, 3), (512, 4))]
    u0s = [adg.eval_modes(c, [1.0, 0.3], [1.0, 4.0], [0.0, 0.5]) for c in cfgs]
    b = adg.BatchSolver(cfgs, u0s)
    b.step(25)
    for i, c in enumerate(cfgs):
        ref = b.state(i).cpu().numpy()
        for pinned in (True, False):
            out = torch.empty((c.K, c.p + 1), dtype=torch.float64)
            if pinned:
                out = out.pin_memory()
            b.state(i, out=out)
            assert np.array_equal(out.numpy(), ref), (i, pinned)
    b.close()


def test_host_entry_points_refuse_device_memory():
    L = adg.load()
    cfg = adg.Config(pde="advection", K=64, p=2, P=4, cfl=0.1, mode="at", L=3, q=2)
    c, keep = cfg.to_c()
    u0 = adg.eval_modes(cfg, [1.0], [1.0], [0.0])
    ctx = C.c_void_p()
    assert L.adg_init_host(C.byref(c), u0.data_ptr(), None, C.byref(ctx)) == _abi.ADG_EINVAL
    assert not ctx.value
    assert L.adg_init_host(C.byref(c), None, None, C.byref(ctx)) == _abi.ADG_EINVAL
    s = adg.Solver(cfg, u0)
    dev = torch.empty((64, 3), dtype=torch.float64, device="cuda")
    assert L.adg_get_state_host(s.ctx, 0, dev.data_ptr(), None) == _abi.ADG_EINVAL
    assert L.adg_get_state_host(s.ctx, 0, None, None) == _abi.ADG_EINVAL
    s.close()
