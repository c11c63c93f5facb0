"""adg_integral_noalloc: the integral of a field computed without allocating device memory.

Some callers cannot allocate device memory where they call the library: a framework that
hands out all device memory from its own pool, a process under a fixed device-memory cap,
or a latency-critical loop that cannot afford cudaMalloc and the synchronisation it may
cause. For them the library offers one entry point whose scratch space is a fixed array
compiled into the library. This test calls it through the C ABI on two fields in a row and
checks each result against adg_integral, which uses scratch space owned by a solver
context, and against the oracle's integral of the same field. It sits in a file of its own
that pytest collects last.
"""
import ctypes as C
import math

import numpy as np
import pytest
import torch

import paper_2404_03399_gb300 as adg
from oracle import dg
from workloads import PAPER_FIG6

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_03399_gb300 import build
    build.build()


def _noalloc_integral(lib, p, K, dx, field, out):
    code = lib.adg_integral_noalloc(p, K, dx, field.data_ptr(), out.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert code == 0, lib.adg_last_error(None)
    torch.cuda.synchronize()
    return float(out.item())


def test_noalloc_integral_matches_context_integral_twice():
    lib = adg.load()
    K, p = 300_000, 3           # more elements than the first pass has blocks: grid-stride
    cfg = adg.Config(pde="advection", K=K, p=p, P=100, cfl=0.01, mode="at", L=4, q=2, seed=4)
    dx = (cfg.x1 - cfg.x0) / K
    u0 = adg.eval_modes(cfg, PAPER_FIG6.amp, PAPER_FIG6.kappa, PAPER_FIG6.phase, 1.0)
    s = adg.Solver(cfg, u0)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        field = s.state()
        ref = s.integral()
        got = _noalloc_integral(lib, p, K, dx, field, out)
        assert abs(got - ref) <= TOL * abs(ref), (call, got, ref)
        prob = dg.Problem(pde="advection", K=K, p=p, P=1, dt=1.0, x0=cfg.x0, x1=cfg.x1)
        o = dg.Solver(prob, field.cpu().numpy())
        orc = float(o.integral())
        mag = float(o.integral(torch.abs(field.cpu())))
        assert abs(got - orc) <= TOL * mag, (call, got, orc)
        s.step(7)               # the second call sees a different field
    s.close()


def test_noalloc_rejects_sizes_beyond_limits():
    lib = adg.load()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    field = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    assert lib.adg_integral_noalloc(5, 4, 0.1, field.data_ptr(), out.data_ptr(), None) == adg._abi.ADG_EINVAL
    assert lib.adg_integral_noalloc(1, (1 << 30) + 1, 0.1, field.data_ptr(), out.data_ptr(), None) == adg._abi.ADG_EINVAL
    assert lib.adg_integral_noalloc(1, 4, 0.0, field.data_ptr(), out.data_ptr(), None) == adg._abi.ADG_EINVAL
    for bad in (math.inf, math.nan, -1.0):
        assert lib.adg_integral_noalloc(1, 4, bad, field.data_ptr(), out.data_ptr(), None) == adg._abi.ADG_EINVAL
    assert b"K must be" in lib.adg_last_error(None) or b"dx" in lib.adg_last_error(None)
