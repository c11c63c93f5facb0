"""Host-only checks of the C ABI: the library builds/loads and exports every symbol that
include/adg.h declares; configuration errors come back as ADG_EINVAL without a GPU; the
library's delay tables and LGL nodes agree with the oracle's independent versions."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

import paper_2404_03399_gb300 as adg
from paper_2404_03399_gb300 import _abi
from oracle import delays as odelays
from oracle.operators import lgl_nodes_weights

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2404_03399_gb300 import build
    build.build()
    return adg.load()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "adg.h")).read()
    declared = set(re.findall(r"\b(adg_[a-z_]+)\s*\(", hdr))
    assert declared, "no declarations parsed"
    assert declared == set(_abi.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


@pytest.mark.parametrize("bad", [
    dict(p=0), dict(p=5), dict(K=10, P=3), dict(P=0), dict(L=0), dict(L=17), dict(q=6),
    dict(x1=-1.0), dict(cfl=0.0), dict(a=0.0), dict(probs=[0.5, 0.6], L=2),
    dict(table=np.full((3, 4), 5, np.uint8), L=4, P=4, K=16),
])
def test_invalid_configs_rejected(lib, bad):
    base = dict(pde="advection", K=16, p=2, P=4, L=3, mode="at", q=2)
    base.update(bad)
    cfg = adg.Config(**base)
    c, keep = cfg.to_c()
    out = np.zeros((2, cfg.P), np.uint8)
    code = lib.adg_delay_table(C.byref(c), 0, 2, out.ctypes.data_as(C.POINTER(C.c_uint8)))
    assert code == _abi.ADG_EINVAL
    assert lib.adg_last_error(None)
    ctx = C.c_void_p()
    code = lib.adg_init(C.byref(c), C.c_void_p(8), None, C.byref(ctx))
    assert code == _abi.ADG_EINVAL and not ctx.value
    host = np.zeros((cfg.K, cfg.p + 1))
    code = lib.adg_init_host(C.byref(c), host.ctypes.data, None, C.byref(ctx))
    assert code == _abi.ADG_EINVAL and not ctx.value


def test_null_arguments(lib):
    ctx = C.c_void_p()
    assert lib.adg_init(None, None, None, C.byref(ctx)) == _abi.ADG_EINVAL
    assert lib.adg_init_host(None, None, None, C.byref(ctx)) == _abi.ADG_EINVAL
    c, keep = adg.Config(K=16, p=2, P=4).to_c()
    assert lib.adg_init_host(C.byref(c), None, None, C.byref(ctx)) == _abi.ADG_EINVAL
    assert b"u0_host" in lib.adg_last_error(None)
    assert lib.adg_step(None, 1) == _abi.ADG_EINVAL
    assert lib.adg_get_state(None, 0, None, None) == _abi.ADG_EINVAL
    assert lib.adg_get_state_host(None, 0, None, None) == _abi.ADG_EINVAL
    assert lib.adg_get_variant(None, 0, None, None) == _abi.ADG_EINVAL
    assert lib.adg_comm_stats(None, 0, None, None, None) == _abi.ADG_EINVAL
    lib.adg_destroy(None)


@pytest.mark.parametrize("seed,P,L,probs", [(0, 16, 4, None), (123, 7, 3, [0.3, 0.4, 0.3]),
                                            (2**63 + 5, 33, 8, None), (9, 4, 3, [0.0, 0.0, 1.0])])
def test_delay_table_matches_oracle(lib, seed, P, L, probs):
    cfg = adg.Config(K=P * 4, p=1, P=P, L=L, mode="async", seed=seed, probs=probs)
    got = adg.delay_table(cfg, 100, 60)
    ref = odelays.delay_table(seed, P, 60, L, probs, first_step=100)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("sync,L,first", [(2, 3, 0), (2, 3, 1001), (1, 8, 37), (5, 1, 12)])
def test_caa_cycle_matches_oracle(lib, sync, L, first):
    # The communication-avoiding cycle of Section 6.3 as the library's delay source.
    P = 6
    cfg = adg.Config(K=P * 4, p=1, P=P, L=L, mode="at", caa_sync=sync, seed=77)
    got = adg.delay_table(cfg, first, 40)
    assert np.array_equal(got, odelays.caa_table(P, 40, sync, L, first_step=first))


def test_viscosity_settings_rejected(lib):
    for kw in (dict(pde="advection", nu=0.1), dict(pde="burgers", nu=-1.0),
               dict(pde="burgers", nu=float("nan"))):
        cfg = adg.Config(K=8, p=1, P=2, L=2, mode="async", **kw)
        with pytest.raises(adg.AdgError) as ei:
            adg.delay_table(cfg, 0, 4)
        assert ei.value.code == _abi.ADG_EINVAL


def test_euler_settings_rejected(lib):
    for kw in (dict(dt=0.0), dict(dt=1e-6, rk="lsrk4"), dict(dt=1e-6, tvb_m=-1.0)):
        cfg = adg.Config(pde="euler", K=8, p=1, P=2, L=2, mode="async", **kw)
        with pytest.raises(adg.AdgError) as ei:
            adg.delay_table(cfg, 0, 4)
        assert ei.value.code == _abi.ADG_EINVAL


def test_caa_rejects_bad_settings(lib):
    tbl = np.zeros((2, 2), dtype=np.uint8)
    for kw in (dict(caa_sync=-1), dict(caa_sync=65), dict(caa_sync=2, table=tbl)):
        cfg = adg.Config(K=8, p=1, P=2, L=3, mode="async", **kw)
        with pytest.raises(adg.AdgError) as ei:
            adg.delay_table(cfg, 0, 4)
        assert ei.value.code == _abi.ADG_EINVAL


def test_caller_table_is_periodic(lib):
    tbl = np.array([[0, 1], [2, 0], [1, 1]], dtype=np.uint8)
    cfg = adg.Config(K=8, p=1, P=2, L=3, mode="async", table=tbl)
    got = adg.delay_table(cfg, 4, 6)
    assert np.array_equal(got, tbl[[(4 + r) % 3 for r in range(6)]])


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lgl_nodes_match_oracle(lib, p):
    x, w = adg.lgl_nodes(p)
    xo, wo = lgl_nodes_weights(p)
    assert np.max(np.abs(x - xo)) < 1e-15 and np.max(np.abs(w - wo)) < 1e-15


def test_init_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cfg = adg.Config(K=16, p=2, P=4)
    c, keep = cfg.to_c()
    ctx = C.c_void_p()
    assert lib.adg_init(C.byref(c), C.c_void_p(8), None, C.byref(ctx)) == _abi.ADG_ECUDA
    assert b"CUDA" in lib.adg_last_error(None) or b"device" in lib.adg_last_error(None)
    # from host buffers too: no CPU fallback
    host = np.zeros((16, 3))
    assert lib.adg_init_host(C.byref(c), host.ctypes.data, None, C.byref(ctx)) == _abi.ADG_ECUDA
    assert not ctx.value
