"""GPU parity of batched runs: many independent instances of uneven size, degree, speed and
delay statistics advanced by the same stage launches (one work list over all instances),
checked per instance against the oracle and, bit for bit, against single-instance runs."""
import math

import numpy as np
import pytest
import torch

import paper_2404_03399_gb300 as adg
from oracle import dg, delays as odelays
from workloads import Modes, batched_instances

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_03399_gb300 import build
    build.build()


def _cfg(w, mode=None, variant="auto"):
    return adg.Config(pde="advection", K=w.K, p=w.p, P=w.P, a=w.a, cfl=w.cfl,
                      mode=mode or w.mode, L=w.L, q=w.q, seed=w.seed, variant=variant)


def _small_batch():
    rng = np.random.default_rng(3)
    ws = []
    spec = [(300, 1, 3, 0.7, "at", 3), (1024, 2, 8, 1.3, "async", 4), (777, 3, 7, -0.9, "at", 5),
            (512, 4, 4, 1.9, "sync", 2), (2048, 3, 16, 0.5, "at", 8), (96, 2, 96, 1.0, "at", 3),
            (1000, 4, 1, 1.1, "at", 3), (4096, 1, 32, 1.6, "at", 2)]
    for i, (K, p, P, a, mode, L) in enumerate(spec):
        modes = Modes(amp=tuple(rng.uniform(0.25, 1.0, 4)), kappa=tuple(float(k) for k in rng.integers(1, 9, 4)),
                      phase=tuple(rng.uniform(0, 2 * math.pi, 4)))
        from workloads import Workload
        ws.append(Workload(name=f"s{i}", pde="advection", K=K, p=p, P=P, modes=modes, a=a, cfl=0.002,
                           mode=mode, L=L, q=min(p + 1, 3), seed=int(rng.integers(0, 2**62))))
    return ws


def _eligible_batch():
    # every instance admits the composed step (a > 0, K/P >= 8): the batch runs it
    rng = np.random.default_rng(5)
    from workloads import Workload
    ws = []
    for i, (K, p, P, a, L) in enumerate([(512, 1, 8, 0.7, 3), (2048, 4, 16, 1.9, 5), (777 * 8, 3, 8, 1.1, 8),
                                          (1024, 2, 1, 1.3, 2), (4096, 3, 64, 0.5, 4)]):
        modes = Modes(amp=tuple(rng.uniform(0.25, 1.0, 3)), kappa=tuple(float(k) for k in rng.integers(1, 9, 3)),
                      phase=tuple(rng.uniform(0, 2 * math.pi, 3)))
        ws.append(Workload(name=f"c{i}", pde="advection", K=K, p=p, P=P, modes=modes, a=a, cfl=0.002,
                           mode="at", L=L, q=min(p + 1, 3), seed=int(rng.integers(0, 2**62))))
    return ws


def _check_single(got, single, i):
    """A batched instance against its single-instance run: bit-identical (both keep the same
    coordinates, the block basis of the element operator for fixed point)."""
    assert np.array_equal(got, single), f"instance {i} differs from its single run"


@pytest.mark.parametrize("kind,variant,single_variant", [
    ("mixed", "auto", "staged"),        # some instances admit no composed step: all staged
    ("eligible", "composed", "composed"),
    ("eligible", "auto", "fixed"),      # every instance admits the fixed-point step
])
def test_small_batch_matches_oracle_and_single_runs(kind, variant, single_variant):
    ws = _small_batch() if kind == "mixed" else _eligible_batch()
    steps = 70
    cfgs = [_cfg(w, variant=variant) for w in ws]
    u0s = [adg.eval_modes(c, w.modes.amp, w.modes.kappa, w.modes.phase) for c, w in zip(cfgs, ws)]
    b = adg.BatchSolver(cfgs, u0s)
    assert all(b.variant(i)[0] == single_variant for i in range(len(ws)))
    b.step(steps)
    for i, (c, w) in enumerate(zip(cfgs, ws)):
        got = b.state(i).cpu().numpy()
        cs = adg.Config(**{**c.__dict__, "variant": single_variant})
        s = adg.Solver(cs, u0s[i])
        s.step(steps)
        single = s.state().cpu().numpy()
        dt = s.dt
        s.close()
        _check_single(got, single, i)
        q = w.q if w.mode == "at" else 1
        tbl = odelays.delay_table(w.seed, w.P, steps, w.L) if (w.mode != "sync" and w.P > 1) else None
        prob = dg.Problem(pde="advection", K=w.K, p=w.p, P=w.P, dt=dt, a=w.a,
                          mode="adg" if tbl is not None else "sync", q=q, delays=tbl)
        ref = dg.run(prob, u0s[i].cpu().numpy(), steps).numpy()
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err < TOL, (i, err)
    b.close()


def test_full_batch_sampled():
    # The 512-instance batched workload, 40 steps (one graph chunk and a remainder), checked
    # at sampled elements of sampled instances against the oracle on a window.
    ws = batched_instances()
    steps = 40
    cfgs = [_cfg(w) for w in ws]
    u0s = [adg.eval_modes(c, w.modes.amp, w.modes.kappa, w.modes.phase) for c, w in zip(cfgs, ws)]
    b = adg.BatchSolver(cfgs, u0s)
    b.step(steps)
    b.check_finite()
    rng = np.random.default_rng(1)
    for i in [int(v) for v in rng.choice(len(ws), 6, replace=False)] + [0, len(ws) - 1]:
        w = ws[i]
        got = b.state(i).cpu().numpy()
        u0 = u0s[i].cpu().numpy()
        dt = b.dt(i)
        tbl = odelays.delay_table(w.seed, w.P, steps, w.L)
        for e in [0, w.K // w.P, int(rng.integers(0, w.K)), w.K - 1]:
            r = 3 * steps + 2
            lo = e - r if w.a >= 0 else e - 2
            W = r + 3
            idx = np.arange(lo, lo + W) % w.K
            prob = dg.Problem(pde="advection", K=W, p=w.p, P=w.P, dt=dt, a=w.a, mode="adg", q=w.q,
                              delays=tbl, window_lo=lo, K_global=w.K)
            ref = dg.run(prob, u0[idx], steps).numpy()[e - lo]
            err = np.max(np.abs(got[e] - ref)) / np.max(np.abs(got))
            assert err < TOL, (i, e, err)
    b.close()


def test_batch_of_fixed_point_steps_in_calls_of_one_and_two():
    # single-step calls take the FP64 path of the fixed-point step; two-step calls run one
    # FP64 -> int64 and one int64 -> FP64 step; both stay on the oracle
    ws = _eligible_batch()
    cfgs = [_cfg(w) for w in ws]
    u0s = [adg.eval_modes(c, w.modes.amp, w.modes.kappa, w.modes.phase) for c, w in zip(cfgs, ws)]
    b = adg.BatchSolver(cfgs, u0s)
    for k in (1, 2, 1, 2, 3):
        b.step(k)
    steps = 9
    for i, (c, w) in enumerate(zip(cfgs, ws)):
        got = b.state(i).cpu().numpy()
        tbl = odelays.delay_table(w.seed, w.P, steps, w.L) if w.P > 1 else None
        prob = dg.Problem(pde="advection", K=w.K, p=w.p, P=w.P, dt=b.dt(i), a=w.a,
                          mode="adg" if tbl is not None else "sync", q=w.q, delays=tbl)
        ref = dg.run(prob, u0s[i].cpu().numpy(), steps).numpy()
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < TOL, i
    b.close()


def test_fixed_point_batch_with_different_coefficients_per_degree():
    # Two Courant numbers among instances of the same degree: the coefficients differ, so the
    # batch reads each instance's own coefficients (the general batched kernel) instead of one
    # set per degree; every instance still equals its single-instance fixed-point run.
    ws = _eligible_batch()
    cfgs = [adg.Config(pde="advection", K=w.K, p=w.p, P=w.P, a=w.a, cfl=0.002 + 0.001 * (i % 2),
                       mode=w.mode, L=w.L, q=w.q, seed=w.seed) for i, w in enumerate(ws)]
    u0s = [adg.eval_modes(c, w.modes.amp, w.modes.kappa, w.modes.phase) for c, w in zip(cfgs, ws)]
    b = adg.BatchSolver(cfgs, u0s)
    assert all(b.variant(i)[0] == "fixed" for i in range(len(ws)))
    b.step(40)
    for i, c in enumerate(cfgs):
        s = adg.Solver(adg.Config(**{**c.__dict__, "variant": "fixed"}), u0s[i])
        s.step(40)
        _check_single(b.state(i).cpu().numpy(), s.state().cpu().numpy(), i)
        s.close()
    b.close()


def _tuned_batch_workloads():
    # 28 instances of the batched workload's distribution, about 1.1 M elements: above the
    # size at which the batch autotuner times its choices
    return batched_instances(n=28, seed=7)


def test_batch_autotuner_choice_and_forced_choices_agree():
    # AUTO: the tuner times fixed point (256-, 512- and 1024-element work items), the FP64
    # composed step and the staged kernels and keeps the fastest; every forced choice runs the
    # same scheme. The fixed-point choices are bit-identical to each other and to the
    # single-instance fixed-point run; every choice stays on the oracle.
    ws = _tuned_batch_workloads()
    assert sum(w.K for w in ws) >= 1 << 20
    steps = 12
    cfgs = [_cfg(w) for w in ws]
    u0s = [adg.eval_modes(c, w.modes.amp, w.modes.kappa, w.modes.phase) for c, w in zip(cfgs, ws)]
    states = {}
    for variant, ept in [("auto", 0), ("fixed", 1), ("fixed", 2), ("fixed", 4), ("composed", 0),
                         ("staged", 0)]:
        cs = [adg.Config(**{**c.__dict__, "variant": variant, "ept": ept}) for c in cfgs]
        b = adg.BatchSolver(cs, u0s)
        kinds = {b.variant(i) for i in range(len(ws))}
        assert len(kinds) == 1, kinds
        kind, e = kinds.pop()
        if variant != "auto":
            assert kind == variant and (ept == 0 or e == ept), (variant, ept, kind, e)
        b.step(steps)
        states[(variant, ept)] = ([b.state(i).cpu().numpy() for i in (0, 5, 27)], kind)
        b.close()
    base = states[("fixed", 2)][0]
    for ept in (1, 4):
        for a, c in zip(states[("fixed", ept)][0], base):
            assert np.array_equal(a, c)
    auto_states, auto_kind = states[("auto", 0)]
    ref_states = states[{"fixed": ("fixed", 2), "composed": ("composed", 0),
                         "staged": ("staged", 0)}[auto_kind]][0]
    for a, c in zip(auto_states, ref_states):
        assert np.array_equal(a, c)
    for k, i in enumerate((0, 5, 27)):
        w = ws[i]
        s = adg.Solver(adg.Config(**{**cfgs[i].__dict__, "variant": "fixed"}), u0s[i])
        s.step(steps)
        single = s.state().cpu().numpy()
        dt = s.dt
        s.close()
        _check_single(base[k], single, i)
        tbl = odelays.delay_table(w.seed, w.P, steps, w.L)
        prob = dg.Problem(pde="advection", K=w.K, p=w.p, P=w.P, dt=dt, a=w.a, mode="adg", q=w.q,
                          delays=tbl)
        ref = dg.run(prob, u0s[i].cpu().numpy(), steps).numpy()
        for (variant, ept), (sts, _) in states.items():
            err = np.max(np.abs(sts[k] - ref)) / np.max(np.abs(ref))
            assert err < TOL, (variant, ept, i, err)


def test_batch_rejects_conflicting_forced_choices():
    ws = _eligible_batch()[:2]
    cfgs = [_cfg(w) for w in ws]
    u0s = [adg.eval_modes(c, w.modes.amp, w.modes.kappa, w.modes.phase) for c, w in zip(cfgs, ws)]
    bad = [adg.Config(**{**cfgs[0].__dict__, "variant": "staged"}),
           adg.Config(**{**cfgs[1].__dict__, "variant": "composed"})]
    with pytest.raises(adg.AdgError) as ei:
        adg.BatchSolver(bad, u0s)
    assert ei.value.code == adg._abi.ADG_EINVAL
    bad = [adg.Config(**{**c.__dict__, "variant": "staged", "ept": 2}) for c in cfgs]
    with pytest.raises(adg.AdgError) as ei:
        adg.BatchSolver(bad, u0s)
    assert ei.value.code == adg._abi.ADG_EINVAL
