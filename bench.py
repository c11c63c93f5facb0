"""Benchmark of the ADG-AT SSP-RK3 step on GB300.

One "step" is one full SSP-RK3 step of ADG-AT over the whole mesh of the large advection
workload (K = 2^24 elements, p = 3, 2^26 DOF in FP64, 16384 PEs, delays uniform in
{0..7}, AT order 3, ring of L+q-1 = 10 levels). The metric is DOF-stage updates per second
(K (p+1) x 3 stages per step). The same line carries the synchronous-DG throughput on the
same mesh, the roofline of the stage kernel, the oracle timed on the host cores, clocks
sampled during the timed region and an end-to-end figure through the C ABI from host
buffers.

Multi-GPU (torchrun, one rank per GPU): the mesh does not shard without a face exchange,
so each rank advances its own replica of the workload (weak scaling, no collective on the
data path); value = all ranks' DOF-stage updates / max over ranks of the timed region.

    python bench.py [--steps 500] [--warmup 5] [--gpus N] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ADG-AT DOF-stage updates/s and % HBM roofline vs sync DG; adjoint/forward cost"
UNIT = "DOF-stage updates/s"
STAGES = 3
# The large advection workload; its Courant number is not fixed by the workload statement
# and is set inside the stability bound of the delayed self-feedback (sigma (p+1)^2 k < 1
# for k <= 7 with the AT extrapolation); the work per step does not depend on it.
from workloads import (ADJOINT_64K as _WADJ, ADVECTION_16M as _W16M, ADVECTION_SMALL,  # noqa: E402
                       BURGERS_1M, batched_instances)

WORKLOAD = dict(name=_W16M.name, pde=_W16M.pde, K=_W16M.K, p=_W16M.p, P=_W16M.P, L=_W16M.L,
                q=_W16M.q, cfl=_W16M.cfl, seed=_W16M.seed,
                modes=(list(_W16M.modes.amp), list(_W16M.modes.kappa), list(_W16M.modes.phase),
                       _W16M.modes.offset))
# Algorithmic work of the kernels that can run the bench step (the composed SSP-RK3 step of
# upwind advection, Np^2 + 5 Np + 3 multiply-adds per element and step in nodal values):
#  - fixed-point integer step (picked where the coefficients fit, as here): each
#    multiply-add is three 32 x 32 -> 64-bit integer products; the bound is the integer
#    multiply pipe (counts below);
#  - FP64 composed step: 2 (Np^2 + 5 Np + 3) / Np flop per DOF-step (19.5 at p = 3);
#  - staged FP64 kernels: 2 (Np + 2) flop per DOF-stage.
NP = WORKLOAD["p"] + 1
MACS_PER_ELEMENT_STEP = NP * NP + 5 * NP + 3
# fixed point: each multiply-add of the kernel is three 32 x 32 -> 64-bit products
# (adg_fixed.cuh); with two elements per thread the kernel forms Np^2 + 5 Np + 3.5 of them per
# element (the neighbour's channel scalars: 7 per pair instead of 8), and in the block basis
# of the element operator (2 x 2 blocks of G whose first rows are shifts and adds)
# 2 floor(Np / 2) + (Np odd) + 5 Np + 3.5 (27.5 at p = 3)
FIXED_MACS_PER_ELEMENT_STEP = MACS_PER_ELEMENT_STEP + 0.5
FIXED_MACS_PER_ELEMENT_STEP_BASIS = 2 * (NP // 2) + (NP % 2) + 5 * NP + 3.5
FLOP_PER_DOF_STEP = 2 * MACS_PER_ELEMENT_STEP / NP
FLOP_PER_DOF_STAGE_STAGED = 2 * (NP + 2)
# A 2N low-storage stage: dt L(U) + A_s dU (one multiply and NP + 1 FMA per DOF) and
# U_s = U_{s-1} + B_s dU_s (one FMA).
FLOP_PER_DOF_STAGE_LS = 2 * (NP + 2) + 1
LOW_STORAGE_STAGES = {"rk1": 1, "rk2": 2, "lsrk3": 3, "lsrk4": 5}
# Viscous Burgers (LDG), per DOF and stage, counted from the two kernels' multiplies and FMAs:
# the q pass 2 Np + 3, the stage (Lax-Friedrichs part and viscous part) 4 Np + 14.
VISC_NP = 3
FLOP_PER_DOF_STAGE_VISC = 6 * VISC_NP + 17
# DRAM bytes per launch measured by ncu on this workload (read + write) for the kernel that
# dominates the step, keyed by variant, elements per thread and coordinates; a kernel changed
# since its counters were taken has no entry (null in the line). k_step_fixed, two per thread,
# int64 -> int64, K = 2^24 (the algorithmic 536,870,912 B each way; part of the written field
# is still in L2 when the launch ends): nodal values 537,010,176 B read + 488,685,824 B
# written; block-basis coordinates 536,897,536 + 487,339,520 B.
TRAFFIC_BYTES_PER_LAUNCH = {"fixed/2/nodal": 537010176 + 488685824,
                            "fixed/2/basis": 536897536 + 487339520}
# Algorithmic HBM bytes: read u^n, write u^{n+1} once per step: 16 B per DOF-step.
BYTES_PER_DOF_STEP = 16
# The staged SSP-RK3 step reads and writes 16 / 24 / 24 B per DOF in its three stages (the
# Burgers workload's 42 MB fields are largely L2-resident, so its fraction of HBM is a bound
# on traffic, not a measure of it).
BYTES_PER_DOF_STEP_STAGED = 64
# Burgers LLF stage at p = 4 (Np = 5): per node v^2 (one multiply), Np FMA of the volume row,
# two lifts and the alpha / beta combination: 2 (Np + 4) + 1 flop per DOF-stage.
FLOP_PER_DOF_STAGE_BURGERS = 2 * (5 + 4) + 1
# steps per directly launched chunk on the large mesh (adg_step)
CHUNK_STEPS = 256


def sm_count() -> int:
    """Streaming multiprocessors of the current device (152 on GB300), read from the device."""
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def peaks():
    """Roofline denominators: HBM from MEASURED_PEAKS.json (else the recipe's fallback); FP64
    ALU peak from unit counts: SMs (read from the device) x 2 DFMA/clk x 2 flop x the maximum SM
    clock (the nominal 1.26 TFLOP/s FP64 of GB300 at 152 SMs and 2.07 GHz)."""
    hbm, src = 6800.0, "fallback"
    sm_mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mp = json.load(f)
        hbm, src = float(mp["hbm_gbs"]), "measured"
        sm_mhz = float(mp.get("sm_max_mhz", sm_mhz))
    except Exception:
        pass
    sms = sm_count()
    fp64_tflops = sms * 2 * 2 * sm_mhz * 1e6 / 1e12
    return hbm, src, fp64_tflops, sms, sm_mhz


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [t.strip() for t in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v == "Active"})
        loaded = [r[0] for r in rows if r[2] > 200.0] or [r[0] for r in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


def make_cfg(mode: str, rk: str = "ssprk3", variant: str = "auto"):
    import paper_2404_03399_gb300 as adg
    w = WORKLOAD
    return adg.Config(pde=w["pde"], K=w["K"], p=w["p"], P=w["P"], cfl=w["cfl"], mode=mode,
                      L=w["L"], q=w["q"] if mode == "at" else 0, seed=w["seed"], rk=rk,
                      variant=variant)


def bench_config(ws: int) -> dict:
    """The workload of the line, the same for both arms."""
    w = WORKLOAD
    return {"workload": w["name"], "K": w["K"], "p": w["p"], "P": w["P"], "L": w["L"],
            "at_order": w["q"], "cfl": w["cfl"], "dof": w["K"] * (w["p"] + 1),
            "parallelism": f"replicas x{ws}",
            "l2": "inputs larger than L2 (537 MB per nodal field)"}


def host_info() -> dict:
    """Host cores and CPU model (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    try:
        avail = len(os.sched_getaffinity(0))
    except Exception:
        avail = os.cpu_count()
    return {"host_cores": os.cpu_count(), "cores_available": avail, "cpu_model": model}


def device_timed(mode: str, steps: int, warmup: int, dist_barrier, sample_clocks: bool, dev: int,
                 rk: str = "ssprk3", variant: str = "auto", exact_error: dict = None):
    import torch
    import paper_2404_03399_gb300 as adg
    cfg = make_cfg(mode, rk, variant)
    amp, kap, ph, off = WORKLOAD["modes"]
    u0 = adg.eval_modes(cfg, amp, kap, ph, off)
    s = adg.Solver(cfg, u0)
    del u0
    stream = torch.cuda.current_stream()
    # the sampler starts before the warm-up steps (and runs until after the timed ones), so
    # that its start-up and the pause for its first sample fall outside the timed region
    clocks = ClockSampler(dev) if sample_clocks else None
    if clocks:
        clocks.__enter__()
    s.step(warmup)
    torch.cuda.synchronize()
    dist_barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s.step(steps)
    ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize()
    dist_barrier()
    if clocks:
        clocks.__exit__(None, None, None)
    ms = ev0.elapsed_time(ev1)
    s.check_finite_ok = True
    try:
        s.check_finite()
    except adg.AdgError:
        s.check_finite_ok = False
    finite = s.check_finite_ok
    variant = s.variant + (s.fixed_basis,)
    if exact_error is not None:
        exact_error.update(linf_vs_translation(s, cfg, warmup + steps))
    s.close()
    return ms, (clocks.summary() if clocks else None), finite, variant


def linf_vs_translation(s, cfg, nsteps: int) -> dict:
    """Max-norm error of the solver's state against the exact solution of linear advection,
    u0(x - a t) at t = nsteps dt, evaluated at the library's nodes (relative to max |u_exact|)."""
    import paper_2404_03399_gb300 as adg
    amp, kap, ph, off = WORKLOAD["modes"]
    t = nsteps * s.dt
    exact = adg.eval_modes(cfg, amp, kap, [f - k * cfg.a * t for f, k in zip(ph, kap)], off)
    u = s.state()
    err = float((u - exact).abs().max() / exact.abs().max())
    del exact, u
    return {"linf_rel": err, "t": t, "steps": nsteps}


def burgers_timed(steps: int, warmup: int, mode: str, cfl: float):
    """The Burgers workload (K = 2^20, p = 4, LLF, 1024 PEs, delays uniform in {0..3}, AT
    order 2 for mode "at") at Courant number cfl: CUDA-event time of `steps` steps after
    `warmup`, finiteness, and the max-norm error against the exact pre-shock solution
    u = u0(x - u t) (characteristics, Newton per node) after all steps."""
    import numpy as np
    import torch
    import paper_2404_03399_gb300 as adg
    w = BURGERS_1M
    cfg = adg.Config(pde="burgers", K=w.K, p=w.p, P=w.P, cfl=cfl, mode=mode, L=w.L,
                     q=w.q if mode == "at" else 0, seed=w.seed)
    m = w.modes
    u0 = adg.eval_modes(cfg, m.amp, m.kappa, m.phase, m.offset)
    s = adg.Solver(cfg, u0)
    del u0
    stream = torch.cuda.current_stream()
    s.step(warmup)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s.step(steps)
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    fin = True
    try:
        s.check_finite()
    except adg.AdgError:
        fin = False
    variant = s.variant[0]
    t = (warmup + steps) * s.dt
    u = s.state()
    s.close()
    xi, _ = adg.lgl_nodes(w.p)
    dx = (cfg.x1 - cfg.x0) / w.K
    x = cfg.x0 + (torch.arange(w.K, dtype=torch.float64, device="cuda")[:, None]
                  + (1.0 + torch.tensor(xi, device="cuda"))[None, :] / 2.0) * dx
    ex = m.offset + m.amp[0] * torch.sin(m.kappa[0] * x + m.phase[0])
    for _ in range(30):   # u = u0(x - u t): Newton on g(u) = u - u0(x - u t)
        arg = m.kappa[0] * (x - ex * t) + m.phase[0]
        g = ex - (m.offset + m.amp[0] * torch.sin(arg))
        ex = ex - g / (1.0 + m.amp[0] * m.kappa[0] * t * torch.cos(arg))
    err = float((u - ex).abs().max() / ex.abs().max()) if fin else float("nan")
    return ms, fin, variant, {"linf_rel": err, "t": t, "steps": warmup + steps}


def caa_timed(steps: int, warmup: int):
    """The large advection mesh under the communication-avoiding delay cycle of Section 6.3
    (L = 3, two synchronised steps of five, ADG-AT2): CUDA-event time of `steps` steps after
    `warmup`, and the PE-face exchanges a distributed run would make (adg_comm_stats)."""
    import torch
    import paper_2404_03399_gb300 as adg
    w = WORKLOAD
    cfg = adg.Config(pde=w["pde"], K=w["K"], p=w["p"], P=w["P"], cfl=w["cfl"], mode="at", L=3,
                     q=2, caa_sync=2)
    amp, kap, ph, off = w["modes"]
    u0 = adg.eval_modes(cfg, amp, kap, ph, off)
    s = adg.Solver(cfg, u0)
    del u0
    stream = torch.cuda.current_stream()
    s.step(warmup)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s.step(steps)
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    st = s.comm_stats()
    variant = s.variant[0]
    s.close()
    return ms, st, variant


def viscous_timed(steps: int, warmup: int):
    """ALDG(2)-AT2-RK2 of Section 6's viscous Burgers experiment (nu = 0.1, the multi-scale
    initial condition, L = 3 with probabilities 0.3 / 0.4 / 0.3) on 2^20 elements and 1024
    PEs, dt = 0.01 dx^2: CUDA-event time of `steps` steps after `warmup`."""
    import torch
    import paper_2404_03399_gb300 as adg
    K = 1 << 20
    dx = 2 * math.pi / K
    cfg = adg.Config(pde="burgers", K=K, p=VISC_NP - 1, P=1024, dt=0.01 * dx * dx, nu=0.1,
                     mode="at", L=3, q=2, probs=[0.3, 0.4, 0.3], seed=5, rk="rk2")
    u0 = adg.eval_modes(cfg, [3.0, 2.0, 1.0], [2.0, 3.0, 5.0], [0.3, 1.1, 2.0])
    s = adg.Solver(cfg, u0)
    del u0
    stream = torch.cuda.current_stream()
    s.step(warmup)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s.step(steps)
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    s.check_finite_ok = True
    try:
        s.check_finite()
    except adg.AdgError:
        s.check_finite_ok = False
    fin = s.check_finite_ok
    s.close()
    return ms, K * VISC_NP, fin


def euler_timed(steps: int, warmup: int):
    """ADG(1)-AT2-RK2 with the limiter for the one-dimensional Euler equations (Section 6's
    Sod experiment, two Riemann problems on [0, 0.02]) on 2^20 elements and 1024 PEs, L = 3
    with probabilities 0.3 / 0.4 / 0.3, dt = 0.1 dx: CUDA-event time of `steps` steps."""
    import numpy as np
    import torch
    import paper_2404_03399_gb300 as adg
    K, p = 1 << 20, 1
    dx = 0.02 / K
    cfg = adg.Config(pde="euler", K=K, p=p, P=1024, x0=0.0, x1=0.02, dt=0.1 * dx, rk="rk2",
                     mode="at", L=3, q=2, probs=[0.3, 0.4, 0.3], seed=3, limiter=True)
    xi, _ = adg.lgl_nodes(p)
    x = (np.arange(K)[:, None] + (1.0 + np.asarray(xi)[None, :]) / 2.0) * dx
    inner = (x >= 0.005) & (x < 0.015)
    rho = np.where(inner, 1.0, 0.125)
    pr = np.where(inner, 1.0, 0.1)
    U0 = torch.tensor(np.stack([rho, 0.0 * rho, pr / 0.4]), device="cuda")
    s = adg.Solver(cfg, U0)
    del U0
    stream = torch.cuda.current_stream()
    s.step(warmup)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    s.step(steps)
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    fin = True
    try:
        s.check_finite()
    except adg.AdgError:
        fin = False
    s.close()
    return ms, K * (p + 1), fin


def e2e_timed(steps: int):
    """Public-API run from host buffers: `adg_init_host` on pinned u0 (the layout kernel reads
    it over the host link), `steps` steps, `adg_get_state_host` into pinned memory (written by
    the layout kernel over the link); all inside one timed region (wall clock around
    synchronised work, bracketed by CUDA events on the same stream)."""
    import torch
    import paper_2404_03399_gb300 as adg
    cfg = make_cfg("at")
    amp, kap, ph, off = WORKLOAD["modes"]
    host_u0 = adg.eval_modes(cfg, amp, kap, ph, off).cpu().pin_memory()
    host_out = torch.empty_like(host_u0).pin_memory()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    ev0.record(stream)
    s = adg.Solver(cfg, host_u0)
    s.step(steps)
    s.state(out=host_out)
    ev1.record(stream)
    ev1.synchronize()
    wall = time.perf_counter() - t0
    s.close()
    nbytes = host_u0.numel() * 8
    return max(wall * 1e3, ev0.elapsed_time(ev1)), nbytes


def batched_timed(steps: int, warmup: int):
    """The 512-instance batched workload (uneven K, p, a, L, seeds) advanced by one work
    list per stage; returns (DOF-stage updates/s, ms per step, total DOF, instances)."""
    import torch
    import paper_2404_03399_gb300 as adg
    ws = batched_instances()
    cfgs = [adg.Config(pde="advection", K=w.K, p=w.p, P=w.P, a=w.a, cfl=w.cfl, mode=w.mode,
                       L=w.L, q=w.q, seed=w.seed) for w in ws]
    u0s = [adg.eval_modes(c, w.modes.amp, w.modes.kappa, w.modes.phase) for c, w in zip(cfgs, ws)]
    b = adg.BatchSolver(cfgs, u0s)
    del u0s
    ndof = sum(w.K * (w.p + 1) for w in ws)
    stream = torch.cuda.current_stream()
    b.step(warmup)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    b.step(steps)
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    b.check_finite()
    variant = "%s, %d element(s) per thread" % b.variant(0)
    b.close()
    return ndof * STAGES * steps / (ms * 1e-3), ms / steps, ndof, len(ws), variant


def adjoint_cost(steps: int = 0, repeats: int = 3):
    """Gradient / forward cost on the adjoint workload (Burgers, K = 65536, p = 3, 1024 PEs,
    delays in {0..3}, AT order 2, 2000 steps, checkpoints every 50): CUDA-event time of
    adg_grad against the same forward steps."""
    import math as _m
    import torch
    import paper_2404_03399_gb300 as adg
    w = _WADJ
    cfg = adg.Config(pde="burgers", K=w.K, p=w.p, P=w.P, L=w.L, q=w.q, mode="at", cfl=w.cfl,
                     seed=w.seed)
    u0 = adg.eval_modes(cfg, w.modes.amp, w.modes.kappa, w.modes.phase, w.modes.offset)
    g = adg.eval_modes(cfg, [1.0], [1.0], [-0.003], 0.5)
    stream = torch.cuda.current_stream()

    def timed(fn):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        fn()
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1)

    nsteps = steps or w.steps
    fwd, grd = [], []
    for _ in range(repeats):
        s = adg.Solver(cfg, u0)
        fwd.append(timed(lambda: s.step(nsteps)))
        s.close()
        s = adg.Solver(cfg, u0)
        grd.append(timed(lambda: s.grad(g, nsteps, 50)))
        s.close()
    f, gms = min(fwd), min(grd)
    return {"forward_ms": f, "grad_ms": gms, "grad_over_forward": gms / f, "steps": nsteps,
            "ckpt_every": 50, "workload": "Burgers K=65536 p=3 1024 PEs L=4 AT2, 2000 steps"}


def oracle_timed(window: int, steps: int, warmup: int = 1, threads: int = 0):
    """The FP64 oracle as it stands, on the host cores: `warmup` untimed and then `steps` timed
    SSP-RK3 steps of ADG-AT on a contiguous window of `window` elements of the large mesh (the
    whole mesh when window = K; its PE faces and delays included). threads > 0 runs torch's
    CPU ops on that many threads. Returns (DOF-stage updates/s, ms per timed step, threads
    used, sample description)."""
    import numpy as np
    import torch
    from oracle import dg, delays
    w = WORKLOAD
    K, p = w["K"], w["p"]
    dx = 2 * math.pi / K
    dt = (w["cfl"] * dx) / 1.0
    old_threads = torch.get_num_threads()
    if threads > 0:
        torch.set_num_threads(threads)
    try:
        used = torch.get_num_threads()
        tbl = delays.delay_table(w["seed"], w["P"], steps + warmup + 2, w["L"])
        x = dg.node_coordinates(window, p, 0.0, 2 * math.pi, 0, K)
        u0 = np.sin(x)
        full = window == K
        prob = dg.Problem(pde="advection", K=window, p=p, P=w["P"], dt=dt, mode="adg", q=w["q"],
                          delays=tbl, window_lo=None if full else 0, K_global=None if full else K)
        s = dg.Solver(prob, u0)
        for _ in range(max(warmup, 1)):
            s.step()
        t0 = time.perf_counter()
        for _ in range(steps):
            s.step()
        el = time.perf_counter() - t0
    finally:
        torch.set_num_threads(old_threads)
    rate = window * (p + 1) * STAGES * steps / el
    where = "the whole K=2^24 mesh" if window == K else \
        f"a {window}-element window ({window // (K // w['P'])} PE faces) of the K=2^24 mesh"
    sample = f"{steps} timed SSP-RK3 steps (after {max(warmup, 1)} untimed) of the oracle on {where}"
    return rate, el / steps * 1e3, used, sample


def small_timed(mode: str) -> dict:
    """The small advection workload (K = 64, p = 2, 16 PEs, delays uniform in {0..3}, sigma =
    0.1, t_end = 2 pi: 640 steps) on the GPU: CUDA-event time of the whole run after one
    untimed run. Latency-bound (192 DOF): a measure of per-step overhead, not of throughput."""
    import torch
    import paper_2404_03399_gb300 as adg
    w = ADVECTION_SMALL
    cfg = adg.Config(pde="advection", K=w.K, p=w.p, P=w.P, cfl=w.cfl, mode=mode, L=w.L,
                     q=w.q if mode == "at" else 0, seed=w.seed)
    m = w.modes
    u0 = adg.eval_modes(cfg, m.amp, m.kappa, m.phase, m.offset)
    stream = torch.cuda.current_stream()
    for rep in range(2):
        s = adg.Solver(cfg, u0)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        s.run(w.t_end)
        ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1)
        s.state()
        n = s.n
        variant = s.variant[0]
        s.close()
    ndof = w.K * (w.p + 1)
    return {"value": ndof * STAGES * n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / n,
            "steps": n, "variant": variant}


def oracle_configs() -> dict:
    """The oracle on samples of every workload, with all of torch's CPU threads and with one:
    the small advection workload (all 640 steps, ADG-AT3), the Burgers workload (2 steps on a
    2^18-element window), the batched workload (2 steps of its first 8 instances), and the
    adjoint workload's gradient / forward cost (10 steps of the oracle's automatic-
    differentiation adjoint on the full K = 65536 mesh)."""
    import numpy as np
    import torch
    from oracle import dg, delays
    out = {}

    def rate_of(fn, units):
        t0 = time.perf_counter()
        fn()
        return units / (time.perf_counter() - t0)

    def both(fn, units):
        old = torch.get_num_threads()
        r_all = rate_of(fn, units)
        torch.set_num_threads(1)
        try:
            r_one = rate_of(fn, units)
        finally:
            torch.set_num_threads(old)
        return {"all_threads": r_all, "one_thread": r_one, "threads": old}

    w = ADVECTION_SMALL
    dx = 2 * math.pi / w.K
    nsmall = math.ceil(w.t_end / (w.cfl * dx))
    tbl = delays.delay_table(w.seed, w.P, nsmall, w.L)
    prob = dg.Problem(pde="advection", K=w.K, p=w.p, P=w.P, dt=w.t_end / nsmall, mode="adg",
                      q=w.q, delays=tbl)
    u0 = dg.modes_initial(w.modes, w.K, w.p)
    out["advection_small"] = both(lambda: dg.run(prob, u0, nsmall),
                                  w.K * (w.p + 1) * STAGES * nsmall)
    out["advection_small"]["sample"] = f"all {nsmall} steps"

    b = BURGERS_1M
    win = 1 << 18
    dxb = 2 * math.pi / b.K
    x = dg.node_coordinates(win, b.p, 0.0, 2 * math.pi, 0, b.K)
    ub = b.modes.offset + np.sin(x)
    tblb = delays.delay_table(b.seed, b.P, 4, b.L)
    probb = dg.Problem(pde="burgers", K=win, p=b.p, P=b.P, dt=0.005 * dxb / 1.5, mode="adg",
                       q=b.q, delays=tblb, window_lo=0, K_global=b.K)
    out["burgers_1m"] = both(lambda: dg.run(probb, ub, 2), win * (b.p + 1) * STAGES * 2)
    out["burgers_1m"]["sample"] = "2 steps on a 2^18-element window"

    ws = batched_instances()[:8]
    runs = []
    for wi in ws:
        dxi = 2 * math.pi / wi.K
        tb = delays.delay_table(wi.seed, wi.P, 4, wi.L)
        pr = dg.Problem(pde="advection", K=wi.K, p=wi.p, P=wi.P, a=wi.a, dt=wi.cfl * dxi / wi.a,
                        mode="adg", q=wi.q, delays=tb)
        runs.append((pr, dg.modes_initial(wi.modes, wi.K, wi.p)))
    units = sum(wi.K * (wi.p + 1) * STAGES * 2 for wi in ws)
    out["batched"] = both(lambda: [dg.run(pr, uu, 2) for pr, uu in runs], units)
    out["batched"]["sample"] = "2 steps of the first 8 instances"

    a = _WADJ
    dxa = 2 * math.pi / a.K
    xa = dg.node_coordinates(a.K, a.p, 0.0, 2 * math.pi)
    ua = a.modes.offset + np.sin(xa)
    ga = 0.5 + np.sin(xa - 0.003)
    tba = delays.delay_table(a.seed, a.P, 10, a.L)
    pra = dg.Problem(pde="burgers", K=a.K, p=a.p, P=a.P, dt=a.cfl * dxa / 1.5, mode="adg",
                     q=a.q, delays=tba)
    t0 = time.perf_counter()
    dg.run(pra, ua, 10)
    tf = time.perf_counter() - t0
    t0 = time.perf_counter()
    dg.gradient(pra, ua, ga, 10)
    tg = time.perf_counter() - t0
    out["adjoint"] = {"forward_s": tf, "grad_s": tg, "grad_over_forward": tg / tf,
                      "threads": torch.get_num_threads(),
                      "sample": "10 steps on the full K = 65536 mesh (store-all autograd)"}
    return out


def cpu_baseline(window: int = 1 << 22, steps: int = 3) -> dict:
    """The oracle on all of torch's CPU threads and on one thread (a 2^20-element window)."""
    rate, _, used, sample = oracle_timed(window, steps)
    one, _, _, one_sample = oracle_timed(1 << 20, 2, 1, threads=1)
    out = {"value": rate, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample,
           "one_thread": {"value": one, "sample": one_sample}}
    out.update(host_info())
    return out


def profile_case(name: str) -> dict:
    """A few steps of a smaller case in two calls (4 + 8 steps, or 3 + 3 for Burgers), for
    ncu captures that stay within a few GB and a few seconds."""
    import torch
    import paper_2404_03399_gb300 as adg
    w = WORKLOAD
    if name == "batched":
        # the 512-instance batched workload, two elements per thread (the tuner's choice
        # outside the profiler), 2 + 4 steps
        ws = batched_instances()
        cfgs = [adg.Config(pde="advection", K=v.K, p=v.p, P=v.P, a=v.a, cfl=v.cfl, mode=v.mode,
                           L=v.L, q=v.q, seed=v.seed, ept=2) for v in ws]
        u0s = [adg.eval_modes(c, v.modes.amp, v.modes.kappa, v.modes.phase)
               for c, v in zip(cfgs, ws)]
        b = adg.BatchSolver(cfgs, u0s)
        del u0s
        for k in (2, 4):
            b.step(k)
        torch.cuda.synchronize()
        out = {"case": name, "instances": len(ws), "variant": list(b.variant(0)), "steps": 6}
        b.close()
        return out
    if name == "e2e_16m":
        # the end-to-end path twice (host u0 in, 4 steps, state out to host): the layout and
        # state-rows kernels over the host link
        ms = [e2e_timed(4)[0] for _ in range(2)]
        return {"case": name, "K": w["K"], "steps": 4, "ms": ms}
    if name == "burgers_1m":
        b = BURGERS_1M
        cfg = adg.Config(pde="burgers", K=b.K, p=b.p, P=b.P, cfl=0.005, mode="at", L=b.L, q=b.q,
                         seed=b.seed)
        m = b.modes
        u0 = adg.eval_modes(cfg, m.amp, m.kappa, m.phase, m.offset)
        calls = (3, 3)
    else:
        K = w["K"] if name == "fixed_16m" else 1 << 22
        # two elements per thread, the choice the autotuner makes outside the profiler (its
        # timing launches run differently under it)
        cfg = adg.Config(pde="advection", K=K, p=w["p"], P=K // (w["K"] // w["P"]), cfl=w["cfl"],
                         mode="at", L=w["L"], q=w["q"], seed=w["seed"], ept=2,
                         rk="lsrk4" if name == "lsrk4_4m" else "ssprk3")
        amp, kap, ph, off = w["modes"]
        u0 = adg.eval_modes(cfg, amp, kap, ph, off)
        calls = (4, 8)
    s = adg.Solver(cfg, u0)
    for k in calls:
        s.step(k)
    torch.cuda.synchronize()
    out = {"case": name, "K": cfg.K, "variant": list(s.variant), "steps": sum(calls)}
    s.close()
    return out


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
        return rank, ws, local, dist
    return 0, 1, 0, None


def aggregate(dist, ms: float, units: float):
    """Max of the timed region over ranks and the sum of units (weak scaling)."""
    if dist is None:
        return ms, units
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def reference_arm(args, rank, ws):
    """The oracle (the reference for this method) on the host cores, on the same metric, unit
    and workload as the GPU arm: `--warmup` untimed and `--steps` timed steps, each over the
    whole mesh when the run fits in about two minutes (about 1.5 s per step on 16 Arm cores),
    else over a window of whole PEs."""
    if rank != 0:
        return
    K, P = WORKLOAD["K"], WORKLOAD["P"]
    kpe = K // P
    n = args.steps + args.warmup
    window = K if n <= 60 else max(kpe, (K * 60 // n) // kpe * kpe)
    if args.ref_window > 0:
        window = min(K, args.ref_window)
    rate, ms_step, used, sample = oracle_timed(window, args.steps, args.warmup)
    base = {"value": rate, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample}
    base.update(host_info())
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "ms_per_step_is": "the timed oracle steps (whole mesh)" if window == K else
                              f"the timed oracle steps on a {window}-element window",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(ws), "cpu_baseline": base,
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip sync-DG and e2e runs")
    ap.add_argument("--ref-window", type=int, default=0,
                    help="reference arm: elements per oracle step (0: the whole mesh when the "
                         "run fits in about two minutes, else a window of whole PEs)")
    ap.add_argument("--adjoint-only", type=int, default=0, metavar="STEPS",
                    help="only time adg_grad against the forward on the adjoint workload for STEPS "
                         "steps (one repeat) and print that dict (for profiling runs)")
    ap.add_argument("--extra-only", choices=["lsrk4", "viscous", "euler"], default=None,
                    help="only time that extra workload (the LSRK4 scheme on the large mesh, "
                         "viscous Burgers, Euler) and print its dict (for profiling runs)")
    ap.add_argument("--profile", choices=["fixed_4m", "fixed_16m", "lsrk4_4m", "burgers_1m",
                                          "batched", "e2e_16m"],
                    default=None,
                    help="run a few steps of a case for ncu captures and print its dict: "
                         "advection K = 2^22 (the large workload's PE size, delays and AT order) "
                         "with the fixed-point step, the same at the full K = 2^24, the K = 2^22 "
                         "case with LSRK4, the Burgers workload (K = 2^20) at Courant number "
                         "0.005, the 512-instance batch, or the end-to-end path from host "
                         "buffers on the large mesh (4 steps, twice)")
    ap.add_argument("--batched-only", type=int, default=0, metavar="STEPS",
                    help="only time the batched workload for STEPS steps and print that dict "
                         "(for profiling runs)")
    args = ap.parse_args()

    rank, ws, local, dist = dist_setup()
    if args.impl == "reference":
        reference_arm(args, rank, ws)
        if dist is not None:
            dist.destroy_process_group()
        return

    import torch
    import paper_2404_03399_gb300 as adg
    torch.cuda.set_device(local)
    adg.load()
    if args.adjoint_only:
        print(json.dumps(adjoint_cost(args.adjoint_only, 1)), flush=True)
        return
    if args.extra_only:
        if args.extra_only == "lsrk4":
            ms, _, fin, (var, _, _) = device_timed("at", 4, 2, lambda: None, False, local, "lsrk4")
            out = {"lsrk4_ms_per_step": ms / 4, "finite": fin, "variant": var}
        elif args.extra_only == "viscous":
            ms, dof, fin = viscous_timed(4, 2)
            out = {"viscous_ms_per_step": ms / 4, "dof": dof, "finite": fin}
        else:
            ms, dof, fin = euler_timed(4, 2)
            out = {"euler_ms_per_step": ms / 4, "dof": dof, "finite": fin}
        print(json.dumps(out), flush=True)
        return
    if args.profile:
        print(json.dumps(profile_case(args.profile)), flush=True)
        return
    if args.batched_only:
        rate, ms, ndof, n, variant = batched_timed(args.batched_only, 3)
        print(json.dumps({"batched": rate, "ms_per_step": ms, "dof": ndof, "instances": n,
                          "variant": variant}), flush=True)
        return
    barrier = (lambda: dist.barrier()) if dist is not None else (lambda: None)

    K, p = WORKLOAD["K"], WORKLOAD["p"]
    ndof = K * (p + 1)
    acc_at = {}
    ms, clocks, finite, (variant, ept, basis) = device_timed("at", args.steps, args.warmup, barrier,
                                                      rank == 0, local, exact_error=acc_at)
    units = ndof * STAGES * args.steps
    ms_max, units_all = aggregate(dist, ms, units)
    value = units_all / (ms_max * 1e-3)

    hbm_gbs, hbm_src, fp64_tflops, sms, sm_mhz = peaks()
    ms_step = ms / args.steps
    step_s = ms_step * 1e-3
    # Roofline of the step against HBM (the metric's roofline): the algorithmic 16 B per DOF
    # (read u^n, write u^{n+1}) over the CUDA-event time of a step, which is one composed-step
    # launch plus the PE-face launch between steps (charged to it: the kernel's own share is
    # the larger one).
    hbm_algo_gbs = ndof * BYTES_PER_DOF_STEP / step_s / 1e9
    roofline = {"bound": "hbm", "achieved": hbm_algo_gbs, "peak": hbm_gbs, "unit": "GB/s",
                "frac": hbm_algo_gbs / hbm_gbs, "traffic": TRAFFIC_BYTES_PER_LAUNCH.get(
                    f"{variant}/{ept}/{'basis' if basis else 'nodal'}"),
                "peak_source": f"{hbm_src} copy bandwidth (MEASURED_PEAKS.json)",
                "bytes_per_dof_step": BYTES_PER_DOF_STEP}
    if variant == "fixed":
        wide = FIXED_MACS_PER_ELEMENT_STEP_BASIS if basis else FIXED_MACS_PER_ELEMENT_STEP
        # 3 products per multiply-add, 2 passes each, 16 lanes per clock per sub-partition
        pipe_s = K * 3 * wide * 2 / (16 * 4 * sms * sm_mhz * 1e6)
        roofline["kernel"] = (f"k_step_fixed (composed SSP-RK3 step in 58-bit block fixed point, "
                              f"{'block-basis coordinates' if basis else 'nodal values'}, "
                              f"{ept} element(s) per thread) + k_face_step")
        roofline["alu"] = {
            "what": f"heavy FMA pipe: {wide} multiply-adds of 58-bit precision per element, three "
                    f"32x32->64-bit products each, every product two passes of the pipe's 16 "
                    f"lanes per clock per SM sub-partition ({sms} SMs x 4, {sm_mhz:.0f} MHz)",
            "pipe_bound_ms": pipe_s * 1e3, "frac": pipe_s / step_s}
    else:
        roofline["kernel"] = f"k_step_fused / k_stage ({variant}, FP64)"
        roofline["fp64"] = {"achieved_tflops": ndof * FLOP_PER_DOF_STEP / step_s / 1e12,
                            "peak_tflops": fp64_tflops,
                            "frac": ndof * FLOP_PER_DOF_STEP / step_s / 1e12 / fp64_tflops}
    arithmetic = ("58-bit block fixed point: int64 values at one scale per field and step "
                  "(unit 2^-57 of the field's largest value; a sum of n products is off by less "
                  "than n/2 + 1/2 units), the state kept in int64 from step to step"
                  + (" as coordinates in the block basis of the element operator (cond_inf "
                     "15.1 at p = 3, which scales the rounding bound)" if basis else "")
                  + "; FP64 in the PE-face stage differences and where the state is read") \
        if variant == "fixed" else "FP64"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "int64" if variant == "fixed" else "f64", "data": "synthetic",
            "config": bench_config(ws), "variant": variant, "arithmetic": arithmetic,
            "roofline": roofline,
            # per step: the composed-step kernel and one PE-face kernel (correction of the step
            # before, differences of the next); per chunk of CHUNK_STEPS steps one step-counter
            # kernel and one more PE-face kernel
            "gpu_launches": 2 * args.steps + 2 * math.ceil(args.steps / CHUNK_STEPS),
            "launches": "direct chunks of up to 256 steps, kernels launched as programmatic "
                        "dependents of the one before",
            "finite": finite, "clocks": clocks}

    if not args.no_extras:
        # end to end first, in the process state the main run left
        ems, nbytes = e2e_timed(args.steps)
        line["e2e"] = {"value": ndof * STAGES * args.steps / (ems * 1e-3), "unit": UNIT,
                       "h2d_bytes_per_step": nbytes / args.steps, "d2h_bytes_per_step": nbytes / args.steps,
                       "what": "adg_init_host from pinned u0 (read in place over the host link), all "
                               "steps, adg_get_state_host into pinned memory"}
        # synchronous DG on the same mesh, the same number of steps in one adg_step call
        acc_sync = {}
        sync_ms, _, _, (svar, _, _) = device_timed("sync", args.steps, args.warmup, barrier, False,
                                               local, exact_error=acc_sync)
        line["sync_dg"] = {"value": ndof * STAGES * args.steps / (sync_ms * 1e-3), "unit": UNIT,
                           "ms_per_step": sync_ms / args.steps, "steps": args.steps,
                           "variant": svar}
        line["at_over_sync"] = value / ws / line["sync_dg"]["value"]
        # the accuracy half of the comparison: both schemes against the exact translated
        # solution after the same steps
        line["accuracy"] = {"advection_16m": {"at": acc_at, "sync": acc_sync,
                                              "norm": "max |u - u_exact| / max |u_exact|"}}
        # the Burgers workload (LLF, K = 2^20, p = 4, 1024 PEs, AT2, L = 4): the staged
        # stage kernels, at the stated Courant number 0.05 and at 0.005, inside the stability
        # bound of the delayed self-feedback
        bline = {"workload": "Burgers u0 = 0.5 + sin x, K = 2^20, p = 4, LLF, SSP-RK3, 1024 PEs, "
                             "delays uniform in {0..3} (L = 4), AT order 2",
                 "dof": BURGERS_1M.ndof, "steps": args.steps,
                 "kernel": "k_stage (one SSP-RK3 stage, PE-face flux and ring write fused), three per step",
                 "flop_per_dof_stage": FLOP_PER_DOF_STAGE_BURGERS}
        for cfl in (BURGERS_1M.cfl, 0.005):
            for mode in ("at", "sync"):
                bms, bfin, bvar, bacc = burgers_timed(args.steps, args.warmup, mode, cfl)
                bstep = bms / args.steps * 1e-3
                bline[f"{mode}_cfl{cfl}"] = {
                    "value": BURGERS_1M.ndof * STAGES / bstep, "unit": UNIT,
                    "ms_per_step": bms / args.steps, "finite": bfin, "variant": bvar,
                    "fp64_frac": BURGERS_1M.ndof * STAGES * FLOP_PER_DOF_STAGE_BURGERS / bstep
                                 / 1e12 / fp64_tflops,
                    "bytes_frac": BURGERS_1M.ndof * BYTES_PER_DOF_STEP_STAGED / bstep / 1e9 / hbm_gbs,
                    "error_vs_characteristics": bacc}
        line["burgers_1m"] = bline
        line["advection_small"] = {mode: small_timed(mode) for mode in ("sync", "async", "at")}
        line["advection_small"]["workload"] = ("K = 64, p = 2, 16 PEs, delays uniform in {0..3}, "
                                               "sigma = 0.1, t_end = 2 pi (640 steps), AT order 3")
        # the same ADG-AT steps in FP64 (the composed step on the FP64 pipe)
        f_ms, _, ffin, (fvar, _, _) = device_timed("at", args.steps, args.warmup, barrier, False,
                                               local, variant="composed")
        f_s = f_ms / args.steps * 1e-3
        line["fp64_composed"] = {
            "value": ndof * STAGES * args.steps / (f_ms * 1e-3), "unit": UNIT,
            "ms_per_step": f_ms / args.steps, "steps": args.steps, "variant": fvar, "dtype": "f64",
            "finite": ffin, "kernel": "k_step_fused (composed SSP-RK3 step in FP64) + k_step_fixup",
            "fp64_tflops": ndof * FLOP_PER_DOF_STEP / f_s / 1e12,
            "fp64_frac": ndof * FLOP_PER_DOF_STEP / f_s / 1e12 / fp64_tflops,
            "hbm_frac": ndof * BYTES_PER_DOF_STEP / f_s / 1e9 / hbm_gbs}
        brate, bms, bdof, bn, bvariant = batched_timed(100, 3)
        line["batched"] = {"value": brate, "unit": UNIT, "ms_per_step": bms, "instances": bn,
                           "dof": bdof, "steps": 100, "variant": bvariant,
                           "hbm_frac": bdof * BYTES_PER_DOF_STEP / (bms * 1e-3) / 1e9 / hbm_gbs,
                           "chosen_by": "the batch autotuner at adg_batch_init",
                           "workload": "512 advection instances, K log-uniform in [1024, 262144], "
                                       "p in 1..4, L in 2..8, AT order min(p+1, 3)"}
        line["adjoint"] = adjoint_cost()
        # the 2N low-storage schemes (staged kernels) on the same mesh, ADG-AT3
        ls = {}
        for rk, S in LOW_STORAGE_STAGES.items():
            lms, _, lfin, (lvar, _, _) = device_timed("at", 10, 3, barrier, False, local, rk)
            step_s = lms / 10 * 1e-3
            staged = lvar == "staged"   # schemes of <= 3 stages run the composed fixed-point step
            ls[rk] = {"value": ndof * S / step_s, "unit": UNIT, "ms_per_step": lms / 10,
                      "stages": S, "variant": lvar, "finite": lfin,
                      "fp64_tflops": ndof * S * FLOP_PER_DOF_STAGE_LS / step_s / 1e12 if staged else None,
                      "fp64_frac": (ndof * S * FLOP_PER_DOF_STAGE_LS / step_s / 1e12 / fp64_tflops
                                    if staged else None)}
        cms, cst, cvar = caa_timed(args.steps, args.warmup)
        line["caa"] = {"value": ndof * STAGES * args.steps / (cms * 1e-3), "unit": UNIT,
                       "ms_per_step": cms / args.steps, "variant": cvar,
                       "workload": "the same mesh, communication-avoiding cycle of Section 6.3 "
                                   "(L = 3, 2 synchronised steps of 5), ADG-AT2",
                       "exchanges": cst["exchanges"], "sync_exchanges": cst["sync_exchanges"],
                       "exchange_saving": 1.0 - cst["exchanges"] / max(cst["sync_exchanges"], 1),
                       "steps_counted": cst["steps"]}
        vms, vdof, vfin = viscous_timed(20, 3)
        vstep = vms / 20 * 1e-3
        line["viscous_burgers"] = {
            "value": vdof * 2 / vstep, "unit": UNIT, "ms_per_step": vms / 20, "finite": vfin,
            "workload": "ALDG(2)-AT2-RK2, nu = 0.1, K = 2^20, 1024 PEs, L = 3 (0.3/0.4/0.3), "
                        "dt = 0.01 dx^2 (Section 6 viscous Burgers, scaled up)",
            "fp64_tflops": vdof * 2 * FLOP_PER_DOF_STAGE_VISC / vstep / 1e12,
            "fp64_frac": vdof * 2 * FLOP_PER_DOF_STAGE_VISC / vstep / 1e12 / fp64_tflops,
            "kernels": "k_ldg_q (q = u_x) then k_lsrk_stage with the viscous term, per stage"}
        ems2, edof, efin = euler_timed(20, 3)
        line["euler_sod"] = {
            "value": edof * 2 / (ems2 / 20 * 1e-3), "unit": UNIT, "ms_per_step": ems2 / 20,
            "finite": efin, "components": 3,
            "workload": "1D Euler, Sod data (two Riemann problems), DG(1), ADG-AT2-RK2 with the "
                        "TVB-minmod limiter, K = 2^20, 1024 PEs, L = 3 (0.3/0.4/0.3), dt = 0.1 dx",
            "kernels": "k_euler_stage then k_euler_limit, per stage"}
        line["low_storage"] = {"schemes": ls, "steps": 10, "mode": "at",
                               "kernel": "schemes of up to three stages: the composed fixed-point "
                                         "step (k_step_fixed, k_face_step); LSRK4: k_lsrk_stage "
                                         "(one 2N stage: dt L(U), dU and U updates, PE faces; an "
                                         "odd stage count adds a copy back into u)",
                               "peak_source": "FP64 unit counts x max SM clock"}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
        if not args.no_extras:
            line["cpu_baseline"]["other_workloads"] = oracle_configs()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
