"""GB300 asynchronous discontinuous Galerkin (ADG / ADG-AT) solver: Python binding.

A thin layer over the C ABI of ``include/adg.h`` (``libadg.so``): it marshals arguments
and uses torch for device memory and streams. Every step of the numerical path runs in
the library's CUDA kernels; there is no CPU fallback.

    cfg = Config(pde="advection", K=64, p=2, P=16, cfl=0.1, mode="at", L=4, q=3)
    u0 = eval_modes(cfg, amp=[1.0], kappa=[1.0], phase=[0.0])   # (K, p+1) on cuda
    s = Solver(cfg, u0)
    s.step(640)
    u = s.state()
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np
import torch

from . import _abi
from ._abi import AdgError, check, load

__all__ = ["Config", "Solver", "BatchSolver", "ADGFunction", "eval_modes", "delay_table",
           "lgl_nodes", "AdgError", "load"]

_PDE = {"advection": _abi.ADG_ADVECTION, "burgers": _abi.ADG_BURGERS, "euler": _abi.ADG_EULER}
_MODE = {"sync": _abi.ADG_SYNC, "async": _abi.ADG_ASYNC, "at": _abi.ADG_ASYNC_AT}


@dataclass
class Config:
    """Mirror of ``adg_config`` (include/adg.h)."""
    pde: str = "advection"
    K: int = 64
    p: int = 2
    P: int = 1
    x0: float = 0.0
    x1: float = 2.0 * math.pi
    a: float = 1.0
    cfl: float = 0.1
    dt: float = 0.0
    mode: str = "sync"          # "sync" | "async" | "at"
    L: int = 1
    q: int = 0                  # AT order; 0 = p+1
    seed: int = 0
    probs: Optional[Sequence[float]] = None
    table: Optional[np.ndarray] = None   # uint8 (T, P), used periodically
    variant: str = "auto"       # "auto" | "staged" | "composed" | "fixed"
    rk: str = "ssprk3"          # "ssprk3" | "rk1" | "rk2" | "lsrk3" | "lsrk4"
    caa_sync: int = 0           # > 0: communication-avoiding delay cycle (Section 6.3)
    nu: float = 0.0             # > 0: viscous Burgers by the local DG method (Eq. burgers)
    limiter: bool = True        # Euler: TVB-minmod slope limiter on every stage output
    tvb_m: float = 0.0          # Euler: TVB constant M (0: minmod)
    ept: int = 0                # elements per thread of the composed kernels (0: autotuned)

    def to_c(self):
        c = _abi.AdgConfig()
        load().adg_config_default(C.byref(c))
        c.pde = _PDE[self.pde]
        c.flux = _abi.ADG_UPWIND if self.pde == "advection" else _abi.ADG_LLF
        c.limiter = 1 if self.limiter else 0
        c.tvb_m = float(self.tvb_m)
        c.rk = {"rk1": _abi.ADG_RK1, "rk2": _abi.ADG_RK2, "ssprk3": _abi.ADG_SSPRK3,
                "lsrk3": _abi.ADG_LSRK3, "lsrk4": _abi.ADG_LSRK4}[self.rk]
        c.K, c.p, c.P = int(self.K), int(self.p), int(self.P)
        c.x0, c.x1, c.a = float(self.x0), float(self.x1), float(self.a)
        c.cfl, c.dt = float(self.cfl), float(self.dt)
        c.mode = _MODE[self.mode]
        c.L = int(self.L)
        c.at_order = int(self.q)
        c.seed = int(self.seed) & ((1 << 64) - 1)
        c.variant = {"auto": 0, "staged": 1, "composed": 2, "fixed": 3}[self.variant]
        c.caa_sync = int(self.caa_sync)
        c.nu = float(self.nu)
        c.ept = int(self.ept)
        keep = []
        if self.probs is not None:
            arr = (C.c_double * len(self.probs))(*[float(v) for v in self.probs])
            keep.append(arr)
            c.probs = C.cast(arr, C.POINTER(C.c_double))
        if self.table is not None:
            t = np.ascontiguousarray(self.table, dtype=np.uint8)
            keep.append(t)
            c.delay_table = t.ctypes.data_as(C.POINTER(C.c_uint8))
            c.table_steps = t.shape[0]
        return c, keep


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _shape(cfg) -> tuple:
    """Field shape: (K, p+1), or (3, K, p+1) for the Euler equations."""
    return (3, cfg.K, cfg.p + 1) if cfg.pde == "euler" else (cfg.K, cfg.p + 1)


def _as_field(x: torch.Tensor, K: int, Np: int, ncomp: int = 1, host: bool = False) -> torch.Tensor:
    if not (isinstance(x, torch.Tensor) and (x.device.type == "cpu" if host else x.is_cuda)):
        raise ValueError("expected a CPU tensor" if host else "expected a CUDA tensor")
    x = x.to(torch.float64).contiguous()
    want = (K, Np) if ncomp == 1 else (ncomp, K, Np)
    if tuple(x.shape) != want:
        raise ValueError(f"expected shape {want}, got {tuple(x.shape)}")
    return x


def eval_modes(cfg: Config, amp, kappa, phase, offset: float = 0.0, device="cuda") -> torch.Tensor:
    """Nodal values of offset + sum A sin(kappa x + phi) at the library's LGL nodes."""
    c, keep = cfg.to_c()
    n = len(amp)
    arr = lambda v: (C.c_double * max(n, 1))(*[float(t) for t in v])
    A, Kp, Ph = arr(amp), arr(kappa), arr(phase)
    u = torch.empty((cfg.K, cfg.p + 1), dtype=torch.float64, device=device)
    check(load().adg_eval_modes(C.byref(c), n, A, Kp, Ph, float(offset), u.data_ptr(),
                                _stream_ptr(None)))
    return u


def delay_table(cfg: Config, first_step: int, steps: int) -> np.ndarray:
    """The delays the library uses for cfg (host only; no GPU needed)."""
    c, keep = cfg.to_c()
    out = np.zeros((steps, cfg.P), dtype=np.uint8)
    check(load().adg_delay_table(C.byref(c), int(first_step), int(steps),
                                 out.ctypes.data_as(C.POINTER(C.c_uint8))))
    return out


def lgl_nodes(p: int):
    x = (C.c_double * (p + 1))()
    w = (C.c_double * (p + 1))()
    check(load().adg_lgl_nodes(int(p), x, w))
    return np.array(list(x)), np.array(list(w))


class Solver:
    """One ADG instance on the current CUDA device (``adg_init`` / ``adg_step`` / ...). u0 is
    a CUDA tensor (``adg_init``) or a CPU tensor (``adg_init_host``: read in place over the
    host link when pinned, staged through device memory otherwise)."""

    def __init__(self, cfg: Config, u0: torch.Tensor, stream: Optional[torch.cuda.Stream] = None):
        self.cfg = cfg
        self.Np = cfg.p + 1
        host = isinstance(u0, torch.Tensor) and u0.device.type == "cpu"
        u0 = _as_field(u0, cfg.K, self.Np, 3 if cfg.pde == "euler" else 1, host=host)
        c, keep = cfg.to_c()
        self._stream = stream
        ctx = C.c_void_p()
        init = load().adg_init_host if host else load().adg_init
        check(init(C.byref(c), u0.data_ptr(), _stream_ptr(stream), C.byref(ctx)))
        self._ctx = ctx

    @property
    def ctx(self):
        if self._ctx is None:
            raise AdgError(_abi.ADG_ESTATE, "solver is closed")
        return self._ctx

    def step(self, nsteps: int) -> None:
        check(load().adg_step(self.ctx, int(nsteps)), self.ctx)

    def run(self, t_end: float) -> None:
        check(load().adg_run(self.ctx, float(t_end)), self.ctx)

    def state(self, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """The FP64 state: into a new CUDA tensor, or into `out` (a contiguous FP64 tensor of
        the field's shape on the GPU, or on the host: ``adg_get_state_host``)."""
        if out is None:
            out = torch.empty(_shape(self.cfg), dtype=torch.float64, device="cuda")
        if out.dtype != torch.float64 or not out.is_contiguous() or tuple(out.shape) != _shape(self.cfg):
            raise ValueError(f"out must be a contiguous float64 tensor of shape {_shape(self.cfg)}")
        n = C.c_int64()
        get = load().adg_get_state_host if out.device.type == "cpu" else load().adg_get_state
        check(get(self.ctx, 0, out.data_ptr(), C.byref(n)), self.ctx)
        self.n = n.value
        return out

    @property
    def dt(self) -> float:
        v = C.c_double()
        check(load().adg_get_dt(self.ctx, 0, C.byref(v)), self.ctx)
        return v.value

    @property
    def variant(self) -> tuple:
        """(variant in use: "staged" | "composed" | "fixed", elements per thread)."""
        v, e = C.c_int32(), C.c_int32()
        check(load().adg_get_variant(self.ctx, 0, C.byref(v), C.byref(e)), self.ctx)
        return {1: "staged", 2: "composed", 3: "fixed"}[v.value], e.value

    @property
    def fixed_basis(self) -> bool:
        """True when the fixed-point state holds block-basis coordinates (adg_get_fixed_basis)."""
        b = C.c_int32()
        check(load().adg_get_fixed_basis(self.ctx, 0, C.byref(b)), self.ctx)
        return bool(b.value)

    def comm_stats(self) -> dict:
        """PE-face exchanges a distributed run of the steps so far would make, against
        synchronous DG (adg_comm_stats)."""
        n, ex, sy = C.c_int64(), C.c_int64(), C.c_int64()
        check(load().adg_comm_stats(self.ctx, 0, C.byref(n), C.byref(ex), C.byref(sy)), self.ctx)
        return {"steps": n.value, "exchanges": ex.value, "sync_exchanges": sy.value}

    def integral(self) -> float:
        v = C.c_double()
        check(load().adg_integral(self.ctx, 0, C.byref(v)), self.ctx)
        return v.value

    def check_finite(self) -> None:
        check(load().adg_check_finite(self.ctx), self.ctx)

    def misfit(self, target: torch.Tensor) -> float:
        """J = 1/2 ||u - g||_M^2 of the current state against target g."""
        g = _as_field(target, self.cfg.K, self.Np, 3 if self.cfg.pde == "euler" else 1)
        J = C.c_double()
        check(load().adg_misfit(self.ctx, 0, g.data_ptr(), C.byref(J)), self.ctx)
        return J.value

    def grad(self, target: torch.Tensor, nsteps: int, ckpt_every: int = 50):
        """(J, dJ/du0) of J = 1/2 ||u_N - g||_M^2 over nsteps from the current state."""
        g = _as_field(target, self.cfg.K, self.Np, 3 if self.cfg.pde == "euler" else 1)
        out = torch.empty_like(g)
        J = C.c_double()
        check(load().adg_grad(self.ctx, g.data_ptr(), int(nsteps), int(ckpt_every),
                              out.data_ptr(), C.byref(J)), self.ctx)
        return J.value, out

    def close(self) -> None:
        if self._ctx is not None:
            load().adg_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSolver:
    """Many independent advection instances advanced together (``adg_batch_init``)."""

    def __init__(self, cfgs: Sequence[Config], u0s: Sequence[torch.Tensor],
                 stream: Optional[torch.cuda.Stream] = None):
        self.cfgs = list(cfgs)
        n = len(self.cfgs)
        arr = (_abi.AdgConfig * n)()
        keep = []
        fields = []
        for i, (cf, u) in enumerate(zip(self.cfgs, u0s)):
            c, k = cf.to_c()
            arr[i] = c
            keep.append(k)
            fields.append(_as_field(u, cf.K, cf.p + 1, 3 if cf.pde == "euler" else 1))
        ptrs = (C.c_void_p * n)(*[f.data_ptr() for f in fields])
        ctx = C.c_void_p()
        check(load().adg_batch_init(arr, ptrs, n, _stream_ptr(stream), C.byref(ctx)))
        self._ctx = ctx

    def step(self, nsteps: int) -> None:
        check(load().adg_step(self._ctx, int(nsteps)), self._ctx)

    def state(self, i: int, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Instance i's FP64 state, into a new CUDA tensor or into `out` (GPU or host)."""
        cf = self.cfgs[i]
        shape = (cf.K, cf.p + 1)
        if out is None:
            out = torch.empty(shape, dtype=torch.float64, device="cuda")
        if out.dtype != torch.float64 or not out.is_contiguous() or tuple(out.shape) != shape:
            raise ValueError(f"out must be a contiguous float64 tensor of shape {shape}")
        get = load().adg_get_state_host if out.device.type == "cpu" else load().adg_get_state
        check(get(self._ctx, int(i), out.data_ptr(), None), self._ctx)
        return out

    def dt(self, i: int) -> float:
        v = C.c_double()
        check(load().adg_get_dt(self._ctx, int(i), C.byref(v)), self._ctx)
        return v.value

    def variant(self, i: int) -> tuple:
        """(variant instance i runs: "staged" | "composed" | "fixed", elements per thread)."""
        v, e = C.c_int32(), C.c_int32()
        check(load().adg_get_variant(self._ctx, int(i), C.byref(v), C.byref(e)), self._ctx)
        return {1: "staged", 2: "composed", 3: "fixed"}[v.value], e.value

    def fixed_basis(self, i: int) -> bool:
        """True when instance i's fixed-point state holds block-basis coordinates."""
        b = C.c_int32()
        check(load().adg_get_fixed_basis(self._ctx, int(i), C.byref(b)), self._ctx)
        return bool(b.value)

    def integral(self, i: int) -> float:
        """Discrete integral (dx/2) sum_e w^T u^e of instance i's current state."""
        v = C.c_double()
        check(load().adg_integral(self._ctx, int(i), C.byref(v)), self._ctx)
        return v.value

    def check_finite(self) -> None:
        check(load().adg_check_finite(self._ctx), self._ctx)

    def close(self) -> None:
        if self._ctx is not None:
            load().adg_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ADGFunction(torch.autograd.Function):
    """u_N = ADG-AT forward map of u0 over nsteps; backward returns d(J)/d(u0) where
    J = 1/2 ||u_N - target||_M^2 is evaluated by the library's discrete adjoint.

    Usage: J = ADGFunction.apply(u0, cfg, target, nsteps, ckpt_every) returns the misfit
    as a 0-d tensor; J.backward() fills u0.grad."""

    @staticmethod
    def forward(ctx, u0, cfg, target, nsteps, ckpt_every=50):
        s = Solver(cfg, u0.detach())
        try:
            J, g = s.grad(target, nsteps, ckpt_every)
        finally:
            s.close()
        ctx.save_for_backward(g)
        return torch.tensor(J, dtype=torch.float64, device=u0.device)

    @staticmethod
    def backward(ctx, gJ):
        (g,) = ctx.saved_tensors
        return gJ * g, None, None, None, None
