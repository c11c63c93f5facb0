"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds no arithmetic of the DG method: it only names workloads and draws
parameters (Fourier-mode amplitudes, wavenumbers, phases, random nodal arrays, batch
instance descriptors, fixed delay tables). Each consumer evaluates initial conditions at
its own nodes.

Workloads (sizes follow the paper's experiments, Section 6, and the hot-path configs):

* ``advection_small`` -- u_t + u_x = 0 on [0, 2pi], u0 = sin x, K = 64, p = 2, 16 PEs
  of 4 elements, CFL 0.1, t_end = 2pi (640 steps), delays uniform in {0..3} (L = 4).
* ``burgers_1m``      -- inviscid Burgers, u0 = 0.5 + sin x, K = 2^20, p = 4, LLF flux,
  CFL 0.05, 1024 PEs, delays uniform in {0..3}, AT order 2.
* ``batched_512``     -- 512 independent advection instances (K log-uniform in
  [1024, 262144] rounded to 256, p in {1..4}, a in [0.5, 2], four random modes,
  L in {2..8}).
* ``adjoint_64k``     -- Burgers as ``burgers_1m`` but K = 65536, p = 3, 2000 steps,
  checkpoint every 50.
* ``advection_16m``   -- advection, K = 2^24, p = 3, 16384 PEs, delays uniform in
  {0..7} (L = 8), AT order 3, 500 SSP-RK3 steps.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence, Tuple

import numpy as np

TWO_PI = 2.0 * math.pi


@dataclass(frozen=True)
class Modes:
    """u0(x) = offset + sum_m amp[m] * sin(kappa[m] * x + phase[m]) (Eq. initialcond)."""

    amp: Tuple[float, ...]
    kappa: Tuple[float, ...]
    phase: Tuple[float, ...]
    offset: float = 0.0


@dataclass(frozen=True)
class Workload:
    name: str
    pde: str                 # "advection" | "burgers"
    K: int
    p: int
    P: int
    modes: Modes
    a: float = 1.0
    cfl: float = 0.1
    mode: str = "at"         # "sync" | "async" | "at"
    L: int = 4
    q: int = 1
    seed: int = 0
    probs: Optional[Tuple[float, ...]] = None   # None: uniform over {0..L-1}
    steps: int = 0
    t_end: float = 0.0
    x0: float = 0.0
    x1: float = TWO_PI

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)

    @property
    def ndof(self) -> int:
        return self.K * (self.p + 1)


SIN = Modes(amp=(1.0,), kappa=(1.0,), phase=(0.0,))
HALF_PLUS_SIN = Modes(amp=(1.0,), kappa=(1.0,), phase=(0.0,), offset=0.5)
# Phases for paper-style multi-scale tests: the paper includes phases but prints no values.
PAPER_FIG6 = Modes(amp=(2.0, 1.0), kappa=(2.0, 3.0), phase=(0.3, 1.1))
PAPER_MULTISCALE = Modes(amp=(3.0, 2.0, 1.0), kappa=(2.0, 3.0, 5.0), phase=(0.3, 1.1, 2.0))

ADVECTION_SMALL = Workload(
    name="advection_small", pde="advection", K=64, p=2, P=16, modes=SIN, a=1.0, cfl=0.1,
    mode="at", L=4, q=3, seed=0, steps=640, t_end=TWO_PI)
BURGERS_1M = Workload(
    name="burgers_1m", pde="burgers", K=1 << 20, p=4, P=1024, modes=HALF_PLUS_SIN, cfl=0.05,
    mode="at", L=4, q=2, seed=0, steps=1000)
# Courant numbers of the adjoint and large workloads are chosen inside the stability bound
# of the delayed self-feedback at PE faces (the workload statements leave them open or
# inherit values at which the common-level scheme grows).
ADJOINT_64K = Workload(
    name="adjoint_64k", pde="burgers", K=65536, p=3, P=1024, modes=HALF_PLUS_SIN, cfl=0.01,
    mode="at", L=4, q=2, seed=0, steps=2000)
ADVECTION_16M = Workload(
    name="advection_16m", pde="advection", K=1 << 24, p=3, P=16384, modes=SIN, a=1.0,
    cfl=0.002, mode="at", L=8, q=3, seed=0, steps=500)

WORKLOADS = {w.name: w for w in (ADVECTION_SMALL, BURGERS_1M, ADJOINT_64K, ADVECTION_16M)}


def random_nodal(K: int, p: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded random nodal array of shape (K, p+1), FP64, uniform in [-scale, scale]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, size=(K, p + 1))


def random_modes(rng: np.random.Generator, n: int = 4, kmax: int = 16) -> Modes:
    return Modes(amp=tuple(float(v) for v in rng.uniform(0.25, 1.0, n)),
                 kappa=tuple(float(v) for v in rng.integers(1, kmax + 1, n)),
                 phase=tuple(float(v) for v in rng.uniform(0.0, TWO_PI, n)))


def batched_instances(n: int = 512, seed: int = 0, kmin: int = 1024, kmax: int = 262144,
                      cfl: float = 0.002, elems_per_pe: int = 256) -> List[Workload]:
    """Instance list of the batched workload: K log-uniform in [kmin, kmax] rounded to a
    multiple of 256, p uniform in {1..4}, a uniform in [0.5, 2], four random modes,
    L uniform in {2..8} with uniform delays, AT order min(p+1, 3), P = K/256. The Courant
    number 0.002 and the order cap keep every instance inside the stability bound of the
    delayed self-feedback at PE faces (AT order 5 at p = 4 with delays up to 7 is not)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        K = int(round(math.exp(rng.uniform(math.log(kmin), math.log(kmax))) / 256.0)) * 256
        K = max(256, K)
        p = int(rng.integers(1, 5))
        a = float(rng.uniform(0.5, 2.0))
        L = int(rng.integers(2, 9))
        out.append(Workload(
            name=f"batch{i}", pde="advection", K=K, p=p, P=max(1, K // elems_per_pe),
            modes=random_modes(rng), a=a, cfl=cfl, mode="at", L=L, q=min(p + 1, 3),
            seed=int(rng.integers(0, 2**63 - 1)), steps=100))
    return out


def constant_table(steps: int, P: int, k: int) -> np.ndarray:
    """A delay table holding the same delay k at every step and PE face."""
    return np.full((steps, P), k, dtype=np.uint8)


def caa_table(P: int, sync_steps: int = 2, L: int = 3) -> np.ndarray:
    """Periodic communication-avoiding pattern (Section 6.3, 2D experiment): `sync_steps`
    synchronised steps followed by steps with delays 0, 1, ..., L-1. Used periodically."""
    rows = [0] * sync_steps + list(range(L))
    return np.repeat(np.array(rows, dtype=np.uint8)[:, None], P, axis=1)
