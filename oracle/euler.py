"""One-dimensional compressible Euler equations by nodal DG (oracle; test infrastructure).

What it computes (Section 6, the Sod shock-tube experiment; Eq. compressible-euler-3d in one
dimension), with the readings taken where the paper is silent:

* State U = (rho, m = rho u, E) with E = rho u^2 / 2 + p / (gamma - 1), gamma = 1.4; flux
  f(U) = (m, m u + p, (E + p) u).
* Nodal DG on the LGL nodes as for the scalar equations (oracle.dg): per element and component
      dU/dt = (2/dx) M^{-1} [ S f(U) + F_L e_0 - F_R e_p ],
  with the local Lax-Friedrichs (Rusanov) flux F = (f(U^-) + f(U^+))/2 - lambda (U^+ - U^-)/2,
  lambda = max(|u^-| + c^-, |u^+| + c^+), c = sqrt(gamma p / rho).
* PE faces: the flux is the AT sum over the common delayed level (Eq. at-flux-gen), of the
  Lax-Friedrichs flux of the stored traces (U^-, U^+) of the same stage's input.
* Time integration: strong-stability-preserving RK in Shu and Osher's form,
      v_s = Lambda( alpha_s u + beta_s (v_{s-1} + dt L(v_{s-1})) ),  v_0 = u,  u^{n+1} = v_S,
  SSP-RK2 (alpha, beta) = (0, 1), (1/2, 1/2) (the paper's scheme), SSP-RK3 as in oracle.dg,
  forward Euler (0, 1); Lambda the slope limiter below (or the identity).
* Limiter (the MUSCL / TVB-minmod slope limiter of the paper's reference): per element and
  component, with the cell average a0 and the coefficient a1 of the Legendre polynomial P_1 = xi
  of the element's polynomial (both exact integrals),
      a1' = minmod(2 a1, d+, d-) / 2,   d+ = a0^{e+1} - a0^e,   d- = a0^e - a0^{e-1},
  unless |a1| <= M dx^2 / 2 (TVB: a1 is kept); where a1' != a1 the element becomes the linear
  a0 + a1' xi, otherwise it is left as it is. At a PE face the neighbour across it is not
  used (one-sided: minmod of 2 a1 and the difference inside the PE), so the limiter needs no
  exchange.

Also the exact solution of the Riemann problem (Toro's pressure function, solved by Newton's
method) for the Sod pins. Everything in float64 (numpy / torch CPU).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Dict, Optional, Tuple

import numpy as np
import torch

from .atflux import at_coefficients_f64
from .dg import _matvec_rows
from .operators import ref_ops

F64 = torch.float64
GAMMA = 1.4

SHU_OSHER = {
    "rk1": [(0.0, 1.0)],
    "rk2": [(0.0, 1.0), (0.5, 0.5)],
    "ssprk3": [(0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0)],
}


def pressure(U):
    rho, m, E = U[0], U[1], U[2]
    return (GAMMA - 1.0) * (E - 0.5 * m * m / rho)


def flux(U):
    rho, m, E = U[0], U[1], U[2]
    u = m / rho
    p = pressure(U)
    return torch.stack([m, m * u + p, (E + p) * u])


def llf(UL, UR):
    """Local Lax-Friedrichs flux of traces UL = U^-, UR = U^+ (components first)."""
    lam = torch.maximum(torch.abs(UL[1] / UL[0]) + torch.sqrt(GAMMA * pressure(UL) / UL[0]),
                        torch.abs(UR[1] / UR[0]) + torch.sqrt(GAMMA * pressure(UR) / UR[0]))
    return 0.5 * (flux(UL) + flux(UR)) - 0.5 * lam * (UR - UL)


def conserved(rho, u, p):
    return np.stack([rho, rho * u, 0.5 * rho * u * u + p / (GAMMA - 1.0)])


@dataclass
class EulerProblem:
    K: int
    p: int
    P: int
    dt: float
    x0: float = 0.0
    x1: float = 0.02
    rk: str = "rk2"
    mode: str = "sync"           # "sync" | "adg"
    q: int = 1
    delays: Optional[np.ndarray] = None
    limiter: bool = True
    tvb_m: float = 0.0

    @property
    def dx(self) -> float:
        return (self.x1 - self.x0) / self.K


class EulerSolver:
    """Steps an EulerProblem; ``u`` is a (3, K, Np) float64 tensor."""

    def __init__(self, prob: EulerProblem, u0):
        self.prob = prob
        ops = ref_ops(prob.p)
        t = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64), dtype=F64)
        self.S, self.Minv, self.e0, self.ep = t(ops.S), t(ops.Minv), t(ops.e0), t(ops.ep)
        self.xi = t(ops.nodes)
        M = np.asarray(ops.M)
        self.avg_w = t(0.5 * M.sum(axis=0))           # a0 = sum_j avg_w[j] v_j
        self.p1_w = t(1.5 * (M @ ops.nodes))          # a1 = sum_j p1_w[j] v_j
        self.dx = prob.dx
        self.u = u0 if isinstance(u0, torch.Tensor) else t(u0)
        self.n = 0
        if prob.K % prob.P:
            raise ValueError("K must be a multiple of P")
        self.Kpe = prob.K // prob.P
        faces = np.arange(prob.K)
        is_pe = (faces % self.Kpe == 0) if prob.P > 1 else np.zeros(prob.K, bool)
        self.pe_local = torch.as_tensor(np.nonzero(is_pe)[0], dtype=torch.long)
        self.pe_index = torch.as_tensor(faces[is_pe] // self.Kpe, dtype=torch.long)
        self.history: Dict[Tuple[int, int], Tuple[torch.Tensor, torch.Tensor]] = {}
        maxdelay = int(np.max(prob.delays)) if prob.delays is not None and prob.delays.size else 0
        self.lookback = maxdelay + prob.q - 1

    def traces(self, Y):
        """(U^-, U^+) at every face f (the left face of element f): U^- = Y[:, f-1, p]."""
        return torch.roll(Y[:, :, -1], 1, dims=1), Y[:, :, 0]

    def delayed_flux(self, n: int, s: int):
        prob = self.prob
        row = prob.delays[n % prob.delays.shape[0]]
        ks = np.minimum(row[self.pe_index.numpy()].astype(np.int64), n)
        out = []
        for idx in range(self.pe_local.numel()):
            k = int(ks[idx])
            qe = min(prob.q, n - k + 1)
            c = at_coefficients_f64(k, qe)
            acc = None
            for i in range(qe):
                if c[i] == 0.0:
                    continue
                TL, TR = self.history[(n - k - i, s)]
                term = c[i] * llf(TL[:, idx], TR[:, idx])
                acc = term if acc is None else acc + term
            out.append(acc)
        return torch.stack(out, dim=1)

    def L(self, Y, n: int, s: int):
        UL, UR = self.traces(Y)
        if self.pe_local.numel() > 0:
            self.history[(n, s)] = (UL[:, self.pe_local], UR[:, self.pe_local])
        F = llf(UL, UR)
        if self.prob.mode == "adg" and self.pe_local.numel() > 0:
            F = F.clone()
            F[:, self.pe_local] = self.delayed_flux(n, s)
        FR = torch.roll(F, -1, dims=1)
        fv = flux(Y)
        out = []
        for c in range(3):
            body = _matvec_rows(self.S, fv[c]) + F[c][:, None] * self.e0[None, :] \
                - FR[c][:, None] * self.ep[None, :]
            out.append((2.0 / self.dx) * _matvec_rows(self.Minv, body))
        return torch.stack(out)

    def limit(self, V):
        prob = self.prob
        if not prob.limiter:
            return V
        a0 = (V * self.avg_w).sum(dim=2)               # (3, K)
        a1 = (V * self.p1_w).sum(dim=2)
        dp = torch.roll(a0, -1, dims=1) - a0
        dm = a0 - torch.roll(a0, 1, dims=1)
        K = prob.K
        e = torch.arange(K)
        left_pe = (e % self.Kpe == 0) if prob.P > 1 else torch.zeros(K, dtype=torch.bool)
        right_pe = ((e + 1) % self.Kpe == 0) if prob.P > 1 else torch.zeros(K, dtype=torch.bool)
        two = 2.0 * a1
        sgn = torch.sign(two)
        mag = torch.abs(two)
        ok = torch.ones_like(two, dtype=torch.bool)
        for d, skip in ((dp, right_pe), (dm, left_pe)):
            use = ~skip[None, :].expand_as(d)
            ok = ok & (~use | (torch.sign(d) == sgn))
            mag = torch.where(use, torch.minimum(mag, torch.abs(d)), mag)
        mm = torch.where(ok, sgn * mag, torch.zeros_like(mag))
        a1n = 0.5 * mm
        keep = torch.abs(a1) <= prob.tvb_m * self.dx * self.dx / 2.0
        a1n = torch.where(keep, a1, a1n)
        change = a1n != a1
        lin = a0[:, :, None] + a1n[:, :, None] * self.xi[None, None, :]
        return torch.where(change[:, :, None], lin, V)

    def step(self):
        dt, n, u = self.prob.dt, self.n, self.u
        v = u
        for s, (al, be) in enumerate(SHU_OSHER[self.prob.rk]):
            w = be * (v + dt * self.L(v, n, s))
            if al != 0.0:
                w = al * u + w
            v = self.limit(w)
        self.u = v
        self.n = n + 1
        for key in [k for k in self.history if k[0] < self.n - self.lookback - 1]:
            del self.history[key]

    def run(self, nsteps: int):
        for _ in range(nsteps):
            self.step()
        return self.u

    def integrals(self):
        """(int rho, int m, int E) = sum_e (dx/2) sum_j w_j U_j."""
        return (self.u * self.avg_w).sum(dim=(1, 2)) * self.dx


def run(prob: EulerProblem, u0, nsteps: int):
    return EulerSolver(prob, u0).run(nsteps)


# --- exact Riemann solution (Toro, Riemann Solvers and Numerical Methods, chapter 4) ---------

def _pressure_function(p, rho_k, p_k):
    """f_K(p) and its derivative: shock branch for p > p_K, rarefaction branch otherwise."""
    c_k = math.sqrt(GAMMA * p_k / rho_k)
    if p > p_k:
        A = 2.0 / ((GAMMA + 1.0) * rho_k)
        B = (GAMMA - 1.0) / (GAMMA + 1.0) * p_k
        f = (p - p_k) * math.sqrt(A / (p + B))
        df = math.sqrt(A / (B + p)) * (1.0 - (p - p_k) / (2.0 * (B + p)))
    else:
        e = (GAMMA - 1.0) / (2.0 * GAMMA)
        f = 2.0 * c_k / (GAMMA - 1.0) * ((p / p_k) ** e - 1.0)
        df = 1.0 / (rho_k * c_k) * (p / p_k) ** (-(GAMMA + 1.0) / (2.0 * GAMMA))
    return f, df


def star_state(left, right):
    """(p*, u*) of the Riemann problem with primitive states (rho, u, p): the root of
    f_L(p) + f_R(p) + u_R - u_L = 0 by Newton's method."""
    rl, ul, pl = left
    rr, ur, pr = right
    p = 0.5 * (pl + pr)
    for _ in range(100):
        fl, dfl = _pressure_function(p, rl, pl)
        fr, dfr = _pressure_function(p, rr, pr)
        dp = (fl + fr + ur - ul) / (dfl + dfr)
        p = max(p - dp, 1e-12)
        if abs(dp) < 1e-15 * p:
            break
    fl, _ = _pressure_function(p, rl, pl)
    fr, _ = _pressure_function(p, rr, pr)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(left, right, s):
    """Primitive (rho, u, p) of the exact solution at similarity coordinate s = (x - x_d) / t."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right)
    g = GAMMA
    if s <= us:   # left of the contact
        cl = math.sqrt(g * pl / rl)
        if ps > pl:   # left shock
            sl = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
            if s <= sl:
                return rl, ul, pl
            return rl * (ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1), us, ps
        csl = cl * (ps / pl) ** ((g - 1) / (2 * g))
        if s <= ul - cl:
            return rl, ul, pl
        if s >= us - csl:
            return rl * (ps / pl) ** (1 / g), us, ps
        u = 2 / (g + 1) * (cl + (g - 1) / 2 * ul + s)
        c = 2 / (g + 1) * (cl + (g - 1) / 2 * (ul - s))
        rho = rl * (c / cl) ** (2 / (g - 1))
        return rho, u, pl * (c / cl) ** (2 * g / (g - 1))
    cr = math.sqrt(g * pr / rr)
    if ps > pr:   # right shock
        sr = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
        if s >= sr:
            return rr, ur, pr
        return rr * (ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1), us, ps
    csr = cr * (ps / pr) ** ((g - 1) / (2 * g))
    if s >= ur + cr:
        return rr, ur, pr
    if s <= us + csr:
        return rr * (ps / pr) ** (1 / g), us, ps
    u = 2 / (g + 1) * (-cr + (g - 1) / 2 * ur + s)
    c = 2 / (g + 1) * (cr - (g - 1) / 2 * (ur - s))
    rho = rr * (c / cr) ** (2 / (g - 1))
    return rho, u, pr * (c / cr) ** (2 * g / (g - 1))


SOD_LEFT = (1.0, 0.0, 1.0)
SOD_RIGHT = (0.125, 0.0, 0.1)


def sod_periodic(x, t):
    """Primitive (rho, u, p) of the periodic Sod setup on [0, 0.02]: the left state of
    Eq. sod-initial on [0.005, 0.015), the right state elsewhere, so two Riemann problems sit
    0.01 apart (at 0.005 mirrored, at 0.015 as printed) and their waves do not meet for
    t <= 0.002. t = 0 gives the initial condition."""
    rho, u, p = (np.empty_like(x) for _ in range(3))
    for idx, xv in np.ndenumerate(x):
        if t == 0.0:
            st = SOD_LEFT if 0.005 <= xv < 0.015 else SOD_RIGHT
        elif xv < 0.01:   # mirrored problem at 0.005: right state on the left
            r_, u_, p_ = sample(SOD_LEFT, SOD_RIGHT, (0.005 - xv) / t)
            st = (r_, -u_, p_)
        else:
            st = sample(SOD_LEFT, SOD_RIGHT, (xv - 0.015) / t)
        rho[idx], u[idx], p[idx] = st
    return rho, u, p
