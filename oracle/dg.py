"""Fully discrete DG / ADG / ADG-AT solver in FP64 (oracle; test infrastructure).

What it computes, with the readings taken where the paper is silent:

* Mesh (Section 2): K uniform elements of width dx = (x1 - x0)/K on a periodic domain;
  element e spans [x0 + e dx, x0 + (e+1) dx]; node i of element e sits at
  x0 + e dx + (1 + xi_i) dx / 2 with xi the LGL nodes. Initial data are nodal values.
* Semi-discrete operator (Eqs. DGweakform, DGscheme): with f(u) collocated at the nodes,
      du^e/dt = (2/dx) M^{-1} [ S f(u^e) + e_0 F_L^e - e_p F_R^e ],
  where F_L^e, F_R^e are the numerical fluxes at the left and right faces of element e.
  For f = a u and F = a (B+ u^- + B- u^+) this is Eq. DGscheme term by term.
* Numerical fluxes: upwind (Section 6.1: a u^- for a >= 0, a u^+ for a < 0) for linear
  advection; local Lax-Friedrichs (Section 6.1) with lambda = max(|u^-|, |u^+|) for
  inviscid Burgers f = u^2/2.
* Viscous Burgers u_t + (u^2/2)_x = nu u_xx (Eq. burgers, nu > 0) by the local DG method
  (Section 6: Lax-Friedrichs for the advective term, alternating fluxes for the viscous
  one): q = u_x in the weak sense, element by element
      q^e = (2/dx) M^{-1} [ -S u^e + uhat_R e_p - uhat_L e_0 ],      uhat = u^- ,
  and the viscous term adds nu [ -S q^e + qhat_R e_p - qhat_L e_0 ] to the bracket above,
  qhat = q^+ (the alternating pair). At a PE face all three face values (uhat, the
  Lax-Friedrichs flux, qhat) come from the common delayed level through the AT sum.
* PE decomposition (Section 2, Fig. 2): P contiguous blocks of K/P elements; the face
  between elements e-1 and e is a PE face iff they lie in different PEs (none for P = 1).
  PE face j sits at element j K/P.
* Delays (Section 3): delay k = D[n][j] for step n at PE face j, clamped to k <= n at the
  start. Both elements of the face use the common level n - k (Eq. asyncEulerDGconserved),
  so the flux is single-valued. ``mode="naive"`` instead lets each side use its own delay
  (Eq. asyncEulerDG) and is kept only to show the loss of conservation.
* AT flux (Section 5, Eq. at-flux-gen): F = sum_{i<q'} c_i(k; q') fhat(T_{n-k-i}) with
  q' = min(q, n - k + 1); q = 1 is the standard delayed flux.
* Inside a Runge-Kutta step the delayed face values of stage s are the stage-s inputs of
  the delayed step (stage-consistent reading of Eq. async-dg2-rk2-l2).
* Time integration: explicit Runge-Kutta in Butcher form, Y_s = u + dt sum_j a_sj k_j,
  k_s = L(Y_s), u+ = u + dt sum_s b_s k_s. The low-storage (2N) schemes of Section 6 enter
  through their Butcher form (``two_register_tableau``); their stage inputs are the U_{s-1}
  of the 2N recurrence.

Everything runs in torch float64 on the CPU, vectorised over elements, so that
``gradient`` can take the exact discrete gradient by automatic differentiation.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, Optional, Tuple

import numpy as np
import torch

from .atflux import at_coefficients_f64
from .operators import ref_ops

F64 = torch.float64

def two_register_tableau(A, B):
    """Butcher form (a, b) of a 2N-storage Runge-Kutta scheme in Williamson's form,
        dU_s = A_s dU_{s-1} + dt L(U_{s-1}),   U_s = U_{s-1} + B_s dU_s,   s = 1 .. S, A_1 = 0,
    U_0 = u^n, u^{n+1} = U_S. With k_j = L(U_{j-1}) the recurrence unrolls to
        dU_s = dt sum_{j<=s} (A_{j+1} ... A_s) k_j,
        U_s = U_0 + dt sum_{j<=s} k_j sum_{r=j}^{s} B_r (A_{j+1} ... A_r),
    so stage s+1 (input U_s) has a_{s+1,j} = sum_{r=j}^{s} B_r A_{j+1} ... A_r and b_j is the
    same sum for s = S. A and B may be Fractions (exact) or floats; entries keep their type."""
    S = len(A)

    def coef(s, j):   # weight of dt k_j (0-based j) in U_s
        tot = 0
        for r in range(j, s):
            prod = 1
            for m in range(j + 1, r + 1):
                prod = prod * A[m]
            tot = tot + B[r] * prod
        return tot

    a = [[coef(s, j) if j < s else 0 for j in range(S)] for s in range(S)]
    b = [coef(S, j) for j in range(S)]
    return a, b


# Low-storage schemes of the kind the paper's experiments use (Section 6, after Williamson
# 1980 and Kennedy et al. 2000); their published 2N coefficients (A_s, B_s).
from fractions import Fraction as _Fr  # noqa: E402

TWO_REGISTER = {
    # Williamson's three-stage, third-order scheme.
    "lsrk3": ([_Fr(0), _Fr(-5, 9), _Fr(-153, 128)], [_Fr(1, 3), _Fr(15, 16), _Fr(8, 15)]),
    # Carpenter and Kennedy's five-stage, fourth-order scheme.
    "lsrk4": ([_Fr(0), _Fr(-567301805773, 1357537059087), _Fr(-2404267990393, 2016746695238),
               _Fr(-3550918686646, 2091501179385), _Fr(-1275806237668, 842570457699)],
              [_Fr(1432997174477, 9575080441755), _Fr(5161836677717, 13612068292357),
               _Fr(1720146321549, 2090206949498), _Fr(3134564353537, 4481467310338),
               _Fr(2277821191437, 14882151754819)]),
}


def _float_tableau(ab):
    a, b = ab
    return [[float(x) for x in row] for row in a], [float(x) for x in b]


# Butcher tableaux (a, b).
TABLEAUX = {
    # Forward Euler, Eq. EulerDG.
    "rk1": ([[0.0]], [1.0]),
    # Two-stage RK of Eq. dg2-rk2: k1 = dt L(u), k2 = dt L(u + k1), u+ = u + (k1 + k2)/2.
    "rk2": ([[0.0, 0.0], [1.0, 0.0]], [0.5, 0.5]),
    # Three-stage strong-stability-preserving RK (Shu and Osher), in Butcher form.
    "ssprk3": ([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.25, 0.25, 0.0]],
               [1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0]),
    # Classical fourth-order RK.
    "rk4": ([[0.0, 0.0, 0.0, 0.0], [0.5, 0.0, 0.0, 0.0], [0.0, 0.5, 0.0, 0.0],
             [0.0, 0.0, 1.0, 0.0]], [1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0]),
    # The 2N schemes above, in Butcher form.
    "lsrk3": _float_tableau(two_register_tableau(*TWO_REGISTER["lsrk3"])),
    "lsrk4": _float_tableau(two_register_tableau(*TWO_REGISTER["lsrk4"])),
}


@dataclass
class Problem:
    pde: str                     # "advection" | "burgers"
    K: int
    p: int
    P: int
    dt: float
    a: float = 1.0
    x0: float = 0.0
    x1: float = 2.0 * math.pi
    rk: str = "ssprk3"
    mode: str = "sync"           # "sync" | "adg" | "naive"
    q: int = 1                   # AT order (1 = standard flux)
    delays: Optional[np.ndarray] = None        # (T, P) uint8, row n mod T at step n
    delays_minus: Optional[np.ndarray] = None  # naive mode: delay seen by the right element
    window_lo: Optional[int] = None            # window mode: global index of local element 0
    K_global: Optional[int] = None             # window mode: elements of the full mesh
    nu: float = 0.0                            # Burgers viscosity (LDG for nu > 0)

    @property
    def dx(self) -> float:
        Kg = self.K_global if self.K_global is not None else self.K
        return (self.x1 - self.x0) / Kg


def dt_from_cfl(pde: str, cfl: float, dx: float, a: float, u0: np.ndarray) -> float:
    """Fixed time step from the Courant number sigma = a dt / dx (Section 2); for Burgers
    the speed is max |u0|. Evaluated as (cfl * dx) / speed."""
    speed = abs(a) if pde == "advection" else float(np.max(np.abs(u0)))
    return (cfl * dx) / speed


def node_coordinates(K: int, p: int, x0: float, x1: float, e_lo: int = 0, K_global=None):
    ops = ref_ops(p)
    Kg = K_global if K_global is not None else K
    dx = (x1 - x0) / Kg
    e = np.arange(e_lo, e_lo + K, dtype=np.float64)[:, None]
    return x0 + e * dx + (1.0 + ops.nodes[None, :]) * (dx / 2.0)


def modes_initial(modes, K: int, p: int, x0: float = 0.0, x1: float = 2.0 * math.pi,
                  e_lo: int = 0, K_global=None) -> np.ndarray:
    """Nodal values of u0 = offset + sum A sin(kappa x + phi) (Eq. initialcond)."""
    x = node_coordinates(K, p, x0, x1, e_lo, K_global)
    u = np.full_like(x, float(modes.offset))
    for A, kap, ph in zip(modes.amp, modes.kappa, modes.phase):
        u = u + A * np.sin(kap * x + ph)
    return u


def _matvec_rows(A: torch.Tensor, X: torch.Tensor) -> torch.Tensor:
    """Y[e, i] = sum_j A[i, j] X[e, j], summed in the order j = 0, 1, ... per element."""
    Np = A.shape[1]
    cols = []
    for i in range(A.shape[0]):
        acc = A[i, 0] * X[:, 0]
        for j in range(1, Np):
            acc = acc + A[i, j] * X[:, j]
        cols.append(acc)
    return torch.stack(cols, dim=1)


class Solver:
    """Steps a Problem. ``u`` is a (K, Np) float64 tensor; ``n`` the global step index."""

    def __init__(self, prob: Problem, u0):
        self.prob = prob
        ops = ref_ops(prob.p)
        self.ops = ops
        t = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64), dtype=F64)
        self.S = t(ops.S)
        self.Minv = t(ops.Minv)
        self.M = t(ops.M)
        self.e0 = t(ops.e0)
        self.ep = t(ops.ep)
        self.w = t(ops.weights)
        self.dx = prob.dx
        self.u = u0 if isinstance(u0, torch.Tensor) else t(u0)
        self.n = 0
        self.tab_a, self.tab_b = TABLEAUX[prob.rk]
        Kg = prob.K_global if prob.K_global is not None else prob.K
        if Kg % prob.P != 0:
            raise ValueError("K must be a multiple of P")
        self.Kpe = Kg // prob.P
        self.window = prob.window_lo is not None
        lo = prob.window_lo or 0
        # Local face f is the left face of local element f (global face lo + f).
        gfaces = np.arange(lo, lo + prob.K)
        if prob.P > 1:
            is_pe = (gfaces % self.Kpe) == 0
        else:
            is_pe = np.zeros(prob.K, dtype=bool)
        self.pe_local = torch.as_tensor(np.nonzero(is_pe)[0], dtype=torch.long)
        self.pe_index = torch.as_tensor((gfaces[is_pe] // self.Kpe) % prob.P, dtype=torch.long)
        self.history: Dict[Tuple[int, int], Tuple[torch.Tensor, torch.Tensor]] = {}
        maxdelay = 0
        for tbl in (prob.delays, prob.delays_minus):
            if tbl is not None and tbl.size:
                maxdelay = max(maxdelay, int(np.max(tbl)))
        self.lookback = maxdelay + prob.q - 1
        self._coef = {}

    # --- fluxes -------------------------------------------------------------------------
    def f(self, u):
        if self.prob.pde == "advection":
            return self.prob.a * u
        return 0.5 * u * u

    def fhat(self, uL, uR):
        if self.prob.pde == "advection":
            a = self.prob.a
            return a * uL if a >= 0 else a * uR
        lam = torch.maximum(torch.abs(uL), torch.abs(uR))
        return 0.5 * (self.f(uL) + self.f(uR)) - 0.5 * lam * (uR - uL)

    def coef(self, k: int, q: int):
        key = (k, q)
        if key not in self._coef:
            self._coef[key] = at_coefficients_f64(k, q)
        return self._coef[key]

    # --- one semi-discrete evaluation -----------------------------------------------------
    def traces(self, Y):
        """(u^-, u^+) at every local face f: u^- = Y[f-1, p], u^+ = Y[f, 0]."""
        uL = torch.roll(Y[:, -1], 1)
        uR = Y[:, 0]
        if self.window:
            uL = torch.cat([Y[:1, 0], uL[1:]])
        return uL, uR

    def delay(self, table, n: int, j: torch.Tensor):
        row = table[n % table.shape[0]]
        return np.minimum(row[j.numpy()].astype(np.int64), n)

    def delayed_flux(self, n: int, s: int, side: int, table, q: int):
        """Flux at the PE faces from stored levels. side 0: both traces from the common
        delayed level; side +1 / -1 (naive): only the far trace is delayed."""
        P_loc = self.pe_local.numel()
        ks = self.delay(table, n, self.pe_index)
        out = []
        for idx in range(P_loc):
            k = int(ks[idx])
            qe = min(q, n - k + 1)
            c = self.coef(k, qe)
            acc = None
            for i in range(qe):
                if c[i] == 0.0:
                    continue
                TL, TR = self.history[(n - k - i, s)][:2]
                uL, uR = TL[idx], TR[idx]
                if side == +1:      # left element's view: own u^- current, far u^+ delayed
                    uL = self.history[(n, s)][0][idx]
                elif side == -1:    # right element's view: far u^- delayed, own u^+ current
                    uR = self.history[(n, s)][1][idx]
                term = c[i] * self.fhat(uL, uR)
                acc = term if acc is None else acc + term
            out.append(acc)
        return torch.stack(out)

    def delayed_value(self, n: int, s: int, pick, table, q: int):
        """AT sum over the stored levels at the PE faces of one stored face quantity: pick maps
        a stored entry (u^-, u^+, q^+) to its value (common delayed level)."""
        ks = self.delay(table, n, self.pe_index)
        out = []
        for idx in range(self.pe_local.numel()):
            k = int(ks[idx])
            qe = min(q, n - k + 1)
            c = self.coef(k, qe)
            acc = None
            for i in range(qe):
                if c[i] == 0.0:
                    continue
                term = c[i] * pick(self.history[(n - k - i, s)], idx)
                acc = term if acc is None else acc + term
            out.append(acc)
        return torch.stack(out)

    def ldg_q(self, Y, uL, n: int, s: int):
        """q = u_x of the local DG method with uhat = u^- (delayed / AT at PE faces)."""
        prob = self.prob
        uhat = uL
        if prob.mode == "adg" and self.pe_local.numel() > 0:
            uhat = uL.index_put((self.pe_local,), self.delayed_value(
                n, s, lambda h, i: h[0][i], prob.delays, prob.q))
        uhat_R = torch.roll(uhat, -1)
        if self.window:
            uhat_R = torch.cat([uhat_R[:-1], Y[-1:, -1]])
        body = -_matvec_rows(self.S, Y) + uhat_R[:, None] * self.ep[None, :] \
            - uhat[:, None] * self.e0[None, :]
        return (2.0 / self.dx) * _matvec_rows(self.Minv, body)

    def L(self, Y, n: int, s: int):
        prob = self.prob
        uL, uR = self.traces(Y)
        viscous = prob.pde == "burgers" and prob.nu != 0.0
        if viscous and prob.mode == "naive":
            raise ValueError("the viscous operator takes the common-level scheme")
        Q = None
        if self.pe_local.numel() > 0:   # the current level's traces (q^+ once it is formed)
            self.history[(n, s)] = (uL[self.pe_local], uR[self.pe_local], None)
        if viscous:
            Q = self.ldg_q(Y, uL, n, s)
            if self.pe_local.numel() > 0:
                self.history[(n, s)] = (uL[self.pe_local], uR[self.pe_local], Q[self.pe_local, 0])
        F = self.fhat(uL, uR)
        FL_view = F          # flux used by element f at its left face f
        FR_view = F          # flux used by element f-1 at its right face f
        if prob.mode != "sync" and self.pe_local.numel() > 0:
            if prob.mode == "adg":
                Fpe = self.delayed_flux(n, s, 0, prob.delays, prob.q)
                FL_view = F.index_put((self.pe_local,), Fpe)
                FR_view = FL_view
            elif prob.mode == "naive":
                Fr = self.delayed_flux(n, s, -1, prob.delays_minus, 1)
                Fl = self.delayed_flux(n, s, +1, prob.delays, 1)
                FL_view = F.index_put((self.pe_local,), Fr)
                FR_view = F.index_put((self.pe_local,), Fl)
            else:
                raise ValueError(prob.mode)
        FR = torch.roll(FR_view, -1)
        if self.window:
            last = self.fhat(Y[-1:, -1], Y[-1:, -1])
            FR = torch.cat([FR[:-1], last])
        fv = self.f(Y)
        body = _matvec_rows(self.S, fv) + FL_view[:, None] * self.e0[None, :] \
            - FR[:, None] * self.ep[None, :]
        if viscous:
            qhat = Q[:, 0]                     # q^+ at every face f: Q[f, 0]
            if prob.mode == "adg" and self.pe_local.numel() > 0:
                qhat = qhat.index_put((self.pe_local,), self.delayed_value(
                    n, s, lambda h, i: h[2][i], prob.delays, prob.q))
            qhat_R = torch.roll(qhat, -1)
            if self.window:
                qhat_R = torch.cat([qhat_R[:-1], Q[-1:, -1]])
            body = body + prob.nu * (-_matvec_rows(self.S, Q) + qhat_R[:, None] * self.ep[None, :]
                                     - qhat[:, None] * self.e0[None, :])
        return (2.0 / self.dx) * _matvec_rows(self.Minv, body)

    # --- time stepping -------------------------------------------------------------------
    def step(self):
        dt = self.prob.dt
        n = self.n
        u = self.u
        ks = []
        for s in range(len(self.tab_b)):
            Y = u
            for j in range(s):
                if self.tab_a[s][j] != 0.0:
                    Y = Y + (dt * self.tab_a[s][j]) * ks[j]
            ks.append(self.L(Y, n, s))
        unew = u
        for s, bs in enumerate(self.tab_b):
            unew = unew + (dt * bs) * ks[s]
        self.u = unew
        self.n = n + 1
        drop = [key for key in self.history if key[0] < self.n - self.lookback - 1]
        for key in drop:
            del self.history[key]

    def run(self, nsteps: int):
        for _ in range(nsteps):
            self.step()
        return self.u

    # --- diagnostics ---------------------------------------------------------------------
    def integral(self, u=None):
        """Discrete integral of u_h: sum_e (dx/2) w^T u^e (exact for the LGL quadrature of
        M 1 = w, i.e. int u_h = (dx/2) 1^T M u^e)."""
        u = self.u if u is None else u
        return (self.dx / 2.0) * torch.sum(u @ self.w)


def run(prob: Problem, u0, nsteps: int):
    s = Solver(prob, u0)
    s.run(nsteps)
    return s.u


def misfit(prob: Problem, u, g):
    """J = 1/2 sum_e (dx/2) (u^e - g^e)^T M (u^e - g^e): the L2 misfit of the final field."""
    ops = ref_ops(prob.p)
    M = torch.as_tensor(ops.M, dtype=F64)
    d = u - g
    return 0.5 * (prob.dx / 2.0) * torch.sum((d @ M) * d)


def gradient(prob: Problem, u0: np.ndarray, g: np.ndarray, nsteps: int):
    """(J, dJ/du0) of the misfit after nsteps, by reverse-mode automatic differentiation of
    the forward solver above (delays are data and are not differentiated)."""
    x = torch.tensor(np.asarray(u0), dtype=F64, requires_grad=True)
    uN = run(prob, x, nsteps)
    J = misfit(prob, uN, torch.as_tensor(np.asarray(g), dtype=F64))
    J.backward()
    return float(J.detach()), x.grad.detach().numpy()
