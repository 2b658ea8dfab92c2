"""The learned schedule: features, the decision rule, and phi_1 under it.

ORACLE — test infrastructure only (see oracle/__init__.py).

The plain method fixes the substep count s by a conservative a priori rule
on the spectral interval (Sec. III-C) and ends each substep's Newton
iteration by the a posteriori estimate |d_{j+1}| ||w_{j+1}|| <= tol ||p||.
The learned schedule asks a small network instead, for each candidate
s = 2^q (q = 0..Q), for the degree the estimate will need and whether it
will be met within m_max.  It takes the cheapest q the network accepts and
runs s = 2^q substeps in one of two ways:

  adaptive (the default): every substep ends, as in the plain method, at the
      first degree whose a posteriori estimate passes; m only sets how many
      Newton steps are issued before the first look at the estimate.  A
      substep that reaches m_max without passing sends the call to the plain
      method.
  fixed count: exactly m Newton steps in every substep with no test in
      between, and the estimate applied once at the end of each substep; any
      failed check sends the call to the plain method.

If the network accepts no q the plain method runs.  So an accepted result
meets the same tolerance test as the plain one.

Features of a call at candidate q (all cheap scalars the library already
has): with c = (alpha+beta)/2, gamma = (beta-alpha)/4, tau = h/2^q and
rho = max(|alpha|, |beta|):

  x0  log10(tau gamma)               x6  1 for a CSR operator, else 0
  x1  clip(c/gamma, -8, 8) / 4       x7  grid dimension / 3 (0 for CSR)
  x2  log10(tol) / 10                x8  coefficient ratio (below)
  x3  q / 10 (= log2(s)/10)          x9  log10(1 + min(Peclet, 1e30))
  x4  log10(h rho) / 3               x10 clip(log10(||v||_2/sqrt(n)), -30, 30) / 10
  x5  k (the phi index; 1 here)      x11 log10(n) / 8

Coefficient statistics, from the caller's inputs: a stencil's ratio is
mean(D)/max(D) over the grid and its Peclet number is
max over points and axes of |b_e(x)| dx_e / (2 D(x)); a CSR operator's
ratio is mean|diag|/max|diag| and its Peclet number is 0.

Decision, from the network outputs o_q = (o_q0, o_q1): the predicted degree
is mhat_q = m_max * o_q0, need_q = mhat_q (1 + rho_m) + delta_m, and q is
accepted when o_q1 >= z_min and need_q <= m_max, with
m_q = clamp(ceil(need_q), 1, m_max).  Of the accepted q the one with the
fewest operator applications 2^q (m_q + 1) - 1 is taken (ties: the smaller
q); then s = 2^q and m = m_q.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import leja as L
from . import mlp as M
from . import newton as Nw
from .operators import ShiftedOperator

Q_MAX = 12
KIND_STENCIL = 0
KIND_CSR = 1


@dataclass
class Meta:
    """Decision constants stored with a trained network."""
    z_min: float = 0.0
    rho_m: float = 0.05
    delta_m: float = 2.0
    m_max: int = 100
    q_max: int = Q_MAX


def stencil_stats(D, b, dx):
    """(ratio, peclet) of a stencil operator's inputs: D (array or scalar),
    b (one array or scalar per axis, x first), dx (per axis)."""
    D = np.asarray(D, dtype=np.float64)
    ratio = float(np.mean(D) / np.max(D))
    pe = 0.0
    for bax, dxe in zip(b, dx):
        bb = np.abs(np.asarray(bax, dtype=np.float64))
        pe = max(pe, float(np.max(bb * dxe / (2.0 * D))))
    return ratio, pe


def csr_stats(diag):
    a = np.abs(np.asarray(diag, dtype=np.float64))
    return float(np.mean(a) / np.max(a)), 0.0


def features(q, h, alpha, beta, tol, k, kind, dim, n, ratio, peclet, v_norm):
    c = 0.5 * (alpha + beta)
    gamma = 0.25 * (beta - alpha)
    tau = h / (1 << q)
    rho = max(abs(alpha), abs(beta))
    rms = v_norm / math.sqrt(n)
    lr = max(-30.0, min(30.0, math.log10(rms))) if rms > 0 else -30.0
    return np.array([
        math.log10(tau * gamma),
        max(-8.0, min(8.0, c / gamma)) / 4.0,
        math.log10(tol) / 10.0,
        q / 10.0,
        math.log10(h * rho) / 3.0,
        float(k),
        1.0 if kind == KIND_CSR else 0.0,
        (dim / 3.0) if kind == KIND_STENCIL else 0.0,
        ratio,
        math.log10(1.0 + min(peclet, 1e30)),
        lr / 10.0,
        math.log10(n) / 8.0,
    ])


def feature_table(h, alpha, beta, tol, k, kind, dim, n, ratio, peclet, v_norm, q_max=Q_MAX):
    return np.stack([features(q, h, alpha, beta, tol, k, kind, dim, n, ratio, peclet, v_norm)
                     for q in range(q_max + 1)])


def decide(outputs, meta: Meta):
    """(s, m) from the network outputs for q = 0..q_max, or None."""
    best = None
    for q in range(min(meta.q_max, len(outputs) - 1) + 1):
        o0, o1 = float(outputs[q][0]), float(outputs[q][1])
        need = meta.m_max * o0 * (1.0 + meta.rho_m) + meta.delta_m
        if o1 >= meta.z_min and need <= meta.m_max:
            m = max(1, min(meta.m_max, int(math.ceil(need))))
            cost = (1 << q) * (m + 1) - 1
            if best is None or cost < best[0]:
                best = (cost, 1 << q, m)
    return None if best is None else (best[1], best[2])


@dataclass
class LearnedStats:
    s: int = 0
    m: int = 0
    accepted: bool = False      # the proposal passed every substep's check
    proposed: bool = False      # the network accepted some q
    plain: object = None        # Stats of the plain fallback, when taken
    degrees: list = None        # per substep, of the proposal's attempt


def phi1_learned(op, h, v, tol, theta, meta: Meta, kind, dim, ratio, peclet, xi=None,
                 sizes=M.SIZES, fixed=False):
    """h phi_1(hA) v under the learned schedule (adaptive, or fixed count);
    falls back to the plain method.  The network is evaluated in FP32, the
    precision of the library's inference kernel.  Returns (y, LearnedStats)."""
    ls = LearnedStats()
    v = np.asarray(v, dtype=np.float64).reshape(op.shape)
    alpha, beta = op.gershgorin()
    gamma = 0.25 * (beta - alpha)
    vn = float(np.sqrt(np.sum(v * v)))
    if gamma > 0 and vn > 0:
        X = feature_table(h, alpha, beta, tol, 1, kind, dim, v.size, ratio, peclet, vn,
                          meta.q_max)
        O = M.forward(theta, X.astype(np.float32), sizes, dtype=np.float32)
        sm = decide(O, meta)
        if sm is not None:
            ls.proposed = True
            ls.s, ls.m = sm
            if fixed:
                y, ok = Nw.h_phi1_fixed(op, h, v, tol, ls.s, ls.m, Nw.Stats(), xi)
                ls.degrees = [ls.m] * ls.s
            else:
                y, ls.degrees, ok = Nw.h_phi1_at(op, h, v, tol, ls.s, meta.m_max, xi)
            if ok:
                ls.accepted = True
                return y, ls
    st = Nw.Stats()
    y = Nw.h_phi1_substeps(op, h, v, tol, st, xi=xi)
    ls.plain = st
    return y, ls


def exp_step_learned(op, u, h, tol, theta, meta, kind, dim, ratio, peclet, rosenbrock=True,
                     nonlin=Nw.NONLIN_LOGISTIC, xi=None, fixed=False):
    """One exponential Euler (rosenbrock=False) or Rosenbrock-Euler step with
    phi_1 under the learned schedule."""
    u = np.asarray(u, dtype=np.float64).reshape(op.shape)
    g, dg = Nw.nonlinearity(u, nonlin)
    F = op.matvec(u) + g
    J = ShiftedOperator(op, dg) if rosenbrock else op
    y, ls = phi1_learned(J, h, F, tol, theta, meta, kind, dim, ratio, peclet, xi, fixed=fixed)
    return u + y, ls
