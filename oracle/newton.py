"""The Leja/Newton iteration for phi_k(hA)v and the two exponential steps.

ORACLE — test infrastructure only (see oracle/__init__.py).

Paper anchors: the exponential Euler method (Eq. (2)), matrix functions by
polynomial interpolation at Leja points reduced to repeated products
(alpha*A + beta*I)x (Eq. (3), Sec. II-C and Sec. III-C).  The loop below
writes out the Newton form of that interpolant:

    w_0 = r,  p_0 = d_0 w_0,
    w_{j+1} = (A w_j)/gamma - (c/gamma + xi_j) w_j      (an Eq. (3) product)
    p_{j+1} = p_j + d_{j+1} w_{j+1},
    stop when |d_{j+1}| * ||w_{j+1}||_2 <= tol * ||p_{j+1}||_2,

and, where s > 1 substeps are needed, integrates y' = A y + v from y = 0
(y(h) = h phi_1(hA) v exactly):  y_{i+1} = y_i + tau * phi_1(tau A)(A y_i + v);
for k >= 2 the forcing t^{k-1}/(k-1)! v, two Newton runs per substep
(h_phik_substeps).
Readings where the paper is silent: the tolerance applies per substep and is
relative to ||p||; a substep that reaches m_max without meeting it doubles s
and restarts; ||v|| = 0 returns 0; gamma = 0 (A = cI) returns phi_k(hc) v.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import leja as L
from .operators import ShiftedOperator

NONLIN_NONE = 0
NONLIN_LOGISTIC = 1
NONLIN_COMBUSTION = 2
# below this u the combustion term and its derivative are 0 (their limit as
# u -> 0+; in FP64 the exponential already underflows to 0 there)
COMBUSTION_CUT = 0.025


class NotConverged(RuntimeError):
    pass


@dataclass
class Stats:
    alpha: float = 0.0
    beta: float = 0.0
    s: int = 1
    degrees: list = field(default_factory=list)   # Newton degree per substep (final attempt)
    matvecs: int = 0
    restarts: int = 0
    m_sched: int = 0


def _norm(x):
    return float(np.sqrt(np.sum(x * x)))


def newton_phi(op, r, d, xi, c, gamma, tol, m_max, stats):
    """p ~= phi_k(tau A) r for the divided differences d of phi_k(tau*(c+gamma*xi)).
    Returns (p, degree, converged)."""
    if _norm(r) == 0.0:
        return np.zeros_like(r), 0, True
    w = r.copy()
    p = d[0] * w
    for j in range(m_max):
        shift = c / gamma + xi[j]
        w = op.matvec(w) / gamma - shift * w
        stats.matvecs += 1
        p = p + d[j + 1] * w
        if abs(d[j + 1]) * _norm(w) <= tol * _norm(p):
            return p, j + 1, True
    return p, m_max, False


def _interval(op):
    alpha, beta = op.gershgorin()
    return alpha, beta, 0.5 * (alpha + beta), 0.25 * (beta - alpha)


def h_phi1_substeps(op, h, v, tol, stats, m_max=L.M_MAX, xi=None):
    """y_s ~= h * phi_1(hA) v by s substeps of y' = A y + v from y = 0."""
    alpha, beta, c, gamma = _interval(op)
    stats.alpha, stats.beta = alpha, beta
    v = np.asarray(v, dtype=np.float64).reshape(op.shape)
    if _norm(v) == 0.0:
        stats.s, stats.degrees = 1, [0]
        return np.zeros_like(v)
    if gamma == 0.0:
        stats.s, stats.degrees = 1, [0]
        return h * L.phi_scalar(1, h * c) * v
    if xi is None:
        xi = L.leja_points(m_max)
    s, stats.m_sched, _ = L.plain_schedule(1, h, c, gamma, tol, xi, m_max)
    while s <= L.S_MAX:
        tau = h / s
        d = L.divided_differences(1, tau, c, gamma, xi[: m_max + 1])
        y = np.zeros_like(v)
        degrees = []
        ok = True
        for i in range(s):
            if i == 0:
                r = v.copy()
            else:
                r = op.matvec(y) + v
                stats.matvecs += 1
            p, deg, conv = newton_phi(op, r, d, xi, c, gamma, tol, m_max, stats)
            degrees.append(deg)
            if not conv:
                ok = False
                break
            y = y + tau * p
        if ok:
            stats.s, stats.degrees = s, degrees
            return y
        stats.restarts += 1
        s *= 2
    raise NotConverged("phi_1: no s <= S_MAX converged")


def newton_phi_fixed(op, r, d, xi, c, gamma, tol, m, stats):
    """Exactly m Newton steps with no test in between; then the estimate of
    the last step decides: ok = |d_m| ||w_m|| <= tol ||p_m||.  Returns (p, ok).
    The iterates are those of newton_phi; only the stopping differs."""
    if _norm(r) == 0.0:
        return np.zeros_like(r), True
    w = r.copy()
    p = d[0] * w
    for j in range(m):
        shift = c / gamma + xi[j]
        w = op.matvec(w) / gamma - shift * w
        stats.matvecs += 1
        p = p + d[j + 1] * w
    ok = abs(d[m]) * _norm(w) <= tol * _norm(p)
    return p, ok


def h_phi1_fixed(op, h, v, tol, s, m, stats, xi=None):
    """y ~= h phi_1(hA) v with a given substep count s and exactly m Newton
    steps in every substep; ok = every substep's final estimate passed.
    Returns (y, ok).  gamma > 0 and ||v|| > 0 are the caller's to check."""
    alpha, beta, c, gamma = _interval(op)
    stats.alpha, stats.beta = alpha, beta
    v = np.asarray(v, dtype=np.float64).reshape(op.shape)
    if xi is None:
        xi = L.leja_points(L.M_MAX)
    tau = h / s
    d = L.divided_differences(1, tau, c, gamma, xi[: m + 1])
    y = np.zeros_like(v)
    ok_all = True
    for i in range(s):
        if i == 0:
            r = v.copy()
        else:
            r = op.matvec(y) + v
            stats.matvecs += 1
        p, ok = newton_phi_fixed(op, r, d, xi, c, gamma, tol, m, stats)
        ok_all = ok_all and ok
        y = y + tau * p
    stats.s, stats.degrees = s, [m] * s
    return y, ok_all


def h_phi1_at(op, h, v, tol, s, m_max=L.M_MAX, xi=None):
    """The a posteriori iteration at a given s with no restart: returns
    (y, degrees, converged) where converged says every substep met the
    tolerance within m_max steps (degrees then lists them)."""
    stats = Stats()
    alpha, beta, c, gamma = _interval(op)
    v = np.asarray(v, dtype=np.float64).reshape(op.shape)
    if xi is None:
        xi = L.leja_points(m_max)
    tau = h / s
    d = L.divided_differences(1, tau, c, gamma, xi[: m_max + 1])
    y = np.zeros_like(v)
    degrees = []
    for i in range(s):
        r = v.copy() if i == 0 else op.matvec(y) + v
        p, deg, conv = newton_phi(op, r, d, xi, c, gamma, tol, m_max, stats)
        degrees.append(deg)
        if not conv:
            return y, degrees, False
        y = y + tau * p
    return y, degrees, True


def h_phik_substeps(op, k, h, v, tol, stats, m_max=L.M_MAX, xi=None, fixed_s=None):
    """y_s ~= h^k phi_k(hA) v, k >= 2, by s substeps of y' = A y + t^{k-1}/(k-1)! v
    from y = 0 (y(t) = t^k phi_k(tA) v).  A substep of length tau from t_i is
    exactly (variation of constants on the polynomial forcing)
        y_{i+1} = e^{tau A} y_i + psi_i(tau A) v,
        psi_i(z) = sum_{j=1..k} t_i^{k-j}/(k-j)! tau^j phi_j(z),
    a sum of positive multiples of phi_j, so one Newton run with the divided
    differences of psi_i (the same combination of the phi_j tables) gives the
    second term, and one run of phi_0 = exp the first: two runs per substep, no
    products with A outside the Newton loop (an expansion of phi_j in powers of
    A would amplify rounding by (tau rho)^k).  The first substep is psi_0 =
    tau^k phi_k alone.  Reading: the a-priori rule of phi_k at h picks s; a run
    reaching m_max doubles s.  stats.degrees holds the two runs' degrees summed
    per substep."""
    alpha, beta, c, gamma = _interval(op)
    stats.alpha, stats.beta = alpha, beta
    v = np.asarray(v, dtype=np.float64).reshape(op.shape)
    if xi is None:
        xi = L.leja_points(m_max)
    if fixed_s:
        s = int(fixed_s)
    else:
        s, stats.m_sched, _ = L.plain_schedule(k, h, c, gamma, tol, xi, m_max)
    while s <= L.S_MAX:
        tau = h / s
        dj = [L.divided_differences(j, tau, c, gamma, xi[: m_max + 1]) for j in range(k + 1)]
        y = np.zeros_like(v)
        degrees = []
        ok = True
        p_first = None
        for i in range(s):
            ti = i * tau
            dpsi = sum((ti ** (k - j) / math.factorial(k - j)) * tau ** j * dj[j]
                       for j in range(1, k + 1))
            deg = 0
            if i > 0:
                e, d0, conv = newton_phi(op, y, dj[0], xi, c, gamma, tol, m_max, stats)
                deg += d0
                if not conv:
                    ok = False
                    break
            q, d1, conv = newton_phi(op, v, dpsi, xi, c, gamma, tol, m_max, stats)
            deg += d1
            degrees.append(deg)
            if not conv:
                ok = False
                break
            if i == 0:
                p_first = q
                y = q
            else:
                y = e + q
        if ok:
            stats.s, stats.degrees = s, degrees
            return y, p_first
        if fixed_s:
            raise NotConverged("phi_k: the fixed s did not converge")
        stats.restarts += 1
        s *= 2
    raise NotConverged("phi_k: no s <= S_MAX converged")


def phi_apply(op, k, h, v, tol, m_max=L.M_MAX, xi=None, fixed_s=None):
    """phi_k(hA) v.  k = 1: substepped ODE form; k = 0: (e^{tau A})^s v;
    k >= 2: h_phik_substeps (with s = 1 the Newton sum itself).  fixed_s
    (k >= 2): run that s, no schedule.  Returns (result, Stats)."""
    stats = Stats()
    v = np.asarray(v, dtype=np.float64).reshape(op.shape)
    if k == 1:
        y = h_phi1_substeps(op, h, v, tol, stats, m_max, xi)
        return y / h, stats
    alpha, beta, c, gamma = _interval(op)
    stats.alpha, stats.beta = alpha, beta
    if _norm(v) == 0.0:
        stats.degrees = [0]
        return np.zeros_like(v), stats
    if gamma == 0.0:
        stats.degrees = [0]
        return L.phi_scalar(k, h * c) * v, stats
    if xi is None:
        xi = L.leja_points(m_max)
    if k >= 2:
        y, p1 = h_phik_substeps(op, k, h, v, tol, stats, m_max, xi, fixed_s)
        return (p1 / h ** k if stats.s == 1 else y / h ** k), stats
    s, stats.m_sched, _ = L.plain_schedule(k, h, c, gamma, tol, xi, m_max)
    while s <= L.S_MAX:
        tau = h / s
        d = L.divided_differences(k, tau, c, gamma, xi[: m_max + 1])
        y = v.copy()
        degrees = []
        ok = True
        for _ in range(s):
            y, deg, conv = newton_phi(op, y, d, xi, c, gamma, tol, m_max, stats)
            degrees.append(deg)
            if not conv:
                ok = False
                break
        if ok:
            stats.s, stats.degrees = s, degrees
            return y, stats
        stats.restarts += 1
        s *= 2
    raise NotConverged("phi_k: no s <= S_MAX converged")


def combustion(u):
    """The combustion model's reaction term (Sec. III-C, the nonlinearity
    evaluated pointwise on the GPU): g(u) = (2 - u) exp(20 (1 - 1/u)) / 4, and
    its derivative g'(u) = exp(20 (1 - 1/u)) (20 (2 - u) / u^2 - 1) / 4 (the
    product rule).  Reading: for u <= COMBUSTION_CUT both are 0."""
    u = np.asarray(u, dtype=np.float64)
    g = np.zeros_like(u)
    dg = np.zeros_like(u)
    m = u > COMBUSTION_CUT
    um = u[m]
    e = np.exp(20.0 * (1.0 - 1.0 / um))
    g[m] = 0.25 * (2.0 - um) * e
    dg[m] = 0.25 * e * (20.0 * (2.0 - um) / (um * um) - 1.0)
    return g, dg


def nonlinearity(u, kind):
    """g(u) and g'(u): none (0, 0), logistic u(1-u), 1-2u, or the combustion
    term of Sec. III-C."""
    if kind == NONLIN_LOGISTIC:
        return u * (1.0 - u), 1.0 - 2.0 * u
    if kind == NONLIN_COMBUSTION:
        return combustion(u)
    return np.zeros_like(u), np.zeros_like(u)


def exp_euler_step(op, u, h, tol, nonlin=NONLIN_NONE, xi=None, bvec=None):
    """Eq. (2) with A -> -A:  u_{n+1} = e^{hA}u_n + h phi_1(hA) g(u_n)
    = u_n + h phi_1(hA)(A u_n + g(u_n)).  bvec: the constant forcing b_D of
    inhomogeneous Dirichlet data (StencilOperator.boundary_vector), added to
    A u_n + g(u_n)."""
    stats = Stats()
    u = np.asarray(u, dtype=np.float64).reshape(op.shape)
    g, _ = nonlinearity(u, nonlin)
    F = op.matvec(u) + g
    if bvec is not None:
        F = F + np.asarray(bvec, dtype=np.float64).reshape(op.shape)
    stats.matvecs += 1
    return u + h_phi1_substeps(op, h, F, tol, stats, xi=xi), stats


def exp_rosenbrock_step(op, u, h, tol, nonlin=NONLIN_LOGISTIC, xi=None, bvec=None):
    """Exponential Rosenbrock-Euler: J_n = A + diag(g'(u_n)),
    u_{n+1} = u_n + h phi_1(h J_n)(A u_n + b_D + g(u_n)); bvec = b_D as in
    exp_euler_step (a constant forcing: J_n is unchanged)."""
    stats = Stats()
    u = np.asarray(u, dtype=np.float64).reshape(op.shape)
    g, dg = nonlinearity(u, nonlin)
    F = op.matvec(u) + g
    if bvec is not None:
        F = F + np.asarray(bvec, dtype=np.float64).reshape(op.shape)
    stats.matvecs += 1
    J = ShiftedOperator(op, dg)
    return u + h_phi1_substeps(J, h, F, tol, stats, xi=xi), stats
