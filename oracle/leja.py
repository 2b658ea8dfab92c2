"""Leja points, scalar phi_k, divided differences and the a-priori schedule.

ORACLE — test infrastructure only (see oracle/__init__.py).

The paper (Sec. II-C, text after Eq. (2), and Sec. III-C first paragraph)
computes phi-functions of A by polynomial interpolation on a known bound of
the field of values, "interpolation at Leja points", which Horner's scheme
reduces to repeated products (alpha*A + beta*I)x (Eq. (3)).  It does not
spell the method out; this module writes out the standard real-Leja method
(Caliari, Vianello & Bergamaschi 2004, cited by the paper) from its
mathematical definition:

  * the spectral interval [alpha, beta] is mapped to [-2, 2] (an interval of
    logarithmic capacity 1) by  xi = (z - c)/gamma,  c = (alpha+beta)/2,
    gamma = (beta-alpha)/4;
  * Leja points: xi_0 = 2, xi_j = argmax_{x in [-2,2]} prod_{i<j} |x - xi_i|,
    ties broken towards the larger x (a reading: the paper is silent);
  * Newton divided differences d_j = f[xi_0..xi_j] of
    f(xi) = phi_k(tau*c + tau*gamma*xi), computed here by the plain recurrence
    in decimal arithmetic at a precision raised until it no longer changes
    any entry;
  * the plain a-priori substep rule: the smallest s = 2^q for which the
    degree-<=m_max scalar interpolant meets max_G |f - p_m| <= tol*max_G |f|
    on 2001 equispaced points G of [-2, 2] (a reading of "conservative a
    priori choice"; the paper gives no rule).
"""
from __future__ import annotations

import math
from decimal import Decimal, localcontext

import numpy as np

M_MAX = 100          # largest Newton degree per substep
S_MAX = 2 ** 20      # largest number of substeps
DEC_PREC = 120       # decimal digits for scalar phi (and the starting precision of the
                     # divided differences)
N_GRID = 2001        # points of G in the schedule rule
TIE_LOG = 1e-12      # two Leja candidates tie when their log-products differ less


# --------------------------------------------------------------------------
# Leja points on [-2, 2]
# --------------------------------------------------------------------------
def _log_abs_prod(x: float, pts: list[float]) -> float:
    return sum(math.log(abs(x - p)) for p in pts)


def _critical_point(pts: list[float], a: float, b: float) -> float:
    """The maximiser of prod|x - p| on the open gap (a, b) between nodes.

    There log prod|x-p| is concave and its derivative g(x) = sum 1/(x-p)
    falls monotonically from +inf to -inf, so its single root is found by
    bisection to the last bit."""
    lo, hi = a, b
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        g = sum(1.0 / (mid - p) for p in pts)
        if g > 0.0:
            lo = mid
        else:
            hi = mid
    glo = abs(sum(1.0 / (lo - p) for p in pts)) if lo != a else math.inf
    ghi = abs(sum(1.0 / (hi - p) for p in pts)) if hi != b else math.inf
    return lo if glo <= ghi else hi


def leja_points(m: int = M_MAX) -> np.ndarray:
    """xi_0 .. xi_m on [-2, 2], by the definition (greedy maximisation).

    Candidates for step j are the two interval ends not yet taken (beyond the
    outermost node the product grows towards the end) and the one critical
    point in each gap between consecutive nodes; the largest product wins,
    ties (log-products within TIE_LOG) go to the larger x."""
    pts = [2.0]
    for _ in range(1, m + 1):
        srt = sorted(pts)
        cands = [e for e in (-2.0, 2.0) if e not in pts]
        cands += [_critical_point(pts, a, b) for a, b in zip(srt[:-1], srt[1:])]
        vals = [_log_abs_prod(x, pts) for x in cands]
        best = max(vals)
        pts.append(max(x for x, v in zip(cands, vals) if v >= best - TIE_LOG))
    return np.array(pts, dtype=np.float64)


# --------------------------------------------------------------------------
# Scalar phi_k
# --------------------------------------------------------------------------
def phi_dec(k: int, z: Decimal, prec: int = DEC_PREC) -> Decimal:
    """phi_k(z) = sum_{i>=0} z^i/(i+k)!  (phi_0 = exp), in the current
    decimal context.  Series for |z| < 1, else the recurrence
    phi_j(z) = (phi_{j-1}(z) - 1/(j-1)!)/z from phi_0 = exp(z)."""
    if abs(z) < 1:
        term = Decimal(1) / Decimal(math.factorial(k))
        total = term
        eps = Decimal(10) ** (-(prec + 10))
        i = 0
        while abs(term) > eps:
            term = term * z / (i + k + 1)
            total += term
            i += 1
        return total
    val = z.exp()
    for j in range(1, k + 1):
        val = (val - Decimal(1) / Decimal(math.factorial(j - 1))) / z
    return val


def phi_scalar(k: int, z: float) -> float:
    """phi_k(z) for a double z, correctly rounded to a double."""
    with localcontext() as ctx:
        ctx.prec = DEC_PREC
        return float(phi_dec(k, Decimal(z)))


# --------------------------------------------------------------------------
# Divided differences
# --------------------------------------------------------------------------
def _dd_at(k, tau, c, gamma, xi, prec):
    with localcontext() as ctx:
        ctx.prec = prec
        T, C, G = Decimal(tau), Decimal(c), Decimal(gamma)
        xs = [Decimal(float(x)) for x in xi]
        tab = [phi_dec(k, T * C + T * G * x, prec) for x in xs]
        n = len(xs)
        for j in range(1, n):
            for i in range(n - 1, j - 1, -1):
                tab[i] = (tab[i] - tab[i - 1]) / (xs[i] - xs[i - j])
        return tab


def divided_differences(k: int, tau: float, c: float, gamma: float,
                        xi: np.ndarray) -> np.ndarray:
    """d_j = f[xi_0..xi_j] for f(xi) = phi_k(tau*c + tau*gamma*xi).

    Plain Newton recurrence f[x_i..x_j] = (f[x_{i+1}..x_j] - f[x_i..x_{j-1}])
    / (x_j - x_i) in decimal arithmetic; the inputs (doubles) are converted
    exactly.  The recurrence cancels about as many digits as the smallest d_j
    is below max|f|, so it is run at a working precision P and again at P+64
    digits, and P grows until every entry of the two runs agrees to 1e-20
    relative; the results are rounded to doubles."""
    prec = DEC_PREC
    prev = _dd_at(k, tau, c, gamma, xi, prec)
    while True:
        nxt = _dd_at(k, tau, c, gamma, xi, prec + 64)
        ok = all(abs(a - b) <= Decimal("1e-20") * abs(b) for a, b in zip(prev, nxt))
        if ok or prec > 4000:
            return np.array([float(t) for t in nxt], dtype=np.float64)
        prec += 64
        prev = nxt


def newton_eval(d: np.ndarray, xi: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Partial sums p_m(x) = sum_{j<=m} d_j prod_{i<j}(x - xi_i), m = 0..len(d)-1,
    as rows of a (len(d), len(x)) array (FP64)."""
    out = np.empty((len(d), len(x)))
    omega = np.ones_like(x)
    acc = np.zeros_like(x)
    for j in range(len(d)):
        acc = acc + d[j] * omega
        out[j] = acc
        omega = omega * (x - xi[j])
    return out


# --------------------------------------------------------------------------
# The plain a-priori schedule
# --------------------------------------------------------------------------
def schedule_error(k: int, tau: float, c: float, gamma: float, xi: np.ndarray,
                   d: np.ndarray) -> tuple[np.ndarray, float]:
    """err_m = max_G |f - p_m| for m = 0..len(d)-1, and max_G |f|."""
    g = np.linspace(-2.0, 2.0, N_GRID)
    with localcontext() as ctx:
        ctx.prec = DEC_PREC
        T, C, Gm = Decimal(tau), Decimal(c), Decimal(gamma)
        f = np.array([float(phi_dec(k, T * C + T * Gm * Decimal(float(x)))) for x in g])
    p = newton_eval(d, xi, g)
    return np.max(np.abs(p - f[None, :]), axis=1), float(np.max(np.abs(f)))


def plain_schedule(k: int, h: float, c: float, gamma: float, tol: float,
                   xi: np.ndarray | None = None, m_max: int = M_MAX):
    """Smallest s = 2^q (s <= S_MAX) such that some degree m <= m_max meets
    max_G|f - p_m| <= tol * max_G|f| with tau = h/s.  Returns
    (s, m_sched, margin) with margin = min_m err_m / (tol * max|f|)."""
    if xi is None:
        xi = leja_points(m_max)
    s = 1
    while s <= S_MAX:
        tau = h / s
        d = divided_differences(k, tau, c, gamma, xi[: m_max + 1])
        err, fmax = schedule_error(k, tau, c, gamma, xi, d)
        ratio = err / (tol * fmax)
        ok = np.nonzero(ratio <= 1.0)[0]
        if ok.size:
            return s, int(ok[0]), float(ratio.min())
        s *= 2
    raise RuntimeError("schedule: no s <= S_MAX meets the tolerance")
