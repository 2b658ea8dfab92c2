"""phi_k(-i h H) v for a Hermitian (real symmetric) operator H: the
complex-valued products (alpha A + beta I)x of Eq. (3) with K = C (Sec. II-C,
Sec. III-D), for Schroedinger-type problems u' = -i H u.

ORACLE -- test infrastructure only (see oracle/__init__.py).

With A = -iH the spectrum of hA is -ih sigma(H), on the imaginary axis.  The
interpolation runs on H's real Gershgorin interval [alpha, beta] mapped to
[-2, 2] with the same real Leja points: the function
    f(xi) = phi_k(-i tau (c + gamma xi))
is complex, so its divided differences d_j are complex, while the Newton
basis of H,
    w_{j+1} = (H w_j)/gamma - (c/gamma + xi_j) w_j,
is the real recurrence (complex only through v).  Then
    p = sum_j d_j w_j ~= phi_k(-i tau H) r,
stopping when |d_{j+1}| ||w_{j+1}|| <= tol ||p||.
Readings: k = 0 applies e^{-i tau H} s times (tau = h/s); k >= 1 takes one
substep only.  The divided differences of the complex f at real nodes are
those of Re f and Im f (the recurrence is linear in f), computed in decimal
arithmetic as for real f.  The schedule is the real a-priori rule applied to
the complex f (max over the grid of |f - p_m|).
"""
from __future__ import annotations

import math
from decimal import Decimal, localcontext

import numpy as np

from . import leja as L


def phi_dec_imag(k: int, y: Decimal, prec: int) -> tuple[Decimal, Decimal]:
    """phi_k(i y) = sum_n (i y)^n / (n + k)!, as (real, imaginary) parts, in
    the current decimal context (whose precision covers the cancellation of
    terms up to e^{|y|})."""
    term = Decimal(1) / Decimal(math.factorial(k))  # y^n/(n+k)! for n = 0
    re, im = term, Decimal(0)
    eps = Decimal(10) ** (-(prec + 10))
    n = 0
    while True:
        n += 1
        term = term * y / (n + k)
        q = n % 4  # i^n = 1, i, -1, -i
        if q == 0:
            re += term
        elif q == 1:
            im += term
        elif q == 2:
            re -= term
        else:
            im -= term
        if n > abs(y) and abs(term) < eps:
            return re, im


def _f_nodes(k, tau, c, gamma, xs, prec):
    T, C, G = Decimal(tau), Decimal(c), Decimal(gamma)
    out = []
    for x in xs:
        y = -(T * C + T * G * x)
        out.append(phi_dec_imag(k, y, prec))
    return out


def _dd_imag_at(k, tau, c, gamma, xi, prec):
    ymax = abs(tau) * (abs(c) + 2 * abs(gamma))
    with localcontext() as ctx:
        ctx.prec = prec + int(ymax * 0.4343) + 20
        xs = [Decimal(float(x)) for x in xi]
        vals = _f_nodes(k, tau, c, gamma, xs, prec)
        tabs = []
        for part in (0, 1):
            tab = [v[part] for v in vals]
            n = len(xs)
            for j in range(1, n):
                for i in range(n - 1, j - 1, -1):
                    tab[i] = (tab[i] - tab[i - 1]) / (xs[i] - xs[i - j])
            tabs.append(tab)
        return tabs


def divided_differences_imag(k: int, tau: float, c: float, gamma: float,
                             xi: np.ndarray) -> np.ndarray:
    """d_j = f[xi_0..xi_j] for f(xi) = phi_k(-i tau (c + gamma xi)), complex.
    Working precision grows until two runs 64 digits apart agree to 1e-20
    relative (as leja.divided_differences)."""
    prec = L.DEC_PREC
    prev = _dd_imag_at(k, tau, c, gamma, xi, prec)
    while True:
        nxt = _dd_imag_at(k, tau, c, gamma, xi, prec + 64)
        ok = all(abs(a - b) <= Decimal("1e-20") * max(abs(b), Decimal("1e-300"))
                 for pa, pb in zip(prev, nxt) for a, b in zip(pa, pb))
        if ok or prec > 4000:
            return np.array([complex(float(a), float(b)) for a, b in zip(*nxt)])
        prec += 64
        prev = nxt


def f_grid(k, tau, c, gamma, x):
    """f on the points x (complex doubles)."""
    with localcontext() as ctx:
        ymax = abs(tau) * (abs(c) + 2 * abs(gamma))
        ctx.prec = L.DEC_PREC + int(ymax * 0.4343) + 20
        vals = _f_nodes(k, tau, c, gamma, [Decimal(float(t)) for t in x], L.DEC_PREC)
        return np.array([complex(float(a), float(b)) for a, b in vals])


def newton_eval_c(d, xi, x):
    """Partial sums p_m(x), m = 0..len(d)-1, of the complex Newton form."""
    out = np.empty((len(d), len(x)), dtype=complex)
    omega = np.ones(len(x))
    acc = np.zeros(len(x), dtype=complex)
    for j in range(len(d)):
        acc = acc + d[j] * omega
        out[j] = acc
        omega = omega * (x - xi[j])
    return out


def schedule_imag(k, h, c, gamma, tol, xi, m_max=L.M_MAX):
    """Smallest s = 2^q such that some m <= m_max meets
    max_G |f - p_m| <= tol max_G |f| at tau = h/s (leja.plain_schedule with the
    complex f).  Returns (s, m)."""
    g = np.linspace(-2.0, 2.0, L.N_GRID)
    s = 1
    while s <= L.S_MAX:
        tau = h / s
        d = divided_differences_imag(k, tau, c, gamma, xi[: m_max + 1])
        f = f_grid(k, tau, c, gamma, g)
        err = np.max(np.abs(newton_eval_c(d, xi, g) - f[None, :]), axis=1)
        ok = np.nonzero(err <= tol * np.max(np.abs(f)))[0]
        if ok.size:
            return s, int(ok[0])
        s *= 2
    raise RuntimeError("schedule_imag: no s <= S_MAX meets the tolerance")


def _matvec_c(op, x):
    return op.matvec(x.real.copy()) + 1j * op.matvec(x.imag.copy())


def newton_imag(op, r, d, xi, c, gamma, tol, m_max):
    """p ~= phi_k(-i tau H) r.  Returns (p, degree, converged)."""
    w = np.asarray(r, dtype=complex)
    p = d[0] * w
    for j in range(m_max):
        w = _matvec_c(op, w) / gamma - (c / gamma + xi[j]) * w
        p = p + d[j + 1] * w
        nw = float(np.sqrt(np.sum(np.abs(w) ** 2)))
        np_ = float(np.sqrt(np.sum(np.abs(p) ** 2)))
        if abs(d[j + 1]) * nw <= tol * np_:
            return p, j + 1, True
    return p, m_max, False


def phi_apply_imag(op, k, h, v, tol, m_max=L.M_MAX, xi=None, fixed_s=None):
    """phi_k(-i h H) v for the real symmetric operator H = op; v complex.
    Returns (result, s, degrees)."""
    alpha, beta = op.gershgorin()
    c, gamma = 0.5 * (alpha + beta), 0.25 * (beta - alpha)
    v = np.asarray(v, dtype=complex).reshape(op.shape)
    if xi is None:
        xi = L.leja_points(m_max)
    if not np.any(v):
        return np.zeros_like(v), 1, [0]
    if gamma == 0.0:
        with localcontext() as ctx:
            ctx.prec = L.DEC_PREC + int(abs(h * c) * 0.4343) + 20
            re, im = phi_dec_imag(k, -Decimal(h) * Decimal(c), L.DEC_PREC)
        return complex(float(re), float(im)) * v, 1, [0]
    s = int(fixed_s) if fixed_s else schedule_imag(k, h, c, gamma, tol, xi, m_max)[0]
    while s <= L.S_MAX:
        if k >= 1 and s > 1:
            raise RuntimeError("phi_k(-ihH), k >= 1: one substep only")
        tau = h / s
        d = divided_differences_imag(k, tau, c, gamma, xi[: m_max + 1])
        y = v
        degrees = []
        ok = True
        for _ in range(s):
            y, deg, conv = newton_imag(op, y, d, xi, c, gamma, tol, m_max)
            degrees.append(deg)
            if not conv:
                ok = False
                break
        if ok:
            return y, s, degrees
        if fixed_s:
            raise RuntimeError("phi_k(-ihH): the fixed s did not converge")
        s *= 2
    raise RuntimeError("phi_k(-ihH): no s <= S_MAX converged")
