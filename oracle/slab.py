"""The oracle's exponential Euler and Rosenbrock-Euler steps on all host cores.

ORACLE — test infrastructure only (see oracle/__init__.py).

The same method as newton.exp_euler_step and newton.exp_rosenbrock_step (the
Newton form of the Leja interpolant, Eq. (3) products, Sec. II-C and III-C;
substeps of y' = J y + F from 0), with the element-wise work split into z-slabs that host
threads process at once (numpy releases the interpreter lock inside its array
loops).  Each slab keeps an operators.StencilOperator built on the slab
extended by one plane on each interior side: the rows of the slab's own planes
are then exactly the rows of the whole-grid operator (their neighbours and
face coefficients lie inside the extended slab), and the extension rows are
discarded.  Every element is computed by the same expressions in the same
order as the serial oracle; only the squared norms differ in summation order
(per-slab sums added in slab order), and the Gershgorin min/max, which is
order-free.  The schedule and the divided differences are the serial oracle's
(leja.plain_schedule, leja.divided_differences).
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import leja as L
from .newton import NONLIN_LOGISTIC, NotConverged, Stats, nonlinearity
from .operators import StencilOperator


def host_threads() -> int:
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class SlabStencil:
    """A 3D stencil operator split into `parts` z-slabs."""

    def __init__(self, n, dx, D, b, c=None, bc=None, parts=None):
        nx, ny, nz = (int(v) for v in n)
        self.shape = (nz, ny, nx)
        parts = max(1, min(parts or host_threads(), nz))
        self.parts = parts
        cuts = [nz * i // parts for i in range(parts + 1)]
        self.slabs = []
        Dfull = np.broadcast_to(np.asarray(D, dtype=np.float64), self.shape)
        bfull = [np.broadcast_to(np.asarray(x, dtype=np.float64), self.shape) for x in b]
        cfull = (None if c is None
                 else np.broadcast_to(np.asarray(c, dtype=np.float64), self.shape))
        bc = tuple(bc) if bc is not None else (0,) * 6
        for z0, z1 in zip(cuts[:-1], cuts[1:]):
            e0, e1 = max(z0 - 1, 0), min(z1 + 1, nz)
            op = StencilOperator((nx, ny, e1 - e0), dx, Dfull[e0:e1], [x[e0:e1] for x in bfull],
                                 None if cfull is None else cfull[e0:e1], bc)
            self.slabs.append((z0, z1, e0, e1, op))
        self.pool = ThreadPoolExecutor(max_workers=parts)

    def close(self):
        self.pool.shutdown()

    def run(self, fn):
        """fn(i, z0, z1, e0, e1, op) on every slab at once; the results in slab order."""
        futs = [self.pool.submit(fn, i, *sl) for i, sl in enumerate(self.slabs)]
        return [f.result() for f in futs]

    @staticmethod
    def own(op_out, z0, z1, e0):
        """The slab's own planes of an array computed on the extended slab."""
        return op_out[z0 - e0: z1 - e0]


def exp_rosenbrock_step(sop: SlabStencil, u, h, tol, nonlin=NONLIN_LOGISTIC, xi=None,
                        m_max=L.M_MAX):
    """u_{n+1} = u_n + h phi_1(h J_n)(A u_n + g(u_n)), J_n = A + diag(g'(u_n)),
    as newton.exp_rosenbrock_step.  Returns (u_{n+1}, Stats)."""
    return _step(sop, u, h, tol, nonlin, xi, m_max, rosenbrock=True)


def exp_euler_step(sop: SlabStencil, u, h, tol, nonlin=NONLIN_LOGISTIC, xi=None,
                   m_max=L.M_MAX):
    """u_{n+1} = u_n + h phi_1(hA)(A u_n + g(u_n)) (Eq. (2)), as
    newton.exp_euler_step.  Returns (u_{n+1}, Stats)."""
    return _step(sop, u, h, tol, nonlin, xi, m_max, rosenbrock=False)


def _step(sop, u, h, tol, nonlin, xi, m_max, rosenbrock):
    stats = Stats()
    u = np.asarray(u, dtype=np.float64).reshape(sop.shape)
    if xi is None:
        xi = L.leja_points(m_max)
    g = np.empty_like(u)
    dg = np.empty_like(u)
    F = np.empty_like(u)

    def setup(i, z0, z1, e0, e1, op):
        gs, dgs = nonlinearity(u[z0:z1], nonlin)
        g[z0:z1], dg[z0:z1] = gs, dgs
        F[z0:z1] = SlabStencil.own(op.matvec(u[e0:e1]), z0, z1, e0) + gs
        d = SlabStencil.own(op.diag, z0, z1, e0)
        if rosenbrock:
            d = d + dgs
        r = SlabStencil.own(op.radius(), z0, z1, e0)
        return float(np.min(d - r)), float(np.max(d + r)), float(np.sum(F[z0:z1] * F[z0:z1]))

    parts = sop.run(setup)
    stats.matvecs += 1
    alpha = min(p[0] for p in parts)
    beta = max(p[1] for p in parts)
    fn2 = sum(p[2] for p in parts)
    stats.alpha, stats.beta = alpha, beta
    c, gamma = 0.5 * (alpha + beta), 0.25 * (beta - alpha)
    if fn2 == 0.0:
        stats.s, stats.degrees = 1, [0]
        return u.copy(), stats
    if gamma == 0.0:
        stats.s, stats.degrees = 1, [0]
        return u + h * L.phi_scalar(1, h * c) * F, stats

    def jmatvec_into(src, dst, i, z0, z1, e0, e1, op):
        # (J x) on the slab's own planes: A x + g'(u) x (Rosenbrock) or A x
        ax = SlabStencil.own(op.matvec(src[e0:e1]), z0, z1, e0)
        dst[z0:z1] = ax + dg[z0:z1] * src[z0:z1] if rosenbrock else ax

    s, stats.m_sched, _ = L.plain_schedule(1, h, c, gamma, tol, xi, m_max)
    while s <= L.S_MAX:
        tau = h / s
        d = L.divided_differences(1, tau, c, gamma, xi[: m_max + 1])
        y = np.zeros_like(u)
        r = np.empty_like(u)
        degrees = []
        ok = True
        for i_sub in range(s):
            if i_sub == 0:
                r[...] = F
            else:
                def resid(i, z0, z1, e0, e1, op):
                    jmatvec_into(y, r, i, z0, z1, e0, e1, op)
                    r[z0:z1] = r[z0:z1] + F[z0:z1]
                sop.run(resid)
                stats.matvecs += 1
            p, deg, conv = _newton(sop, jmatvec_into, r, d, xi, c, gamma, tol, m_max, stats)
            degrees.append(deg)
            if not conv:
                ok = False
                break
            y = y + tau * p
        if ok:
            stats.s, stats.degrees = s, degrees
            return u + y, stats
        stats.restarts += 1
        s *= 2
    raise NotConverged("phi_1: no s <= S_MAX converged")


def _newton(sop, jmatvec_into, r, d, xi, c, gamma, tol, m_max, stats):
    """newton.newton_phi with each iteration's element-wise work on the slabs:
    w_{j+1} = (J w_j)/gamma - (c/gamma + xi_j) w_j, p += d_{j+1} w_{j+1}, and the
    stop test |d_{j+1}| ||w_{j+1}|| <= tol ||p||."""
    r2 = sum(sop.run(lambda i, z0, z1, e0, e1, op: float(np.sum(r[z0:z1] * r[z0:z1]))))
    if r2 == 0.0:
        return np.zeros_like(r), 0, True
    w = r.copy()
    p = d[0] * w
    wn = np.empty_like(w)
    for j in range(m_max):
        shift = c / gamma + xi[j]
        dn = d[j + 1]

        def it(i, z0, z1, e0, e1, op):
            jmatvec_into(w, wn, i, z0, z1, e0, e1, op)
            ws = wn[z0:z1] / gamma - shift * w[z0:z1]
            wn[z0:z1] = ws
            ps = p[z0:z1] + dn * ws
            p[z0:z1] = ps
            return float(np.sum(ws * ws)), float(np.sum(ps * ps))

        parts = sop.run(it)
        stats.matvecs += 1
        nw2 = sum(q[0] for q in parts)
        np2 = sum(q[1] for q in parts)
        w, wn = wn, w
        if abs(dn) * float(np.sqrt(nw2)) <= tol * float(np.sqrt(np2)):
            return p, j + 1, True
    return p, m_max, False
