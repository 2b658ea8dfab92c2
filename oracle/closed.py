"""Closed forms that pin the operator assembly and the Leja iteration.

ORACLE — test infrastructure only (see oracle/__init__.py).

1. Constant-coefficient Dirichlet operator (vertex-centred, ghost 0) in 2D:
   A = T_x (+) T_y, each T tridiagonal Toeplitz with sub a, diag d, super c
   (a = D/dx^2 - b/(2dx), c = D/dx^2 + b/(2dx), d = -2D/dx^2).  For a*c > 0,
   T = S^-1 Q diag(lam) Q^T S with s_i = (c/a)^(i/2),
   Q_ip = sqrt(2/(N+1)) sin(i p pi/(N+1)), lam_p = d + 2 sqrt(ac) cos(p pi/(N+1)),
   i, p = 1..N.  So f(hA)v follows from transforms along each axis.
2. Constant-D pure diffusion with cell-centred homogeneous Neumann ends:
   T = Q diag(lam) Q^T with Q_ip ~ cos((i+1/2) p pi/N),
   lam_p = -(4D/dx^2) sin^2(p pi/(2N)), i, p = 0..N-1.
3. u_t = D Lap u + b.grad u on the whole space from a Gaussian of width sigma:
   u = (s^2/(s^2+2Dt))^(d/2) exp(-|x - x0 + b t|^2 / (2(s^2+2Dt))).
"""
from __future__ import annotations

import math

import numpy as np

from . import leja as L


def _phi_vec(k, z):
    return np.array([L.phi_scalar(k, float(x)) for x in np.ravel(z)]).reshape(np.shape(z))


def dirichlet_factor(N, D, b, dx):
    """(S, Q, lam) of one axis' tridiagonal Toeplitz factor."""
    a = D / dx ** 2 - b / (2 * dx)
    c = D / dx ** 2 + b / (2 * dx)
    d = -2.0 * D / dx ** 2
    i = np.arange(1, N + 1)
    p = np.arange(1, N + 1)
    Q = math.sqrt(2.0 / (N + 1)) * np.sin(np.outer(i, p) * math.pi / (N + 1))
    lam = d + 2.0 * math.sqrt(a * c) * np.cos(p * math.pi / (N + 1))
    s = (c / a) ** (i / 2.0)
    return s, Q, lam


def phi_dirichlet_2d(k, h, v, N, D, b, dx):
    """phi_k(hA) v for the 2D constant-coefficient Dirichlet operator; v is [y, x]."""
    sx, Qx, lx = dirichlet_factor(N[0], D, b[0], dx[0])
    sy, Qy, ly = dirichlet_factor(N[1], D, b[1], dx[1])
    V = np.asarray(v, dtype=np.float64).reshape(N[1], N[0])
    W = (sy[:, None] * sx[None, :]) * V                  # S v
    W = Qy.T @ W @ Qx                                    # Q^T S v
    W = _phi_vec(k, h * (ly[:, None] + lx[None, :])) * W
    W = Qy @ W @ Qx.T                                    # Q f(Lam) Q^T S v
    return W / (sy[:, None] * sx[None, :])


def neumann_factor(N, D, dx):
    i = np.arange(N)
    p = np.arange(N)
    Q = np.cos(np.outer(i + 0.5, p) * math.pi / N)
    Q = Q / np.sqrt(np.sum(Q * Q, axis=0))[None, :]
    lam = -(4.0 * D / dx ** 2) * np.sin(p * math.pi / (2 * N)) ** 2
    return Q, lam


def phi_neumann_3d(k, h, v, N, D, dx):
    """phi_k(hA) v, A = D Lap with cell-centred homogeneous Neumann, v is [z, y, x]."""
    Qx, lx = neumann_factor(N[0], D, dx[0])
    Qy, ly = neumann_factor(N[1], D, dx[1])
    Qz, lz = neumann_factor(N[2], D, dx[2])
    V = np.asarray(v, dtype=np.float64).reshape(N[2], N[1], N[0])
    W = np.einsum("zyx,xp,yq,zr->rqp", V, Qx, Qy, Qz)
    lam = lz[:, None, None] + ly[None, :, None] + lx[None, None, :]
    W = _phi_vec(k, h * lam) * W
    return np.einsum("rqp,xp,yq,zr->zyx", W, Qx, Qy, Qz)


def gaussian(points, t, D, b, x0, sigma):
    """Whole-space solution of u_t = D Lap u + b.grad u from a Gaussian.
    points: array (..., d); b, x0: length-d."""
    dim = points.shape[-1]
    var = sigma ** 2 + 2.0 * D * t
    centre = np.asarray(x0) - np.asarray(b) * t
    r2 = np.sum((points - centre) ** 2, axis=-1)
    return (sigma ** 2 / var) ** (dim / 2.0) * np.exp(-r2 / (2.0 * var))
