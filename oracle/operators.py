"""Row assembly of the sparse operators and their Gershgorin interval.

ORACLE — test infrastructure only (see oracle/__init__.py).

Sign convention: the library integrates u' = A u + g(u); the paper writes
u' + A_p u = g(u) (Eq. (1)), so A = -A_p and the spectrum of A lies in
Re <= ~0.

Stencil operator (Sec. III-A, the seven-point formula; Sec. III-B, the
position-dependent diffusion coefficient), in conservative form
    (A u)_i = sum_axes [ D_{i+1/2}(u_{i+1}-u_i) - D_{i-1/2}(u_i-u_{i-1}) ] / dx^2
            + sum_axes b_i (u_{i+1} - u_{i-1}) / (2 dx)  +  c_i u_i,
with face coefficients D_{i+1/2} = (D_i + D_{i+1})/2.  Homogeneous boundary
conditions are folded into the rows (Sec. III-A, "implement the boundary
conditions directly into the CUDA kernel"):
  * DIRICHLET0: the ghost value is 0; the face coefficient uses D_i alone
    (D is only known inside the grid: a reading).
  * NEUMANN0: the ghost mirrors the boundary value, u_ghost = u_i, so the
    boundary face carries no diffusive flux and the centred advection
    difference becomes one-sided.
Arrays are indexed [z, y, x] (3D) or [y, x] (2D): x is the fastest axis.

CSR operator: A = W + diag(extra) for a sparse W given as CSR (the graph
operator -L = W - diag(deg_w) puts -deg_w in `extra`).
"""
from __future__ import annotations

import numpy as np

DIRICHLET0 = 0
NEUMANN0 = 1


class StencilOperator:
    """Explicit per-row coefficients: diag and one coefficient per neighbour."""

    def __init__(self, n, dx, D, b, c=None, bc=None):
        self.dim = len(n)
        self.n = tuple(int(v) for v in n)
        self.shape = tuple(reversed(self.n))
        self.dx = tuple(float(v) for v in dx)
        if bc is None:
            bc = (DIRICHLET0,) * (2 * self.dim)
        self.bc = tuple(bc)
        self._D, self._b = D, b
        Darr = np.broadcast_to(np.asarray(D, dtype=np.float64), self.shape)
        diag = np.zeros(self.shape)
        self.off = {}
        for ax in range(self.dim):
            npax = self.dim - 1 - ax
            h2 = self.dx[ax] * self.dx[ax]
            bax = np.broadcast_to(np.asarray(b[ax], dtype=np.float64), self.shape)
            n_ax = self.shape[npax]
            for sgn in (-1, +1):
                face = 2 * ax + (0 if sgn < 0 else 1)
                # neighbour D (its own D where the neighbour is a ghost)
                Dn = np.array(Darr)
                exists = np.zeros(self.shape, dtype=bool)
                src = [slice(None)] * self.dim
                dst = [slice(None)] * self.dim
                if sgn > 0:
                    dst[npax] = slice(0, n_ax - 1)
                    src[npax] = slice(1, n_ax)
                else:
                    dst[npax] = slice(1, n_ax)
                    src[npax] = slice(0, n_ax - 1)
                Dn[tuple(dst)] = Darr[tuple(src)]
                exists[tuple(dst)] = True
                Dface = 0.5 * (Darr + Dn)
                coef = np.where(exists, Dface / h2 + sgn * bax / (2.0 * self.dx[ax]), 0.0)
                self.off[(ax, sgn)] = coef
                if self.bc[face] == NEUMANN0:
                    # interior rows lose D_face/dx^2; boundary rows gain the mirrored advection
                    diag += np.where(exists, -Dface / h2, sgn * bax / (2.0 * self.dx[ax]))
                else:
                    diag += -Dface / h2
        if c is not None:
            diag = diag + np.broadcast_to(np.asarray(c, dtype=np.float64), self.shape)
        self.diag = diag

    def face_shape(self, face):
        """Shape of face `face` (2 ax + side): the grid without axis ax."""
        npax = self.dim - 1 - face // 2
        return tuple(v for k, v in enumerate(self.shape) if k != npax)

    def boundary_vector(self, faces) -> np.ndarray:
        """Inhomogeneous Dirichlet data (the paper's boundary functions f of
        Sec. III-A): at a DIRICHLET0 face the ghost value is the prescribed
        value instead of 0, so each row next to that face gains its face
        coefficient, D_i/dx^2 + sgn b_i/(2 dx) (the ghost D is D_i), times the
        value.  faces: one array of face_shape(f) per face, or None (zero).
        Returns b_D, with A u + b_D the operator applied to u and its data."""
        out = np.zeros(self.shape)
        for face, vals in enumerate(faces[: 2 * self.dim]):
            if vals is None:
                continue
            if self.bc[face] != DIRICHLET0:
                raise ValueError(f"face {face}: boundary values need a Dirichlet face")
            ax, sgn = face // 2, (-1 if face % 2 == 0 else 1)
            npax = self.dim - 1 - ax
            vals = np.asarray(vals, dtype=np.float64).reshape(self.face_shape(face))
            sl = [slice(None)] * self.dim
            sl[npax] = 0 if sgn < 0 else self.shape[npax] - 1
            Dx = np.broadcast_to(np.asarray(self._D, dtype=np.float64), self.shape)[tuple(sl)]
            bx = np.broadcast_to(np.asarray(self._b[ax], dtype=np.float64), self.shape)[tuple(sl)]
            h = self.dx[ax]
            out[tuple(sl)] += (Dx / (h * h) + sgn * bx / (2.0 * h)) * vals
        return out

    # (A u)_i = diag_i u_i + sum_nb coef_nb,i u_nb
    def matvec(self, u: np.ndarray) -> np.ndarray:
        u = np.asarray(u, dtype=np.float64).reshape(self.shape)
        out = self.diag * u
        for (ax, sgn), coef in self.off.items():
            npax = self.dim - 1 - ax
            n_ax = self.shape[npax]
            src = [slice(None)] * self.dim
            dst = [slice(None)] * self.dim
            if sgn > 0:
                dst[npax] = slice(0, n_ax - 1)
                src[npax] = slice(1, n_ax)
            else:
                dst[npax] = slice(1, n_ax)
                src[npax] = slice(0, n_ax - 1)
            out[tuple(dst)] += coef[tuple(dst)] * u[tuple(src)]
        return out

    def radius(self) -> np.ndarray:
        r = np.zeros(self.shape)
        for coef in self.off.values():
            r = r + np.abs(coef)
        return r

    def gershgorin(self, extra_diag=None) -> tuple[float, float]:
        """alpha = min_i(a_ii - r_i), beta = max_i(a_ii + r_i), r_i = sum_{j!=i}|a_ij|."""
        d = self.diag if extra_diag is None else self.diag + extra_diag.reshape(self.shape)
        r = self.radius()
        return float(np.min(d - r)), float(np.max(d + r))

    def dense(self) -> np.ndarray:
        """The full matrix, column by column (small grids only)."""
        size = int(np.prod(self.shape))
        M = np.zeros((size, size))
        e = np.zeros(size)
        for j in range(size):
            e[j] = 1.0
            M[:, j] = self.matvec(e).ravel()
            e[j] = 0.0
        return M


class CsrOperator:
    """A = W + diag(extra); W in CSR (rowptr int64, col int32, val float64)."""

    def __init__(self, n, rowptr, col, val, extra_diag=None):
        self.n = int(n)
        self.shape = (self.n,)
        self.rowptr = np.asarray(rowptr, dtype=np.int64)
        self.col = np.asarray(col, dtype=np.int64)
        self.val = np.asarray(val, dtype=np.float64)
        self.row = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        self.extra = (np.zeros(self.n) if extra_diag is None
                      else np.asarray(extra_diag, dtype=np.float64).copy())

    def matvec(self, u: np.ndarray) -> np.ndarray:
        u = np.asarray(u, dtype=np.float64).ravel()
        out = np.bincount(self.row, weights=self.val * u[self.col], minlength=self.n)
        return out + self.extra * u

    def gershgorin(self, extra_diag=None) -> tuple[float, float]:
        on = self.col == self.row
        d = self.extra + np.bincount(self.row[on], self.val[on], minlength=self.n)
        if extra_diag is not None:
            d = d + extra_diag.ravel()
        r = np.bincount(self.row[~on], np.abs(self.val[~on]), minlength=self.n)
        return float(np.min(d - r)), float(np.max(d + r))

    def dense(self) -> np.ndarray:
        M = np.zeros((self.n, self.n))
        np.add.at(M, (self.row, self.col), self.val)
        M[np.arange(self.n), np.arange(self.n)] += self.extra
        return M


class ShiftedOperator:
    """J = A + diag(q): the exponential Rosenbrock-Euler Jacobian."""

    def __init__(self, base, q):
        self.base = base
        self.shape = base.shape
        self.q = np.asarray(q, dtype=np.float64).reshape(base.shape)

    def matvec(self, u):
        u = np.asarray(u, dtype=np.float64).reshape(self.shape)
        return self.base.matvec(u) + self.q * u

    def gershgorin(self):
        return self.base.gershgorin(extra_diag=self.q)

    def dense(self):
        return self.base.dense() + np.diag(self.q.ravel())
