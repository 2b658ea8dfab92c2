"""Inhomogeneous Dirichlet data in the oracle (oracle/operators.py:
StencilOperator.boundary_vector; the paper's boundary functions of Sec.
III-A), pinned to exact facts of the second and centred first differences:
on a vertex-centred grid (dx = 1/(N+1), the ghost points on the boundary) a
linear function with its own boundary values satisfies A u + b_D = b . grad u
exactly, a quadratic one with D = 1 gives the constant Laplacian, zero data
give b_D = 0, and a steady state is left unchanged by a step."""
import numpy as np
import pytest

from oracle import leja as L
from oracle import newton as Nw
from oracle import operators as O


def _grid(n):
    nx, ny, nz = n
    x = np.arange(1, nx + 1) / (nx + 1)
    y = np.arange(1, ny + 1) / (ny + 1)
    z = np.arange(1, nz + 1) / (nz + 1)
    return np.meshgrid(z, y, x, indexing="ij")  # [z, y, x]


def _faces(n, f):
    """f evaluated at the ghost points of every face (x = 0 and 1, ...)."""
    nx, ny, nz = n
    x = np.arange(1, nx + 1) / (nx + 1)
    y = np.arange(1, ny + 1) / (ny + 1)
    z = np.arange(1, nz + 1) / (nz + 1)
    Zy, Yz = np.meshgrid(z, y, indexing="ij")      # x faces: [z, y]
    Zx, Xz = np.meshgrid(z, x, indexing="ij")      # y faces: [z, x]
    Yx, Xy = np.meshgrid(y, x, indexing="ij")      # z faces: [y, x]
    return [f(0.0 * Zy, Yz, Zy), f(1.0 + 0 * Zy, Yz, Zy),
            f(Xz, 0.0 * Zx, Zx), f(Xz, 1.0 + 0 * Zx, Zx),
            f(Xy, Yx, 0.0 * Yx), f(Xy, Yx, 1.0 + 0 * Yx)]


N = (9, 7, 6)


def _op(D, b):
    dx = tuple(1.0 / (k + 1) for k in N)
    return O.StencilOperator(N, dx, D, b, bc=(O.DIRICHLET0,) * 6)


def test_linear_function_gives_advection_only():
    c0, c = 0.3, (1.5, -2.0, 0.7)
    f = lambda x, y, z: c0 + c[0] * x + c[1] * y + c[2] * z
    Z, Y, X = _grid(N)
    u = f(X, Y, Z)
    b = (0.4, -1.1, 2.0)
    op = _op(0.8, b)
    r = op.matvec(u) + op.boundary_vector(_faces(N, f))
    np.testing.assert_allclose(r, np.dot(b, c), rtol=0, atol=1e-10)


def test_quadratic_function_gives_constant_laplacian():
    f = lambda x, y, z: x * x + y * y + z * z
    Z, Y, X = _grid(N)
    op = _op(1.0, (0.0, 0.0, 0.0))
    r = op.matvec(f(X, Y, Z)) + op.boundary_vector(_faces(N, f))
    np.testing.assert_allclose(r, 6.0, rtol=0, atol=1e-9)


def test_zero_data_and_neumann_face():
    op = _op(1.3, (0.2, 0.0, -0.5))
    zero = [np.zeros(op.face_shape(k)) for k in range(6)]
    assert not op.boundary_vector(zero).any() and not op.boundary_vector([None] * 6).any()
    opn = O.StencilOperator(N, (0.1, 0.1, 0.1), 1.0, (0.0, 0.0, 0.0),
                            bc=(O.NEUMANN0,) + (O.DIRICHLET0,) * 5)
    with pytest.raises(ValueError):
        opn.boundary_vector([np.ones(opn.face_shape(0))] + [None] * 5)


def test_steady_state_is_kept_by_both_steps():
    """u linear with its own boundary data and b = 0 solves A u + b_D = 0:
    F = 0, so both steps return u exactly (phi_1 of a zero vector is 0)."""
    f = lambda x, y, z: 1.0 + 0.5 * x - y + 2.0 * z
    Z, Y, X = _grid(N)
    u = f(X, Y, Z)
    op = _op(0.7, (0.0, 0.0, 0.0))
    bv = op.boundary_vector(_faces(N, f))
    xi = L.leja_points(100)
    F = op.matvec(u) + bv
    assert np.abs(F).max() < 1e-10
    ue, _ = Nw.exp_euler_step(op, u, 1e-3, 1e-10, xi=xi, bvec=bv)
    np.testing.assert_allclose(ue, u, rtol=0, atol=1e-13)
    ur, _ = Nw.exp_rosenbrock_step(op, u, 1e-3, 1e-10, nonlin=Nw.NONLIN_NONE, xi=xi, bvec=bv)
    np.testing.assert_allclose(ur, u, rtol=0, atol=1e-13)
