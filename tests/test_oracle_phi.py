"""Pins for the oracle's operators, phi_k(hA)v and the exponential steps.

Anchors: discretisation exactness on polynomials, Gershgorin intervals in
closed form, sine/cosine eigenbases, dense expm (the definition),
conservation laws, the analytic Gaussian, and the convergence order of the
exponential Rosenbrock-Euler step against scipy's ODE solver.
"""
import math

import numpy as np
import pytest
import scipy.integrate

from oracle import closed as C
from oracle import dense as Dn
from oracle import leja as L
from oracle import newton as Nw
from oracle import operators as O


@pytest.fixture(scope="module")
def xi():
    return L.leja_points(L.M_MAX)


def test_gershgorin_closed_form_2d():
    # 64^2 interior, dx = 1/65, D = 0.1, b = -(1, 0.5): alpha = -8D/dx^2 = -3380, beta = 0
    op = O.StencilOperator((64, 64), (1 / 65, 1 / 65), 0.1, (-1.0, -0.5))
    a, b = op.gershgorin()
    assert a == pytest.approx(-3380.0, rel=1e-13)
    assert abs(b) <= 1e-10


def test_gershgorin_graph_laplacian():
    # -L of a weighted graph: alpha = -2 max deg_w, beta = 0
    rng = np.random.default_rng(0)
    n = 40
    W = np.triu(rng.uniform(0.5, 2.0, (n, n)) * (rng.random((n, n)) < 0.2), 1)
    W = W + W.T
    rows, cols = np.nonzero(W)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    deg = W.sum(axis=1)
    op = O.CsrOperator(n, rowptr, cols, W[rows, cols], -deg)
    a, b = op.gershgorin()
    assert a == pytest.approx(-2 * deg.max(), rel=1e-14)
    assert abs(b) <= 1e-13
    assert np.allclose(op.dense(), W - np.diag(deg), atol=0)


def _grid(n, dx, centred):
    off = 0.5 if centred else 1.0
    return (np.arange(n) + off) * dx


def test_stencil_exact_on_quadratics_3d():
    # conservative form with face-averaged D is exact for D linear and u quadratic:
    # div(D grad x^2) = 2a + 4 b1 x for D = a + b1 x; centred advection exact too
    n = (9, 7, 6)
    dx = (0.1, 0.13, 0.17)
    x = _grid(n[0], dx[0], True)
    y = _grid(n[1], dx[1], True)
    z = _grid(n[2], dx[2], True)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    a0, b1 = 1.3, 0.4
    D = a0 + b1 * X
    bx, by, bz = 0.7 + 0 * X, -0.2 + 0.1 * Y, 0.3 * Z
    op = O.StencilOperator(n, dx, D, (bx, by, bz), c=0.25, bc=(O.NEUMANN0,) * 6)
    u = X ** 2 + 2 * Y ** 2 - Z ** 2 + X * Y
    Au = op.matvec(u)
    exact = (2 * a0 + 4 * b1 * X) + b1 * Y + D * (4.0 - 2.0) \
        + bx * (2 * X + Y) + by * (4 * Y + X) + bz * (-2 * Z) + 0.25 * u
    inner = (slice(1, -1),) * 3
    assert np.allclose(Au[inner], exact[inner], rtol=1e-12, atol=1e-10)


def test_neumann_fold_second_order():
    # u = cos(pi x) satisfies the homogeneous Neumann condition; with cell-centred
    # mirror ghosts, A u = -pi^2 D u + O(dx^2) on every row, boundary rows included
    errs = []
    for n in (16, 32, 64):
        dx = 1.0 / n
        x = _grid(n, dx, True)
        op = O.StencilOperator((n, 3), (dx, 1.0), 0.5, (0.0, 0.0),
                               bc=(O.NEUMANN0,) * 4)
        u = np.tile(np.cos(math.pi * x), (3, 1))
        errs.append(np.abs(op.matvec(u) + 0.5 * math.pi ** 2 * u).max())
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.05)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.05)


def test_dirichlet_fold_second_order():
    # u = sin(pi x) sin(pi y) vanishes on the boundary: A u = -2 pi^2 D u + O(dx^2)
    errs = []
    for n in (15, 31, 63):
        dx = 1.0 / (n + 1)
        x = _grid(n, dx, False)
        op = O.StencilOperator((n, n), (dx, dx), 0.3, (0.0, 0.0))
        u = np.outer(np.sin(math.pi * x), np.sin(math.pi * x))
        errs.append(np.abs(op.matvec(u) + 2 * 0.3 * math.pi ** 2 * u).max())
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.1)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.1)


def test_neumann_pure_diffusion_symmetric_conservative():
    rng = np.random.default_rng(3)
    n = (5, 4, 3)
    D = rng.uniform(0.5, 2.0, (3, 4, 5))
    op = O.StencilOperator(n, (0.2, 0.25, 1 / 3), D, (0.0, 0.0, 0.0), bc=(O.NEUMANN0,) * 6)
    M = op.dense()
    assert np.allclose(M, M.T, atol=1e-12)
    assert np.allclose(M.sum(axis=0), 0.0, atol=1e-11)


def test_phi1_closed_form_2d_config(xi):
    # the 64^2 advection-diffusion operator: separable, S^-1 Q f(Lam) Q^T S
    rng = np.random.default_rng(11)
    n, dx, D, b = 64, 1 / 65, 0.1, (-1.0, -0.5)
    op = O.StencilOperator((n, n), (dx, dx), D, b)
    v = rng.standard_normal((n, n))
    y, st = Nw.phi_apply(op, 1, 1e-3, v, 1e-10, xi=xi)
    ex = C.phi_dirichlet_2d(1, 1e-3, v, (n, n), D, b, (dx, dx))
    assert np.linalg.norm(y - ex) / np.linalg.norm(ex) <= 1e-9
    assert st.s == 1 and 5 <= st.degrees[0] <= 30


def test_closed_form_matches_dense():
    # the closed form itself against the definition, small grid
    n, dx, D, b = 9, 0.1, 0.2, (0.8, -0.3)
    op = O.StencilOperator((n, n), (dx, dx), D, b)
    v = np.random.default_rng(5).standard_normal((n, n))
    ex = C.phi_dirichlet_2d(1, 0.02, v, (n, n), D, b, (dx, dx))
    de = Dn.phi_dense(op.dense(), 1, 0.02, v)
    assert np.allclose(ex.ravel(), de, rtol=0, atol=1e-13 * np.abs(de).max())


@pytest.mark.parametrize("k", [0, 1, 2])
@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 1, 1), (0, 1, 1, 0)])
def test_phi_vs_dense_variable_coefficients(xi, k, bc):
    rng = np.random.default_rng(100 + k)
    n = (13, 11)
    dx = (1 / 14, 1 / 12)
    D = rng.uniform(0.05, 0.3, (11, 13))
    b = (rng.uniform(-1, 1, (11, 13)), rng.uniform(-1, 1, (11, 13)))
    c = rng.uniform(-2, 0.5, (11, 13))
    op = O.StencilOperator(n, dx, D, b, c=c, bc=bc)
    v = rng.standard_normal((11, 13))
    h = 2e-3 if k < 2 else 5e-4
    tol = 1e-11
    y, st = Nw.phi_apply(op, k, h, v, tol, xi=xi)
    ex = Dn.phi_dense(op.dense(), k, h, v)
    assert np.linalg.norm(y.ravel() - ex) / np.linalg.norm(ex) <= 100 * tol


def test_phi1_substeps_vs_dense(xi):
    # a large h forces s > 1: the ODE substep form must still give phi_1(hA)v
    rng = np.random.default_rng(7)
    n = (10, 10)
    op = O.StencilOperator(n, (0.1, 0.1), 1.0, (0.5, -0.5), bc=(0, 1, 0, 1))
    v = rng.standard_normal((10, 10))
    y, st = Nw.phi_apply(op, 1, 5.0, v, 1e-10, xi=xi)
    assert st.s > 1
    ex = Dn.phi_dense(op.dense(), 1, 5.0, v)
    assert np.linalg.norm(y.ravel() - ex) / np.linalg.norm(ex) <= 1e-8


def test_phi_diagonal_and_scalar_operator(xi):
    # diagonal A: phi_1(h lam_i) v_i; and A = cI (gamma = 0): phi_k(hc) v
    n = 50
    lam = -np.linspace(0.0, 400.0, n)
    op = O.CsrOperator(n, np.zeros(n + 1, dtype=np.int64), np.zeros(0, np.int64),
                       np.zeros(0), lam)
    v = np.random.default_rng(1).standard_normal(n)
    y, st = Nw.phi_apply(op, 1, 0.01, v, 1e-12, xi=xi)
    ex = np.array([math.expm1(0.01 * l) / (0.01 * l) if l != 0 else 1.0 for l in lam]) * v
    assert np.linalg.norm(y - ex) / np.linalg.norm(ex) <= 1e-10
    op2 = O.CsrOperator(n, np.zeros(n + 1, dtype=np.int64), np.zeros(0, np.int64),
                        np.zeros(0), np.full(n, -3.0))
    for k in (0, 1, 2):
        y2, st2 = Nw.phi_apply(op2, k, 0.1, v, 1e-12, xi=xi)
        assert st2.degrees == [0]
        assert np.allclose(y2, L.phi_scalar(k, -0.3) * v, rtol=1e-15)
    y3, _ = Nw.phi_apply(op2, 1, 0.1, np.zeros(n), 1e-12, xi=xi)
    assert not y3.any()


def test_neumann_closed_form_3d(xi):
    n = (8, 7, 6)
    dx = (1 / 8, 1 / 7, 1 / 6)
    op = O.StencilOperator(n, dx, 0.05, (0.0, 0.0, 0.0), bc=(O.NEUMANN0,) * 6)
    v = np.random.default_rng(2).standard_normal((6, 7, 8))
    y, _ = Nw.phi_apply(op, 1, 0.05, v, 1e-11, xi=xi)
    ex = C.phi_neumann_3d(1, 0.05, v, n, 0.05, dx)
    assert np.linalg.norm(y - ex) / np.linalg.norm(ex) <= 1e-9
    # conservation: column sums of A vanish, so sum(e^{hA} v) = sum(v)
    e, _ = Nw.phi_apply(op, 0, 0.05, v, 1e-12, xi=xi)
    assert abs(e.sum() - v.sum()) <= 1e-11 * np.abs(v).sum()


def test_graph_laplacian_invariants(xi):
    rng = np.random.default_rng(9)
    n = 60
    W = np.triu(rng.uniform(0.5, 2.0, (n, n)) * (rng.random((n, n)) < 0.15), 1)
    W = W + W.T
    rows, cols = np.nonzero(W)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    op = O.CsrOperator(n, rowptr, cols, W[rows, cols], -W.sum(axis=1))
    y, _ = Nw.phi_apply(op, 1, 0.7, np.ones(n), 1e-12, xi=xi)      # A 1 = 0
    assert np.allclose(y, 1.0, atol=1e-12)
    v = rng.standard_normal(n)
    y, _ = Nw.phi_apply(op, 1, 0.7, v, 1e-12, xi=xi)                # 1^T A = 0
    assert abs(y.sum() - v.sum()) <= 1e-11 * np.abs(v).sum()


def test_analytic_gaussian_second_order(xi):
    # u_t = D Lap u + b.grad u from a narrow Gaussian far from the boundary:
    # the discrete e^{tA} u0 approaches the whole-space solution at O(dx^2)
    D, b, sig, t = 0.01, (0.3, -0.2), 0.06, 0.5
    errs = []
    for n in (31, 63):
        dx = 1.0 / (n + 1)
        x = (np.arange(n) + 1) * dx
        Y, X = np.meshgrid(x, x, indexing="ij")
        pts = np.stack([X, Y], axis=-1)
        u0 = C.gaussian(pts, 0.0, D, b, (0.5, 0.5), sig)
        op = O.StencilOperator((n, n), (dx, dx), D, b)
        ut, _ = Nw.phi_apply(op, 0, t, u0, 1e-12, xi=xi)
        errs.append(np.abs(ut - C.gaussian(pts, t, D, b, (0.5, 0.5), sig)).max())
    assert errs[0] < 0.02
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_exp_euler_linear_is_exponential(xi):
    rng = np.random.default_rng(4)
    op = O.StencilOperator((9, 8), (0.1, 0.11), 0.4, (0.2, 0.1), bc=(1, 0, 0, 1))
    u = rng.standard_normal((8, 9))
    un, _ = Nw.exp_euler_step(op, u, 0.01, 1e-12, Nw.NONLIN_NONE, xi=xi)
    ex = Dn.phi_dense(op.dense(), 0, 0.01, u)
    assert np.linalg.norm(un.ravel() - ex) / np.linalg.norm(ex) <= 1e-10


def test_exp_rosenbrock_matches_dense_formula(xi):
    # u+ = u + h phi_1(h J) F, J = A + diag(1 - 2u), F = A u + u(1-u), by dense expm
    rng = np.random.default_rng(8)
    op = O.StencilOperator((7, 6, 5), (0.14, 0.16, 0.2), rng.uniform(0.5, 1.5, (5, 6, 7)),
                           (rng.uniform(-1, 1, (5, 6, 7)),) * 3, bc=(O.NEUMANN0,) * 6)
    u = rng.uniform(0.0, 1.0, (5, 6, 7))
    h = 3e-3
    un, st = Nw.exp_rosenbrock_step(op, u, h, 1e-12, xi=xi)
    A = op.dense()
    uf = u.ravel()
    J = A + np.diag(1.0 - 2.0 * uf)
    F = A @ uf + uf * (1.0 - uf)
    ex = uf + h * Dn.phi_dense(J, 1, h, F)
    assert np.linalg.norm(un.ravel() - ex) / np.linalg.norm(ex) <= 1e-11


def test_exp_rosenbrock_second_order(xi):
    # exponential Rosenbrock-Euler is second order: halving h quarters the error
    rng = np.random.default_rng(12)
    op = O.StencilOperator((6, 6), (1 / 7, 1 / 7), 0.05, (0.2, -0.1))
    u0 = rng.uniform(0.2, 0.8, (6, 6))
    A = op.dense()
    T = 0.4
    ref = scipy.integrate.solve_ivp(lambda t, u: A @ u + u * (1 - u), (0, T), u0.ravel(),
                                    method="DOP853", rtol=1e-13, atol=1e-13).y[:, -1]
    errs = []
    for nsteps in (4, 8, 16):
        u = u0.copy()
        for _ in range(nsteps):
            u, _ = Nw.exp_rosenbrock_step(op, u, T / nsteps, 1e-13, xi=xi)
        errs.append(np.abs(u.ravel() - ref).max())
    assert 3.3 < errs[0] / errs[1] < 4.7
    assert 3.3 < errs[1] / errs[2] < 4.7


@pytest.mark.parametrize("k", [2, 3, 4])
@pytest.mark.parametrize("s", [2, 4, 8])
def test_phik_substeps_vs_dense(xi, k, s):
    """phi_k, k >= 2, by s substeps of the polynomial-forcing ODE (the phi
    recurrence turning each substep into k products and one phi_k run)
    against the augmented-matrix definition."""
    rng = np.random.default_rng(40 + 10 * k + s)
    n = (11, 9)
    op = O.StencilOperator(n, (1 / 12, 1 / 10), 0.2, (0.4, -0.3), bc=(0, 1, 0, 0))
    v = rng.standard_normal((9, 11))
    h = 0.05
    y, st = Nw.phi_apply(op, k, h, v, 1e-12, xi=xi, fixed_s=s)
    assert st.s == s and len(st.degrees) == s
    ex = Dn.phi_dense(op.dense(), k, h, v)
    assert np.linalg.norm(y.ravel() - ex) / np.linalg.norm(ex) <= 1e-9


@pytest.mark.parametrize("k", [2, 3])
def test_phik_schedule_picks_substeps(xi, k):
    """h rho large enough that the a-priori rule needs s > 1 for phi_k."""
    rng = np.random.default_rng(77 + k)
    n = (10, 10)
    op = O.StencilOperator(n, (0.1, 0.1), 1.0, (0.5, -0.5), bc=(0, 1, 0, 1))
    v = rng.standard_normal((10, 10))
    y, st = Nw.phi_apply(op, k, 5.0, v, 1e-10, xi=xi)
    assert st.s > 1
    ex = Dn.phi_dense(op.dense(), k, 5.0, v)
    assert np.linalg.norm(y.ravel() - ex) / np.linalg.norm(ex) <= 1e-7


def test_phik_substeps_diagonal_closed_form(xi):
    """A diagonal: phi_k(h lam) = (e^z - sum_{j<k} z^j/j!)/z^k, z = h lam,
    pointwise, through 4 substeps."""
    n = 30
    lam = -np.linspace(1.0, 300.0, n)
    op = O.CsrOperator(n, np.zeros(n + 1, dtype=np.int64), np.zeros(0, np.int64),
                       np.zeros(0), lam)
    v = np.random.default_rng(3).standard_normal(n)
    h = 0.02
    for k in (2, 3):
        y, st = Nw.phi_apply(op, k, h, v, 1e-13, xi=xi, fixed_s=4)
        z = h * lam
        ex = np.array([(math.exp(t) - sum(t ** j / math.factorial(j) for j in range(k))) / t ** k
                       for t in z]) * v
        assert np.linalg.norm(y - ex) / np.linalg.norm(ex) <= 1e-9
