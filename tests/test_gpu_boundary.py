"""Inhomogeneous Dirichlet data through the C ABI (ei_set_dirichlet_values)
against the oracle (StencilOperator.boundary_vector with the exponential
steps).  The boundary functions are the paper's two examples of Sec. III-A,
z(1-z)xy and sin(pi z) exp(-xy), evaluated at the ghost points of a
vertex-centred grid.

Bars: FP64 1e-9 relative on the step's increment with identical degrees;
FP32 1e-5; a steady state (a linear function with its own data, b = 0) moves
by less than 1e-12; errors as include/ei.h states."""
import numpy as np
import pytest

from oracle import leja as L
from oracle import newton as Nw
from oracle import operators as O

from gpu_helpers import dev, rel_err, require_gpu, stencil_context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return require_gpu()


@pytest.fixture(scope="module")
def xi():
    return L.leja_points(100)


def f_poly(x, y, z):
    return z * (1 - z) * x * y


def f_trig(x, y, z):
    return np.sin(np.pi * z) * np.exp(-x * y)


def _axes(n):
    return [np.arange(1, k + 1) / (k + 1) for k in n]


def faces_of(n, f):
    """f at the ghost points of each face, in the library's face layout."""
    x, y, z = _axes(n) if len(n) == 3 else (*_axes(n), np.array([0.0]))
    Zy, Yz = np.meshgrid(z, y, indexing="ij")
    Zx, Xz = np.meshgrid(z, x, indexing="ij")
    Yx, Xy = np.meshgrid(y, x, indexing="ij")
    out = [f(0 * Zy, Yz, Zy), f(1 + 0 * Zy, Yz, Zy), f(Xz, 0 * Zx, Zx), f(Xz, 1 + 0 * Zx, Zx),
           f(Xy, Yx, 0 * Yx), f(Xy, Yx, 1 + 0 * Yx)]
    return out[: 2 * len(n)]


def _fields(rng, shape):
    D = 0.5 + rng.uniform(0, 1, shape)
    b = tuple(rng.uniform(-1, 1, shape) for _ in range(3))
    return D, b


@pytest.mark.parametrize("func", [f_poly, f_trig])
@pytest.mark.parametrize("method", ["euler", "rosenbrock"])
def test_steps_with_boundary_data(env, xi, func, method):
    torch, ei = env
    rng = np.random.default_rng(31)
    n = (37, 22, 19)
    dx = tuple(1.0 / (k + 1) for k in n)
    D, b = _fields(rng, (19, 22, 37))
    u0 = rng.uniform(0, 1, (19, 22, 37))
    op = O.StencilOperator(n, dx, D, b, bc=(O.DIRICHLET0,) * 6)
    faces = faces_of(n, func)
    bv = op.boundary_vector(faces)
    h, tol = 2e-4, 1e-10
    if method == "euler":
        ref, ost = Nw.exp_euler_step(op, u0, h, tol, Nw.NONLIN_LOGISTIC, xi=xi, bvec=bv)
    else:
        ref, ost = Nw.exp_rosenbrock_step(op, u0, h, tol, xi=xi, bvec=bv)
    ctx = stencil_context(torch, ei, n, dx, D, b, 0.0, (0,) * 6)
    ctx.set_dirichlet_values([dev(torch, f) for f in faces])
    u = dev(torch, u0)
    m = ei.EXP_EULER if method == "euler" else ei.EXP_ROSENBROCK
    st = ctx.step(m, h, u, ei.NONLIN_LOGISTIC, tol)
    got = u.cpu().numpy()
    assert rel_err(got - u0, ref - u0) <= 1e-9
    assert st.s == ost.s and st.degree_list() == list(ost.degrees)
    ctx.close()


def test_steady_state_and_clearing(env, xi):
    torch, ei = env
    n = (40, 33, 17)
    dx = tuple(1.0 / (k + 1) for k in n)
    lin = lambda x, y, z: 1.0 + 0.5 * x - y + 2.0 * z
    x, y, z = _axes(n)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    u0 = lin(X, Y, Z)
    ctx = stencil_context(torch, ei, n, dx, 0.7, (0.0, 0.0, 0.0), 0.0, (0,) * 6)
    ctx.set_dirichlet_values([dev(torch, f) for f in faces_of(n, lin)])
    u = dev(torch, u0)
    ctx.step(ei.EXP_EULER, 1e-3, u, ei.NONLIN_NONE, 1e-10)
    assert np.abs(u.cpu().numpy() - u0).max() < 1e-12
    # cleared: the homogeneous step, as the oracle without data
    ctx.set_dirichlet_values(None)
    op = O.StencilOperator(n, dx, 0.7, (0.0, 0.0, 0.0), bc=(O.DIRICHLET0,) * 6)
    ref, _ = Nw.exp_euler_step(op, u0, 1e-3, 1e-10, xi=xi)
    u = dev(torch, u0)
    ctx.step(ei.EXP_EULER, 1e-3, u, ei.NONLIN_NONE, 1e-10)
    assert rel_err(u.cpu().numpy() - u0, ref - u0) <= 1e-9
    ctx.close()


def test_2d_some_faces_and_fp32(env, xi):
    """2D, data on two of the Dirichlet faces, Neumann faces without data; the
    FP32 operator on FP32-representable inputs."""
    torch, ei = env
    rng = np.random.default_rng(7)
    n = (45, 38)
    dx = tuple(1.0 / (k + 1) for k in n)
    bc = (0, 0, 1, 0)
    D = (0.5 + rng.uniform(0, 1, (38, 45))).astype(np.float32).astype(np.float64)
    b = [rng.uniform(-1, 1, (38, 45)).astype(np.float32).astype(np.float64) for _ in range(2)]
    u0 = rng.uniform(0, 1, (38, 45)).astype(np.float32).astype(np.float64)
    fc = faces_of(n, lambda x, y, z: np.cos(3 * x) + y * y)
    faces = [fc[0].astype(np.float32).astype(np.float64), None, None,
             fc[3].astype(np.float32).astype(np.float64)]
    op = O.StencilOperator(n, dx, D, b, bc=bc)
    bv = op.boundary_vector(faces)
    h = 5e-4
    ref, _ = Nw.exp_euler_step(op, u0, h, 1e-12, Nw.NONLIN_LOGISTIC, xi=xi, bvec=bv)
    for prec, bar in ((0, 1e-9), (1, 1e-5)):
        dt = torch.float64 if prec == 0 else torch.float32
        ctx = stencil_context(torch, ei, n, dx, D, b, 0.0, bc, prec=prec)
        ctx.set_dirichlet_values([None if f is None else dev(torch, f, dt) for f in faces])
        u = dev(torch, u0, dt)
        ctx.step(ei.EXP_EULER, h, u, ei.NONLIN_LOGISTIC, 1e-10 if prec == 0 else 1e-6)
        assert rel_err(u.cpu().numpy().astype(np.float64) - u0, ref - u0) <= bar
        ctx.close()


def test_errors(env):
    torch, ei = env
    n = (20, 12, 9)
    dx = (0.05, 0.05, 0.05)
    ctx = stencil_context(torch, ei, n, dx, 1.0, (0.0, 0.0, 0.0), 0.0, (1, 0, 0, 0, 0, 0))
    with pytest.raises(ei.EIError) as e:  # face 0 is Neumann
        ctx.set_dirichlet_values([torch.zeros(12 * 9, dtype=torch.float64, device="cuda")])
    assert e.value.status == ei.ERR_INVALID_ARG
    with pytest.raises(ValueError):  # wrong face size, refused by the binding
        ctx.set_dirichlet_values([None, torch.zeros(5, dtype=torch.float64, device="cuda")])
    ctx.close()
    g = ei.Context()
    with pytest.raises(ei.EIError) as e:  # no stencil operator
        g.set_dirichlet_values([None] * 6)
    assert e.value.status == ei.ERR_STATE
    g.close()
