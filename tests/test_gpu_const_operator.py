"""The table form of a constant-coefficient stencil operator on the GPU.

When D, b and c are all constants, the float-float two-iteration Newton kernel
reads the scaled operator (A - cI)/gamma from a table: the six off-diagonals
and the diagonal of each class of points by the faces they touch (64 classes).
Each case runs one operator twice, given by constants (the table form:
stats.coef_table > 0) and by arrays holding the same constants (the
coefficient arrays: stats.coef_table == 0), and compares
- each with the FP64 oracle at the 1e-9 relative 2-norm bound, with identical
  substeps and degrees;
- the two forms with each other at 1e-14 relative: the table holds the very
  values of the scaled coefficient arrays, and the forms differ only where an
  off-diagonal towards a ghost point multiplies the zero the ghost holds.
Shapes: ragged tiles in x and y, z extents of 2 to 21 planes, an extent of 1
or 2 on one axis (classes on both faces at once, no interior class), 2D, and
mixes of Dirichlet and Neumann faces.
"""
import numpy as np
import pytest

from oracle import leja as L
from oracle import newton as Nw
from oracle import operators as O

from gpu_helpers import dev, rel_err, require_gpu, stencil_context

pytestmark = pytest.mark.gpu

TOL = 1e-9
SAME = 1e-14

CASES = [
    # n, bc, D, b, c
    ((37, 29, 21), (1, 0, 1, 1, 0, 1), 0.8, (0.5, -0.3, 0.2), -0.7),
    ((33, 9, 3), (0,) * 6, 1.0, (0.0, 0.0, 0.0), 0.0),
    ((40, 2, 7), (0, 1, 1, 0, 1, 0), 0.3, (-1.0, 0.4, 0.6), 0.2),
    ((1, 12, 17), (1, 1, 0, 1, 0, 0), 0.5, (0.3, 0.2, -0.1), 0.0),
    ((61, 45), (1, 0, 0, 1), 0.6, (0.7, -0.2), -0.3),
]


@pytest.fixture(scope="module")
def env():
    return require_gpu()


@pytest.fixture(scope="module")
def xi():
    return L.leja_points(100)


def _forms(torch, ei, n, dx, D, b, c, bc):
    shape = tuple(reversed(n))
    const = stencil_context(torch, ei, n, dx, D, b, c, bc)
    arrays = stencil_context(torch, ei, n, dx, np.full(shape, D),
                             [np.full(shape, x) for x in b], np.full(shape, c), bc)
    return const, arrays


def _oracle_op(n, dx, D, b, c, bc):
    shape = tuple(reversed(n))
    return O.StencilOperator(n, dx, np.full(shape, D), tuple(np.full(shape, x) for x in b),
                             c=np.full(shape, c), bc=bc)


def _h(n, dx, D, target):
    # h rho near `target`, rho ~ 4 D sum 1/dx^2
    return target / (4.0 * D * sum(1.0 / (d * d) for d in dx))


@pytest.mark.parametrize("case", range(len(CASES)))
def test_phi1_table_form(env, xi, case):
    torch, ei = env
    n, bc, D, b, c = CASES[case]
    dx = tuple(1.0 / (v + 1) for v in n)
    shape = tuple(reversed(n))
    v0 = np.random.default_rng(70 + case).standard_normal(shape)
    h, tol = _h(n, dx, D, 30.0), 1e-10
    ref, ost = Nw.phi_apply(_oracle_op(n, dx, D, b, c, bc), 1, h, v0, tol, xi=xi)
    const, arrays = _forms(torch, ei, n, dx, D, b, c, bc)
    outs = []
    for ctx, table in ((const, True), (arrays, False)):
        v = dev(torch, v0)
        out = torch.empty_like(v)
        st = ctx.phi_apply(1, h, v, out, tol, {"arith": ei.ARITH_DF})
        assert st.arith_used == ei.ARITH_DF
        assert (st.coef_table > 0) == table
        got = out.cpu().numpy()
        assert rel_err(got, ref) <= TOL
        assert st.s == ost.s and st.degree_list() == list(ost.degrees)
        outs.append(got)
        ctx.close()
    assert rel_err(outs[0], outs[1]) <= SAME


@pytest.mark.parametrize("case", [0, 2])
def test_phi1_table_form_substeps(env, xi, case):
    # s > 1: the table serves every substep's Newton loop
    torch, ei = env
    n, bc, D, b, c = CASES[case]
    dx = tuple(1.0 / (v + 1) for v in n)
    shape = tuple(reversed(n))
    v0 = np.random.default_rng(80 + case).standard_normal(shape)
    h, tol = _h(n, dx, D, 1500.0), 1e-10
    ref, ost = Nw.phi_apply(_oracle_op(n, dx, D, b, c, bc), 1, h, v0, tol, xi=xi)
    assert ost.s > 1
    const, arrays = _forms(torch, ei, n, dx, D, b, c, bc)
    outs = []
    for ctx, table in ((const, True), (arrays, False)):
        v = dev(torch, v0)
        out = torch.empty_like(v)
        st = ctx.phi_apply(1, h, v, out, tol)
        assert (st.coef_table > 0) == table
        got = out.cpu().numpy()
        assert rel_err(got, ref) <= TOL
        assert st.s == ost.s and st.degree_list() == list(ost.degrees)
        outs.append(got)
        ctx.close()
    assert rel_err(outs[0], outs[1]) <= SAME


def test_combustion_euler_step_table_form(env, xi):
    # the combustion model of Sec. III-C on the Laplacian (Table 4's operator)
    torch, ei = env
    n = (35, 22, 19)
    dx = (1 / 36,) * 3
    shape = tuple(reversed(n))
    rng = np.random.default_rng(91)
    u0 = 1.0 + 0.2 * rng.uniform(0.0, 1.0, shape)
    op = _oracle_op(n, dx, 1.0, (0.0, 0.0, 0.0), 0.0, (0,) * 6)
    h, tol = 2e-4, 1e-10
    ref, ost = Nw.exp_euler_step(op, u0, h, tol, nonlin=Nw.NONLIN_COMBUSTION, xi=xi)
    const, arrays = _forms(torch, ei, n, dx, 1.0, (0.0, 0.0, 0.0), 0.0, (0,) * 6)
    outs = []
    for ctx, table in ((const, True), (arrays, False)):
        u = dev(torch, u0)
        st = ctx.step(ei.EXP_EULER, h, u, ei.NONLIN_COMBUSTION, tol)
        assert (st.coef_table > 0) == table
        got = u.cpu().numpy()
        assert rel_err(got - u0, ref - u0) <= TOL
        assert st.s == ost.s and st.degree_list() == list(ost.degrees)
        outs.append(got)
        ctx.close()
    assert rel_err(outs[0] - u0, outs[1] - u0) <= SAME


def test_rosenbrock_step_keeps_arrays(env, xi):
    # J = A + diag g'(u) varies from point to point: no table
    torch, ei = env
    n = (35, 22, 19)
    dx = (1 / 36,) * 3
    shape = tuple(reversed(n))
    u0 = 1.0 + 0.2 * np.random.default_rng(92).uniform(0.0, 1.0, shape)
    op = _oracle_op(n, dx, 1.0, (0.0, 0.0, 0.0), 0.0, (0,) * 6)
    h, tol = 2e-4, 1e-10
    ref, ost = Nw.exp_rosenbrock_step(op, u0, h, tol, nonlin=Nw.NONLIN_COMBUSTION, xi=xi)
    ctx = stencil_context(torch, ei, n, dx, 1.0, (0.0, 0.0, 0.0), 0.0, (0,) * 6)
    u = dev(torch, u0)
    st = ctx.step(ei.EXP_ROSENBROCK, h, u, ei.NONLIN_COMBUSTION, tol)
    assert st.coef_table == 0
    assert rel_err(u.cpu().numpy() - u0, ref - u0) <= TOL
    assert st.s == ost.s and st.degree_list() == list(ost.degrees)
    ctx.close()
