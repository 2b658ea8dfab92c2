"""The float-float format's range (ei_options.arith = EI_ARITH_DF) on the GPU.

Float-float pairs carry 48 significand bits but only FP32's exponents, so a
float-float call runs only inside the range the library states (include/ei.h,
EI_ARITH_DF); any other call must run in native FP64 and say so in
stats.arith_used.  Each case below is compared with the FP64 oracle at the
1e-9 relative 2-norm bound of the F64 contract, with no absolute floor:
- vectors scaled far below and above the range (v * 1e-40, 1e-150, 1e40, 1e150;
  the squared norms of larger scales overflow FP64 itself, in the oracle too);
- operators whose coefficients sit near the edges (D * 1e-30 with h * 1e30,
  D * 1e25 with h * 1e-25: the same h A);
- steps from a tiny state and a linear step from a huge one;
- complex vectors for phi(-i h H) v;
- controls inside the range, which must stay in float-float.
The pointwise combustion term down to u = 0.05 is held to its relative bound
in tests/test_gpu_combustion.py.
"""
import numpy as np
import pytest

from oracle import leja as L
from oracle import newton as Nw
from oracle import operators as O
from oracle import skew as S
from paper_1309_4616_gb300 import workloads as W

from gpu_helpers import dev, rel_err, require_gpu, stencil_context

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def env():
    return require_gpu()


@pytest.fixture(scope="module")
def xi():
    return L.leja_points(100)


def _fields(seed, n):
    rng = np.random.default_rng(seed)
    shape = tuple(reversed(n))
    D = rng.uniform(0.5, 1.5, shape)
    b = tuple(rng.uniform(-2, 2, shape) for _ in range(3))
    return rng, D, b


@pytest.mark.parametrize("scale,native", [(1.0, False), (1e-10, False), (1e-40, True),
                                          (1e-150, True), (1e40, True), (1e150, True)])
def test_phi1_scaled_vector(env, xi, scale, native):
    torch, ei = env
    n = (37, 29, 21)
    dx = (1 / 37,) * 3
    rng, D, b = _fields(31, n)
    v0 = rng.standard_normal(tuple(reversed(n))) * scale
    op = O.StencilOperator(n, dx, D, b, bc=(1,) * 6)
    h, tol = 2e-4, 1e-10
    ref, ost = Nw.phi_apply(op, 1, h, v0, tol, xi=xi)
    ctx = stencil_context(torch, ei, n, dx, D, b, 0.0, (1,) * 6)
    v = dev(torch, v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply(1, h, v, out, tol, {"arith": ei.ARITH_DF})
    assert st.arith_used == (ei.ARITH_NATIVE_F64 if native else ei.ARITH_DF)
    assert rel_err(out.cpu().numpy(), ref) <= TOL
    assert st.s == ost.s and st.degree_list() == list(ost.degrees)
    ctx.close()


@pytest.mark.parametrize("dscale", [1e-30, 1e25])
def test_phi1_operator_near_the_edges(env, xi, dscale):
    # D * dscale, b * dscale and h / dscale: the same h A, with coefficients near
    # 1e-26 or 1e29 (rho outside [2^-60, 2^60])
    torch, ei = env
    n = (33, 18, 12)
    dx = (1 / 33,) * 3
    rng, D, b = _fields(32, n)
    D, b = D * dscale, tuple(x * dscale for x in b)
    v0 = rng.standard_normal(tuple(reversed(n)))
    op = O.StencilOperator(n, dx, D, b, bc=(0, 1, 1, 0, 1, 1))
    h, tol = 3e-4 / dscale, 1e-10
    ref, ost = Nw.phi_apply(op, 1, h, v0, tol, xi=xi)
    ctx = stencil_context(torch, ei, n, dx, D, b, 0.0, (0, 1, 1, 0, 1, 1))
    v = dev(torch, v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply(1, h, v, out, tol, {"arith": ei.ARITH_DF})
    assert st.arith_used == ei.ARITH_NATIVE_F64
    assert rel_err(out.cpu().numpy(), ref) <= TOL
    assert st.s == ost.s and st.degree_list() == list(ost.degrees)
    ctx.close()


@pytest.mark.parametrize("uscale,native", [(1.0, False), (1e-30, True)])
def test_rosenbrock_step_tiny_state(env, xi, uscale, native):
    torch, ei = env
    n = (29, 23, 17)
    dx = (1 / 29,) * 3
    rng, D, b = _fields(33, n)
    u0 = rng.uniform(0, 1, tuple(reversed(n))) * uscale
    op = O.StencilOperator(n, dx, D, b, bc=(1,) * 6)
    h, tol = 2e-4, 1e-10
    ref, ost = Nw.exp_rosenbrock_step(op, u0, h, tol, xi=xi)
    ctx = stencil_context(torch, ei, n, dx, D, b, 0.0, (1,) * 6)
    u = dev(torch, u0)
    st = ctx.step(ei.EXP_ROSENBROCK, h, u, ei.NONLIN_LOGISTIC, tol, {"arith": ei.ARITH_DF})
    got = u.cpu().numpy()
    assert st.arith_used == (ei.ARITH_NATIVE_F64 if native else ei.ARITH_DF)
    assert rel_err(got - u0, ref - u0) <= TOL
    assert rel_err(got, ref) <= TOL
    assert st.s == ost.s and st.degree_list() == list(ost.degrees)
    ctx.close()


def test_linear_euler_step_huge_state(env, xi):
    # g = 0: u * 1e30 gives F = A u * 1e30, whose squares leave FP32's range
    torch, ei = env
    n = (29, 23, 17)
    dx = (1 / 29,) * 3
    rng, D, b = _fields(34, n)
    u0 = rng.uniform(0, 1, tuple(reversed(n))) * 1e30
    op = O.StencilOperator(n, dx, D, b, bc=(1,) * 6)
    h, tol = 2e-4, 1e-10
    ref, ost = Nw.exp_euler_step(op, u0, h, tol, Nw.NONLIN_NONE, xi=xi)
    ctx = stencil_context(torch, ei, n, dx, D, b, 0.0, (1,) * 6)
    u = dev(torch, u0)
    st = ctx.step(ei.EXP_EULER, h, u, ei.NONLIN_NONE, tol, {"arith": ei.ARITH_DF})
    got = u.cpu().numpy()
    assert st.arith_used == ei.ARITH_NATIVE_F64
    assert rel_err(got - u0, ref - u0) <= TOL
    assert st.s == ost.s and st.degree_list() == list(ost.degrees)
    ctx.close()


@pytest.mark.parametrize("scale,native", [(1.0, False), (1e-40, True), (1e60, True)])
def test_complex_scaled_vector(env, xi, scale, native):
    torch, ei = env
    g = W.spin_bath(9)
    op = O.CsrOperator(g.n, g.rowptr, g.col, g.val, g.diag)
    v0 = W.spin_state(g.n, 8) * scale
    h = 0.8
    ref, s, degs = S.phi_apply_imag(op, 0, h, v0, 1e-10, xi=xi)
    ctx = ei.Context()
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx.set_operator_csr(g.n, cu(g.rowptr), cu(g.col), cu(g.val), cu(g.diag))
    v = cu(v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply_imag(0, h, v, out, 1e-10, {"arith": ei.ARITH_DF})
    assert st.arith_used == (ei.ARITH_NATIVE_F64 if native else ei.ARITH_DF)
    got = out.cpu().numpy()
    assert np.linalg.norm(got - ref) <= TOL * np.linalg.norm(ref)
    assert st.s == s and st.degree_list() == list(degs)
    ctx.close()
