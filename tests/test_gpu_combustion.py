"""The combustion nonlinearity of Sec. III-C on the GPU (through the C ABI)
against the oracle (oracle/newton.py: combustion, exp_euler_step,
exp_rosenbrock_step).

Bars:
- pointwise g and g':
  - float-float: 1e-11 relative. The reciprocal is good to ~1.4e-14 and the
    exponential to ~2^-46; the argument 20(1 - 1/u) turns a relative error e
    of 1/u into 20 e / u <= 100 e on u >= 0.2.
  - native FP64 (the math library): 5e-14, the same amplification of about
    one ulp.
  - FP32 full (expf, IEEE division): 3e-5. The argument's absolute error is
    about 20 (5 * 6e-8 + 2.4e-7) + 3.8e-6 = 1.5e-5 at u = 0.2, plus the few
    ulps of expf.
  - fast (__expf, __fdividef): 1e-4, adding __expf's error of up to
    2 + 1.16|x| ulp at |x| <= 80.
  g' is held to the same bound relative to the size of its two terms,
  e^{20(1-1/u)} (|20 (2-u)/u^2| + 1) / 4, since they cancel where g is largest.
  FP64 arrays (float-float and native) are held to the relative bound at every
  u above the cut, with no absolute floor: below u = 1/4, where
  e^{20(1-1/u)} < 2^-100 leaves the float-float range, the float-float variant
  evaluates in native FP64.  The FP32 variants keep FP32's range: below
  u = 0.2 their bound is absolute (1e-30).
- below the cut both are exactly 0; a NaN u gives NaN.
- steps (exponential Euler and Rosenbrock-Euler) on 3D stencils and CSR:
  - the full form: 1e-9 relative with identical degrees, and the Rosenbrock
    interval within 1e-13;
  - the FP32 form: 3e-5 on the increment;
  - the fast form: 2e-4 on the increment (g and g' to ~5e-5, scaled by the
    step).
"""
import numpy as np
import pytest

from oracle import leja as L
from oracle import newton as Nw
from oracle import operators as O
from paper_1309_4616_gb300 import workloads as W

from gpu_helpers import dev, rel_err, require_gpu, stencil_context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return require_gpu()


@pytest.fixture(scope="module")
def xi():
    return L.leja_points(100)


def _u_sweep():
    # the cut, the range where float-float underflows but FP64 does not,
    # the physical range [1, 2] and beyond
    return np.concatenate([[-1.0, 0.0, 0.01, Nw.COMBUSTION_CUT],
                           np.linspace(0.026, 0.2, 175, endpoint=False),
                           np.linspace(0.2, 2.6, 2401)])


@pytest.mark.parametrize("variant", ["df", "native", "f32", "fast64", "fast32"])
def test_pointwise_against_oracle(env, variant):
    torch, ei = env
    u0 = _u_sweep()
    kind = ei.NONLIN_COMBUSTION_FAST if variant.startswith("fast") else ei.NONLIN_COMBUSTION
    f32 = variant in ("f32", "fast32")
    dt = torch.float32 if f32 else torch.float64
    uin = u0.astype(np.float32).astype(np.float64) if f32 else u0
    gref, dref = Nw.combustion(uin)
    u = dev(torch, uin, dt)
    g = torch.empty_like(u)
    dg = torch.empty_like(u)
    arith = ei.ARITH_NATIVE_F64 if variant == "native" else ei.ARITH_DF
    ei.nonlinearity(kind, u, g, dg, arith=arith)
    torch.cuda.synchronize()
    got_g = g.cpu().numpy().astype(np.float64)
    got_d = dg.cpu().numpy().astype(np.float64)
    rtol = {"df": 1e-11, "native": 5e-14, "f32": 3e-5, "fast64": 1e-4, "fast32": 1e-4}[variant]
    # g' is a difference of two terms that cancel at u* = sqrt(140) - 10: its
    # error is bounded relative to the size of those terms
    uc = np.maximum(uin, 1e-3)
    e4 = 0.25 * np.exp(20.0 * (1.0 - 1.0 / uc))
    dscale = e4 * (np.abs(20.0 * (2.0 - uc) / uc ** 2) + 1.0)
    if variant in ("df", "native"):
        # FP64 arrays: relative at every u above the cut where the exponential
        # factor e4 is a normal double; where FP64 itself goes subnormal
        # (u < ~0.0275), within four subnormal ulps of it
        tiny = np.finfo(np.float64).tiny
        above = uin > Nw.COMBUSTION_CUT
        on = above & (e4 >= tiny)
        sub = above & ~on
        assert on.sum() > 2400 and (uin[on] < 0.05).any()
        assert (np.abs(got_g[on] - gref[on]) <= rtol * np.abs(gref[on])).all()
        assert (np.abs(got_d[on] - dref[on]) <= rtol * dscale[on]).all()
        # (g' = e4 (20 (2-u)/u^2 - 1): a subnormal e4's ulps scale by that factor)
        fac = np.abs(20.0 * (2.0 - uc) / uc ** 2) + 1.0
        assert (np.abs(got_g[sub] - gref[sub]) <= 2e-323).all()
        assert (np.abs(got_d[sub] - dref[sub]) <= 2e-323 * fac[sub]).all()
    else:
        # FP32 arithmetic: relative from u = 0.2, absolute below (FP32's range)
        on = uin >= 0.2
        assert (np.abs(got_g[on] - gref[on]) <= rtol * np.maximum(np.abs(gref[on]), 1e-29)).all()
        assert (np.abs(got_d[on] - dref[on]) <= rtol * np.maximum(dscale[on], 1e-29)).all()
        assert np.abs(got_g[~on] - gref[~on]).max() <= 1e-30
    cut = uin <= Nw.COMBUSTION_CUT
    assert (got_g[cut] == 0).all() and (got_d[cut] == 0).all()


def test_nan_aliasing_logistic_and_invalid(env):
    torch, ei = env
    u = torch.tensor([1.0, float("nan"), 1.5], dtype=torch.float64, device="cuda")
    g = torch.empty_like(u)
    ei.nonlinearity(ei.NONLIN_COMBUSTION, u, g)
    out = g.cpu().numpy()
    assert np.isnan(out[1]) and out[0] == pytest.approx(0.25, rel=1e-14)
    # in place, g aliasing u; the logistic term through the same entry
    x = np.linspace(-1, 2, 101)
    t = dev(torch, x)
    ei.nonlinearity(ei.NONLIN_LOGISTIC, t, t)
    # float-float keeps 48 of the input's 53 bits (2^-48 relative), and 1 - x
    # cancels near x = 1: the error is bounded relative to the size of the
    # terms, |x| (1 + |x|), as for g' above
    err = np.abs(t.cpu().numpy() - x * (1 - x))
    assert (err <= 1e-14 * np.abs(x) * (1 + np.abs(x)) + 1e-16).all()
    with pytest.raises(ei.EIError) as e:
        ei.nonlinearity(7, u, g)
    assert e.value.status == ei.ERR_INVALID_ARG


def _combustion_field(n, seed):
    """u0 in [1, 2]: the physical range of the combustion model, smooth."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = n[2], n[1], n[0]
    z, y, x = np.meshgrid(*(np.linspace(0, 1, k) for k in (nz, ny, nx)), indexing="ij")
    a = rng.uniform(0.5, 1.5, 3)
    return 1.5 + 0.45 * np.sin(np.pi * a[0] * x) * np.cos(np.pi * a[1] * y) * np.sin(np.pi * a[2] * z + 0.3)


@pytest.mark.parametrize("method", ["euler", "rosenbrock"])
@pytest.mark.parametrize("arith", [0, 1])
def test_stencil_steps_full(env, xi, method, arith):
    """The combustion model of Sec. III-C: u_t = Laplace(u) + g(u), homogeneous
    Dirichlet, on a 3D grid with ragged tiles."""
    torch, ei = env
    n = (35, 22, 19)
    dx = (1 / 36,) * 3
    u0 = _combustion_field(n, 3)
    op = O.StencilOperator(n, dx, np.ones((19, 22, 35)), (np.zeros((19, 22, 35)),) * 3,
                           bc=(O.DIRICHLET0,) * 6)
    h, tol = 2e-4, 1e-10
    step = Nw.exp_euler_step if method == "euler" else Nw.exp_rosenbrock_step
    ref, ost = step(op, u0, h, tol, nonlin=Nw.NONLIN_COMBUSTION, xi=xi)
    ctx = stencil_context(torch, ei, n, dx, 1.0, (0.0, 0.0, 0.0), 0.0, (0,) * 6)
    u = dev(torch, u0)
    m = ei.EXP_EULER if method == "euler" else ei.EXP_ROSENBROCK
    st = ctx.step(m, h, u, ei.NONLIN_COMBUSTION, tol, {"arith": arith})
    got = u.cpu().numpy()
    assert rel_err(got - u0, ref - u0) <= 1e-9
    assert st.s == ost.s and st.degree_list() == list(ost.degrees)
    if method == "rosenbrock":
        assert st.alpha == pytest.approx(ost.alpha, rel=1e-13)
        assert st.beta == pytest.approx(ost.beta, rel=1e-13)
    ctx.close()


def test_csr_rosenbrock_full(env, xi):
    torch, ei = env
    g = W.rgg_graph(n=3000, seed=41)
    op = O.CsrOperator(g.n, g.rowptr, g.col, g.val, -g.deg_w)
    u0 = np.random.default_rng(5).uniform(1.0, 2.0, g.n)
    h = 1e-3
    ref, ost = Nw.exp_rosenbrock_step(op, u0, h, 1e-10, nonlin=Nw.NONLIN_COMBUSTION, xi=xi)
    ctx = ei.Context()
    ctx.set_operator_csr(g.n, dev(torch, g.rowptr), dev(torch, g.col), dev(torch, g.val),
                         dev(torch, -g.deg_w))
    u = dev(torch, u0)
    st = ctx.step(ei.EXP_ROSENBROCK, h, u, ei.NONLIN_COMBUSTION, 1e-10)
    assert rel_err(u.cpu().numpy() - u0, ref - u0) <= 1e-9
    assert st.s == ost.s and st.degree_list() == list(ost.degrees)
    ctx.close()


@pytest.mark.parametrize("prec,kind,bar", [(0, 3, 2e-4), (1, 2, 3e-5), (1, 3, 2e-4)])
def test_stencil_rosenbrock_fp32_and_fast(env, xi, prec, kind, bar):
    torch, ei = env
    n = (33, 20, 17)
    dx = (1 / 34,) * 3
    u0 = _combustion_field(n, 4)
    if prec == 1:
        u0 = u0.astype(np.float32).astype(np.float64)
    op = O.StencilOperator(n, dx, np.ones((17, 20, 33)), (np.zeros((17, 20, 33)),) * 3,
                           bc=(O.DIRICHLET0,) * 6)
    h = 2e-4
    tol = 1e-10 if prec == 0 else 1e-6
    ref, _ = Nw.exp_rosenbrock_step(op, u0, h, 1e-12, nonlin=Nw.NONLIN_COMBUSTION, xi=xi)
    ctx = stencil_context(torch, ei, n, dx, 1.0, (0.0, 0.0, 0.0), 0.0, (0,) * 6, prec=prec)
    u = dev(torch, u0, torch.float32 if prec else torch.float64)
    ctx.step(ei.EXP_ROSENBROCK, h, u, kind, tol)
    got = u.cpu().numpy().astype(np.float64)
    assert rel_err(got - u0, ref - u0) <= bar
    ctx.close()
