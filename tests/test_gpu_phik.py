"""phi_k(hA)v for k >= 2 with substeps through the C ABI, against the oracle
(oracle/newton.py: h_phik_substeps, the polynomial-forcing ODE form with the
phi recurrence) and, on small grids, the augmented-matrix definition
(oracle/dense.py).

Bars: FP64 1e-9 relative with identical per-substep degrees and s; FP32 1e-5;
against the dense definition 1e-7 (the method's own tolerance 1e-10)."""
import numpy as np
import pytest

from oracle import dense as Dn
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


def _fields2d(rng, n):
    nx, ny = n
    D = 0.2 + 0.3 * rng.uniform(0, 1, (ny, nx))
    b = (rng.uniform(-1, 1, (ny, nx)), rng.uniform(-1, 1, (ny, nx)))
    return D, b


@pytest.mark.parametrize("k", [2, 3, 4])
@pytest.mark.parametrize("s", [1, 2, 3, 4])
def test_fixed_substeps_stencil(env, xi, k, s):
    torch, ei = env
    rng = np.random.default_rng(10 * k + s)
    n, dx, bc = (47, 33), (1 / 48, 1 / 34), (0, 1, 1, 0)
    D, b = _fields2d(rng, n)
    v0 = rng.standard_normal((33, 47))
    h, tol = 4e-3, 1e-10
    op = O.StencilOperator(n, dx, D, b, bc=bc)
    ref, ost = Nw.phi_apply(op, k, h, v0, tol, xi=xi, fixed_s=s)
    ctx = stencil_context(torch, ei, n, dx, D, b, 0.0, bc)
    v = dev(torch, v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply(k, h, v, out, tol, {"fixed_s": s})
    assert rel_err(out.cpu().numpy(), ref) <= 1e-9
    assert st.s == s and st.degree_list() == list(ost.degrees)
    ctx.close()


@pytest.mark.parametrize("k", [2, 3])
def test_schedule_substeps_against_definition(env, xi, k):
    """A large h rho: the a-priori rule takes s > 1; the result matches the
    oracle and the augmented-matrix phi_k."""
    torch, ei = env
    rng = np.random.default_rng(5 + k)
    n, dx, bc = (14, 12), (0.07, 0.08), (0, 1, 0, 1)
    op = O.StencilOperator(n, dx, 1.0, (0.5, -0.5), bc=bc)
    v0 = rng.standard_normal((12, 14))
    h, tol = 4.0, 1e-10
    ref, ost = Nw.phi_apply(op, k, h, v0, tol, xi=xi)
    assert ost.s > 1
    ctx = stencil_context(torch, ei, n, dx, 1.0, (0.5, -0.5), 0.0, bc)
    v = dev(torch, v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply(k, h, v, out, tol)
    got = out.cpu().numpy()
    assert st.s == ost.s and st.degree_list() == list(ost.degrees)[: len(st.degree_list())]
    assert rel_err(got, ref) <= 1e-9
    ex = Dn.phi_dense(op.dense(), k, h, v0).reshape(got.shape)
    assert rel_err(got, ex) <= 1e-7
    ctx.close()


def test_csr_and_fp32(env, xi):
    torch, ei = env
    g = W.rgg_graph(n=4000, seed=12)
    op = O.CsrOperator(g.n, g.rowptr, g.col, g.val, -g.deg_w)
    v0 = W.random_vector(g.n, 8)
    h = 30.0 / (2 * g.deg_w.max())
    ref, ost = Nw.phi_apply(op, 2, h, v0, 1e-10, xi=xi, fixed_s=4)
    ctx = ei.Context()
    ctx.set_operator_csr(g.n, dev(torch, g.rowptr), dev(torch, g.col), dev(torch, g.val),
                         dev(torch, -g.deg_w))
    v = dev(torch, v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply(2, h, v, out, 1e-10, {"fixed_s": 4})
    assert rel_err(out.cpu().numpy(), ref) <= 1e-9 and st.degree_list() == list(ost.degrees)
    ctx.close()
    # FP32 stencil form, on FP32-representable inputs
    rng = np.random.default_rng(3)
    n, dx, bc = (40, 31), (1 / 41, 1 / 32), (1, 1, 0, 0)
    D, b = _fields2d(rng, n)
    D = D.astype(np.float32).astype(np.float64)
    b = tuple(x.astype(np.float32).astype(np.float64) for x in b)
    v0 = rng.standard_normal((31, 40)).astype(np.float32).astype(np.float64)
    opf = O.StencilOperator(n, dx, D, b, bc=bc)
    ref, _ = Nw.phi_apply(opf, 3, 4e-3, v0, 1e-12, xi=xi, fixed_s=2)
    ctx = stencil_context(torch, ei, n, dx, D, b, 0.0, bc, prec=1)
    v = dev(torch, v0, torch.float32)
    out = torch.empty_like(v)
    ctx.phi_apply(3, 4e-3, v, out, 1e-6, {"fixed_s": 2})
    assert rel_err(out.cpu().numpy().astype(np.float64), ref) <= 1e-5
    ctx.close()
