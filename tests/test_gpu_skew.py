"""phi_k(-i h H) v for a real symmetric H through the C ABI
(ei_phi_apply_imag: the complex products of Eq. (3) with K = C, Sec. II-C), on
the spin-bath Hamiltonian of Sec. III-D, against the oracle (oracle/skew.py)
and scipy's expm of the dense complex matrix.

Bars: FP64 1e-9 relative (2-norm over both parts) with identical s and
per-substep degrees; FP32 1e-5 against the oracle at tol 1e-12 (the FP32
form's own tol 1e-6; rounding of order 6e-8 per step over s(m+1) steps of a
unitary propagation); against expm 1e-8 (the method's tol 1e-10).  Errors as
include/ei.h states."""
import numpy as np
import pytest
import scipy.linalg

from oracle import leja as L
from oracle import operators as O
from oracle import skew as S
from paper_1309_4616_gb300 import workloads as W

from gpu_helpers import dev, require_gpu, stencil_context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return require_gpu()


@pytest.fixture(scope="module")
def xi():
    return L.leja_points(100)


def crel(a, b):
    a = np.asarray(a, dtype=complex).ravel()
    b = np.asarray(b, dtype=complex).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def spin_context(torch, ei, g, prec=0):
    dt = torch.float64 if prec == 0 else torch.float32
    ctx = ei.Context()
    ctx.set_operator_csr(g.n, dev(torch, g.rowptr), dev(torch, g.col), dev(torch, g.val, dt),
                         dev(torch, g.diag, dt), prec=prec)
    return ctx


def cdev(torch, v, dtype=None):
    return dev(torch, np.asarray(v, dtype=complex), dtype or torch.complex128)


@pytest.mark.parametrize("spins,h", [(8, 0.7), (10, 2.0), (12, 6.0)])
def test_propagator_against_oracle(env, xi, spins, h):
    torch, ei = env
    g = W.spin_bath(spins)
    op = O.CsrOperator(g.n, g.rowptr, g.col, g.val, g.diag)
    v0 = W.spin_state(g.n, 3)
    ref, s, degs = S.phi_apply_imag(op, 0, h, v0, 1e-10, xi=xi)
    ctx = spin_context(torch, ei, g)
    v = cdev(torch, v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply_imag(0, h, v, out, 1e-10)
    got = out.cpu().numpy()
    assert crel(got, ref) <= 1e-9
    assert st.s == s and st.degree_list() == list(degs)
    assert abs(np.linalg.norm(got) - 1.0) <= 1e-9  # e^{-ihH} is unitary
    if spins == 8:
        ex = scipy.linalg.expm(-1j * h * op.dense()) @ v0
        assert crel(got, ex) <= 1e-8
    ctx.close()


def test_substeps_and_fixed_s(env, xi):
    """A long time: the rule takes s > 1; a forced s = 2 s matches the oracle
    with the same forced s."""
    torch, ei = env
    g = W.spin_bath(9)
    op = O.CsrOperator(g.n, g.rowptr, g.col, g.val, g.diag)
    v0 = W.spin_state(g.n, 4)
    h = 25.0
    ref, s, degs = S.phi_apply_imag(op, 0, h, v0, 1e-10, xi=xi)
    assert s > 1
    ctx = spin_context(torch, ei, g)
    v = cdev(torch, v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply_imag(0, h, v, out, 1e-10)
    assert st.s == s and st.degree_list() == list(degs)
    assert crel(out.cpu().numpy(), ref) <= 1e-9
    ref2, _, degs2 = S.phi_apply_imag(op, 0, h, v0, 1e-10, xi=xi, fixed_s=2 * s)
    st = ctx.phi_apply_imag(0, h, v, v, 1e-10, {"fixed_s": 2 * s})  # in place
    assert st.s == 2 * s and st.degree_list() == list(degs2)
    assert crel(v.cpu().numpy(), ref2) <= 1e-9
    ctx.close()


@pytest.mark.parametrize("k", [1, 2, 4])
def test_phi_k(env, xi, k):
    torch, ei = env
    g = W.spin_bath(9)
    op = O.CsrOperator(g.n, g.rowptr, g.col, g.val, g.diag)
    v0 = W.spin_state(g.n, 5 + k)
    h = 0.8
    ref, s, degs = S.phi_apply_imag(op, k, h, v0, 1e-10, xi=xi)
    ctx = spin_context(torch, ei, g)
    v = cdev(torch, v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply_imag(k, h, v, out, 1e-10)
    assert st.s == s == 1 and st.degree_list() == list(degs)
    assert crel(out.cpu().numpy(), ref) <= 1e-9
    ctx.close()


def test_native_f64_and_fp32(env, xi):
    torch, ei = env
    g = W.spin_bath(11)
    op = O.CsrOperator(g.n, g.rowptr, g.col, g.val, g.diag)
    v0 = W.spin_state(g.n, 9)
    h = 3.0
    ref, s, degs = S.phi_apply_imag(op, 0, h, v0, 1e-10, xi=xi)
    ctx = spin_context(torch, ei, g)
    v = cdev(torch, v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply_imag(0, h, v, out, 1e-10, {"arith": ei.ARITH_NATIVE_F64})
    assert st.s == s and st.degree_list() == list(degs)
    assert crel(out.cpu().numpy(), ref) <= 1e-9
    ctx.close()
    # FP32: the couplings and the state rounded to FP32 on both sides
    g32 = W.spin_bath(11)
    g32.val = g32.val.astype(np.float32).astype(np.float64)
    g32.diag = g32.diag.astype(np.float32).astype(np.float64)
    v32 = v0.astype(np.complex64).astype(complex)
    op32 = O.CsrOperator(g32.n, g32.rowptr, g32.col, g32.val, g32.diag)
    ref32, _, _ = S.phi_apply_imag(op32, 0, h, v32, 1e-12, xi=xi)
    ctx = spin_context(torch, ei, g32, prec=1)
    v = cdev(torch, v32, torch.complex64)
    out = torch.empty_like(v)
    ctx.phi_apply_imag(0, h, v, out, 1e-6)
    assert crel(out.cpu().numpy().astype(complex), ref32) <= 1e-5
    ctx.close()


def test_sampled_large_grid_stride(env, xi):
    """18 spins (262144 rows, 33 entries a row): more rows than one pass of
    the resident grid, so rows are walked grid-stride; full comparison."""
    torch, ei = env
    g = W.spin_bath(18)
    op = O.CsrOperator(g.n, g.rowptr, g.col, g.val, g.diag)
    v0 = W.spin_state(g.n, 11)
    h = 0.4
    ref, s, degs = S.phi_apply_imag(op, 0, h, v0, 1e-10, xi=xi)
    ctx = spin_context(torch, ei, g)
    v = cdev(torch, v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply_imag(0, h, v, out, 1e-10)
    assert st.s == s and st.degree_list() == list(degs)
    assert crel(out.cpu().numpy(), ref) <= 1e-9
    ctx.close()


def test_degenerate_and_errors(env, xi):
    torch, ei = env
    g = W.spin_bath(8)
    ctx = spin_context(torch, ei, g)
    z = torch.zeros(g.n, dtype=torch.complex128, device="cuda")
    out = torch.full_like(z, 1.0)
    st = ctx.phi_apply_imag(0, 1.0, z, out, 1e-10)
    assert st.s == 1 and st.degree_list() == [0] and torch.count_nonzero(out).item() == 0
    v = cdev(torch, W.spin_state(g.n, 2))
    with pytest.raises(ei.EIError) as e:  # one substep only for k >= 1
        ctx.phi_apply_imag(1, 1.0, v, out, 1e-10, {"fixed_s": 2})
    assert e.value.status == ei.ERR_INVALID_ARG
    bad = v.clone()
    bad[5] = complex(float("nan"), 0.0)
    with pytest.raises(ei.EIError) as e:
        ctx.phi_apply_imag(0, 1.0, bad, out, 1e-10)
    assert e.value.status == ei.ERR_NONFINITE
    with pytest.raises(ValueError):  # a real tensor is refused by the binding
        ctx.phi_apply_imag(0, 1.0, v.real.contiguous(), out, 1e-10)
    ctx.close()
    # H = c I (no off-diagonal entries): the scalar phi_k(-i h c)
    n = 300
    ctx = ei.Context()
    ctx.set_operator_csr(n, torch.zeros(n + 1, dtype=torch.int64, device="cuda"),
                         torch.zeros(0, dtype=torch.int32, device="cuda"),
                         torch.zeros(0, dtype=torch.float64, device="cuda"),
                         torch.full((n,), 1.7, dtype=torch.float64, device="cuda"))
    v0 = W.spin_state(n, 6)
    v = cdev(torch, v0)
    out = torch.empty_like(v)
    for k in (0, 1, 3):
        ctx.phi_apply_imag(k, 2.5, v, out, 1e-10)
        op = O.CsrOperator(n, np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32),
                           np.zeros(0), np.full(n, 1.7))
        ref, _, _ = S.phi_apply_imag(op, k, 2.5, v0, 1e-10, xi=xi)
        assert crel(out.cpu().numpy(), ref) <= 1e-14
    ctx.close()
    # a stencil context has no complex path
    sc = stencil_context(torch, ei, (20, 20), (0.05, 0.05), 1.0, (0.0, 0.0), 0.0, (0, 0, 0, 0))
    w = torch.zeros(400, dtype=torch.complex128, device="cuda")
    with pytest.raises(ei.EIError) as e:
        sc.phi_apply_imag(0, 1.0, w, w, 1e-10)
    assert e.value.status == ei.ERR_STATE
    sc.close()


@pytest.mark.parametrize("lanes", [0, 1, 2, 4, 8, 16, 32])
def test_lanes_per_row_ragged(env, xi, lanes):
    """Every lanes-per-row variant of the complex CSR kernel on a graph with
    ragged rows (degrees from 0 up): H = W - diag(deg) of a random geometric
    graph, more rows than one pass of the grid."""
    torch, ei = env
    g = W.rgg_graph(n=70000, mean_degree=20.0, seed=17)
    op = O.CsrOperator(g.n, g.rowptr, g.col, g.val, -g.deg_w)
    v0 = W.spin_state(g.n, 12)
    h = 0.05
    ref, s, degs = S.phi_apply_imag(op, 0, h, v0, 1e-10, xi=xi)
    ctx = ei.Context()
    ctx.set_operator_csr(g.n, dev(torch, g.rowptr), dev(torch, g.col), dev(torch, g.val),
                         dev(torch, -g.deg_w))
    v = cdev(torch, v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply_imag(0, h, v, out, 1e-10, {"csr_lanes": lanes})
    assert st.s == s and st.degree_list() == list(degs)
    assert crel(out.cpu().numpy(), ref) <= 1e-9
    ctx.close()


def test_m_max_option_and_k1_substep_limit(env, xi):
    """A small m_max: the rule takes more substeps of lower degree, and the
    result, s and degrees match the oracle's with the same m_max.  For k >= 1
    a time step whose rule needs s > 1 is refused (one substep only), as the
    oracle refuses it."""
    torch, ei = env
    g = W.spin_bath(9)
    op = O.CsrOperator(g.n, g.rowptr, g.col, g.val, g.diag)
    v0 = W.spin_state(g.n, 4)
    ctx = spin_context(torch, ei, g)
    v = cdev(torch, v0)
    out = torch.empty_like(v)
    for m_max, h in ((12, 3.0), (20, 1.0)):
        ref, s, degs = S.phi_apply_imag(op, 0, h, v0, 1e-10, m_max=m_max, xi=xi)
        st = ctx.phi_apply_imag(0, h, v, out, 1e-10, {"m_max": m_max})
        assert st.s == s and st.degree_list() == list(degs)
        assert crel(out.cpu().numpy(), ref) <= 1e-9
    a, b = op.gershgorin()
    h = 12.0
    assert S.schedule_imag(1, h, 0.5 * (a + b), 0.25 * (b - a), 1e-10, xi)[0] > 1
    with pytest.raises(RuntimeError):
        S.phi_apply_imag(op, 1, h, v0, 1e-10, xi=xi)
    with pytest.raises(ei.EIError) as e:
        ctx.phi_apply_imag(1, h, v, out, 1e-10)
    assert e.value.status == ei.ERR_NOT_CONVERGED
    ctx.close()
