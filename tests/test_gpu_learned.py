"""The learned schedule through the C ABI against the oracle
(oracle/learned.py), in both modes (adaptive: options.learned = 1; fixed
count: 3): the same network, evaluated in FP32 on both sides, makes the
same proposal (s, m); an accepted proposal gives the oracle's result for it
within 1e-9 (same degrees), a rejected one the plain result within 1e-9.
Hand-built networks make the proposal known in advance; the features the
library reports match the oracle's definition."""
import math

import numpy as np
import pytest

from oracle import leja as L
from oracle import learned as Lr
from oracle import mlp as M
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


def net_from(q_accept, o0):
    """Output 0 = o0 everywhere; output 1 = 10 x3 - q_accept + 0.5 with
    x3 = q/10, so q is accepted from q_accept on (q_accept = -1: always,
    q_accept = 99: never).  o0 and the threshold are exact in FP32."""
    th = np.zeros(M.n_params())
    (W0, _), (W1, _), (W2, _), (W3, b3) = M.unpack(th)
    W0[0, 3] = 1.0
    W1[0, 0] = 1.0
    W2[0, 0] = 1.0
    W3[1, 0] = 10.0
    b3[:] = [o0, -q_accept + 0.5]
    return th.astype(np.float32)


def _model(ei, theta):
    net = ei.Mlp()
    net.set_params(theta)
    net.set_decision(0.0, 0.05, 2.0, 12)
    return net


def _field2d(n, seed):
    rng = np.random.default_rng(seed)
    nx, ny = n
    D = 0.3 + rng.uniform(0, 1, (ny, nx))
    b = [rng.uniform(-1, 1, (ny, nx)), rng.uniform(-1, 1, (ny, nx))]
    return D, b


@pytest.mark.parametrize("mode,q_accept,o0,h,expect", [
    # fixed count (options.learned = 3)
    (3, 1, 0.75, 6e-3, 1), (3, 0, 0.0625, 6e-3, 2), (3, 99, 0.5, 6e-3, 3),
    # adaptive (options.learned = 1): m only batches the launches; at h = 0.03
    # s = 1 reaches m_max (the plain rule needs s = 2) and the call falls back
    (1, 1, 0.75, 6e-3, 1), (1, 0, 0.0625, 6e-3, 1), (1, 0, 0.5, 0.03, 2), (1, 99, 0.5, 6e-3, 3)])
def test_learned_phi1_stencil(env, xi, mode, q_accept, o0, h, expect):
    torch, ei = env
    n, dx, bc = (45, 38), (1 / 46, 1 / 39), (0, 1, 1, 0)
    D, b = _field2d(n, 1)
    v0 = np.random.default_rng(2).standard_normal((n[1], n[0]))
    tol = 1e-10
    op = O.StencilOperator(n, dx, D, b, bc=bc)
    ratio, pe = Lr.stencil_stats(D, b, dx)
    theta = net_from(q_accept, o0)
    y, ls = Lr.phi1_learned(op, h, v0, tol, theta.astype(np.float64), Lr.Meta(), Lr.KIND_STENCIL,
                            2, ratio, pe, xi, fixed=(mode == 3))
    assert (1 if ls.accepted else 2 if ls.proposed else 3) == expect
    ctx = stencil_context(torch, ei, n, dx, D, b, 0.0, bc)
    net = _model(ei, theta)
    ctx.set_schedule_model(net)
    v = dev(torch, v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply(1, h, v, out, tol, {"learned": mode})
    got = out.cpu().numpy()
    assert rel_err(got, y / h) <= 1e-9
    assert st.learned == expect
    if expect != 3:
        assert (st.learned_s, st.learned_m) == (ls.s, ls.m)
        assert ls.s == 2 ** max(q_accept, 0)
    if st.learned == 1:
        assert st.s == ls.s and st.degree_list() == list(ls.degrees)
    else:  # the plain method's degrees
        assert st.s == ls.plain.s and st.degree_list() == list(ls.plain.degrees)
    ctx.close()


@pytest.mark.parametrize("mode", [1, 3])
def test_learned_rosenbrock_3d(env, xi, mode):
    torch, ei = env
    w = W.adr_3d(n=20, h=4e-3)
    op = O.StencilOperator(w.n, w.dx, w.D, w.b, bc=w.bc)
    ratio, pe = Lr.stencil_stats(w.D, w.b, w.dx)
    theta = net_from(0, 0.5)
    ref, ls = Lr.exp_step_learned(op, w.u0, w.h, w.tol, theta.astype(np.float64), Lr.Meta(),
                                  Lr.KIND_STENCIL, 3, ratio, pe, rosenbrock=True, xi=xi,
                                  fixed=(mode == 3))
    assert ls.accepted
    ctx = ei.Context()
    ctx.set_operator_stencil(w.n, w.dx, dev(torch, w.D), [dev(torch, x) for x in w.b], 0.0,
                             list(w.bc), ei.PREC_F64)
    net = _model(ei, theta)
    ctx.set_schedule_model(net)
    u = dev(torch, w.u0)
    st = ctx.step(ei.EXP_ROSENBROCK, w.h, u, ei.NONLIN_LOGISTIC, w.tol, {"learned": mode})
    assert st.learned == 1 and (st.s, st.learned_m) == (ls.s, ls.m)
    assert st.degree_list() == list(ls.degrees)
    assert rel_err(u.cpu().numpy() - w.u0, ref - w.u0) <= 1e-9
    ctx.close()


@pytest.mark.parametrize("mode", [1, 3])
def test_learned_csr(env, xi, mode):
    torch, ei = env
    g = W.rgg_graph(n=6000, seed=11)
    op = O.CsrOperator(g.n, g.rowptr, g.col, g.val, -g.deg_w)
    ratio, pe = Lr.csr_stats(-g.deg_w)
    h = 40.0 / (2.0 * g.deg_w.max())
    v0 = W.random_vector(g.n, 4)
    theta = net_from(0, 0.5)
    y, ls = Lr.phi1_learned(op, h, v0, 1e-10, theta.astype(np.float64), Lr.Meta(), Lr.KIND_CSR,
                            0, ratio, pe, xi, fixed=(mode == 3))
    ctx = ei.Context()
    ctx.set_operator_csr(g.n, dev(torch, g.rowptr), dev(torch, g.col), dev(torch, g.val),
                         dev(torch, -g.deg_w))
    net = _model(ei, theta)
    ctx.set_schedule_model(net)
    v = dev(torch, v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply(1, h, v, out, 1e-10, {"learned": mode})
    assert st.learned == (1 if ls.accepted else 2)
    assert rel_err(out.cpu().numpy(), y / h) <= 1e-9
    ctx.close()


@pytest.mark.parametrize("mode", [1, 3])
def test_learned_fp32_form(env, xi, mode):
    """The FP32 form under an accepted proposal, against the oracle on the
    FP32-rounded inputs (1e-5)."""
    torch, ei = env
    n, dx, bc = (40, 36), (1 / 41, 1 / 37), (1, 1, 0, 0)
    D, b = _field2d(n, 3)
    D32 = D.astype(np.float32).astype(np.float64)
    b32 = [x.astype(np.float32).astype(np.float64) for x in b]
    v0 = np.random.default_rng(5).standard_normal((n[1], n[0])).astype(np.float32)
    h, tol = 5e-3, 1e-6
    op = O.StencilOperator(n, dx, D32, b32, bc=bc)
    ratio, pe = Lr.stencil_stats(D32, b32, dx)
    theta = net_from(0, 0.5)
    y, ls = Lr.phi1_learned(op, h, v0.astype(np.float64), tol, theta.astype(np.float64),
                            Lr.Meta(), Lr.KIND_STENCIL, 2, ratio, pe, xi, fixed=(mode == 3))
    assert ls.accepted
    ctx = stencil_context(torch, ei, n, dx, D, b, 0.0, bc, prec=1)
    net = _model(ei, theta)
    ctx.set_schedule_model(net)
    v = dev(torch, v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply(1, h, v, out, tol, {"learned": mode})
    assert st.learned == 1 and (st.s, st.learned_m) == (ls.s, ls.m)
    assert rel_err(out.cpu().numpy(), y / h) <= 1e-5
    ctx.close()


@pytest.mark.parametrize("kind", ["stencil", "csr"])
def test_reported_features_match_oracle(env, kind):
    torch, ei = env
    if kind == "stencil":
        n, dx, bc = (33, 29), (1 / 34, 1 / 30), (0, 0, 1, 1)
        D, b = _field2d(n, 7)
        ctx = stencil_context(torch, ei, n, dx, D, b, 0.0, bc)
        ratio, pe = Lr.stencil_stats(D, b, dx)
        npts, dim, k = n[0] * n[1], 2, Lr.KIND_STENCIL
    else:
        g = W.rgg_graph(n=3000, seed=2)
        ctx = ei.Context()
        ctx.set_operator_csr(g.n, dev(torch, g.rowptr), dev(torch, g.col), dev(torch, g.val),
                             dev(torch, -g.deg_w))
        ratio, pe = Lr.csr_stats(-g.deg_w)
        npts, dim, k = g.n, 0, Lr.KIND_CSR
    v0 = 0.01 * np.random.default_rng(3).standard_normal(npts)
    v = dev(torch, v0)
    out = torch.empty_like(v)
    alpha, beta = ctx.estimate_spectrum()
    h, tol = 50.0 / max(abs(alpha), abs(beta)), 1e-8
    st = ctx.phi_apply(1, h, v, out, tol, {"learned": 2, "fixed_s": 4})
    assert st.learned == 4 and st.s == 4
    ref = Lr.features(2, h, alpha, beta, tol, 1, k, dim, npts, ratio, pe,
                      float(np.linalg.norm(v0)))
    np.testing.assert_allclose(st.feature_list(), ref, rtol=1e-12, atol=1e-14)
    ctx.close()


def test_no_restart_reports_not_converged(env, xi):
    torch, ei = env
    n, dx = (40, 40), (1 / 41, 1 / 41)
    D, b = _field2d(n, 9)
    v0 = np.random.default_rng(1).standard_normal((40, 40))
    h, tol = 0.05, 1e-10
    op = O.StencilOperator(n, dx, D, b, bc=(0, 0, 0, 0))
    _, degs, conv = Nw.h_phi1_at(op, h, v0, tol, 1, xi=xi)
    assert not conv
    ctx = stencil_context(torch, ei, n, dx, D, b, 0.0, (0, 0, 0, 0))
    v = dev(torch, v0)
    out = torch.zeros_like(v)
    with pytest.raises(ei.EIError) as e:
        ctx.phi_apply(1, h, v, out, tol, {"fixed_s": 1, "no_restart": 1})
    assert e.value.status == ei.ERR_NOT_CONVERGED
    assert float(out.abs().max()) == 0.0
    ctx.close()
