"""Pins of the learned-schedule oracle (oracle/learned.py and the fixed-count
Newton form in oracle/newton.py): the fixed-count phi_1 against the dense
matrix exponential, the vector recursion against the scalar Newton
polynomial on a diagonal operator, the no-restart driver against the plain
one, the decision rule on constructed outputs, and closed-form features."""
import math

import numpy as np
import pytest

from oracle import dense as Dn
from oracle import leja as L
from oracle import learned as Lr
from oracle import mlp as M
from oracle import newton as Nw
from oracle import operators as O


@pytest.fixture(scope="module")
def xi():
    return L.leja_points(100)


def _op2d(n=12, bc=(1, 0, 1, 1)):
    rng = np.random.default_rng(5)
    shape = (n, n)
    D = 0.5 + rng.uniform(0, 1, shape)
    b = [rng.uniform(-1, 1, shape), rng.uniform(-1, 1, shape)]
    dx = (1.0 / n, 1.0 / n)
    return O.StencilOperator((n, n), dx, D, b, bc=bc), D, b, dx


def test_fixed_count_phi1_matches_dense(xi):
    """Enough steps: h phi_1(hA) v to the tolerance, and the final check
    passes; too few: the check fails."""
    op, *_ = _op2d()
    v = np.random.default_rng(1).standard_normal(op.shape)
    h = 2e-3
    ref = h * Dn.phi_dense(op.dense(), 1, h, v.ravel()).reshape(op.shape)
    alpha, beta = op.gershgorin()
    s, m_sched, _ = L.plain_schedule(1, h, 0.5 * (alpha + beta), 0.25 * (beta - alpha), 1e-12, xi)
    st = Nw.Stats()
    y, ok = Nw.h_phi1_fixed(op, h, v, 1e-12, s, m_sched + 4, st, xi)
    assert ok
    assert np.linalg.norm(y - ref) <= 1e-10 * np.linalg.norm(ref)
    assert st.matvecs == s * (m_sched + 4) + (s - 1)
    y2, ok2 = Nw.h_phi1_fixed(op, h, v, 1e-12, s, 3, Nw.Stats(), xi)
    assert not ok2


def test_fixed_count_on_diagonal_operator_is_the_scalar_polynomial(xi):
    """A = diag(lam): component i of the fixed-count sum is the degree-m Newton
    interpolant p_m(x_i) at x_i = (lam_i - c)/gamma, evaluated as a scalar
    polynomial; and it is within the interpolation error of phi_1(tau lam_i)."""
    lam = -np.linspace(0.0, 400.0, 33)
    n = lam.size
    op = O.CsrOperator(n, np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int64),
                       np.zeros(0), lam)
    alpha, beta = op.gershgorin()
    c, gamma = 0.5 * (alpha + beta), 0.25 * (beta - alpha)
    tau, m = 0.01, 30
    d = L.divided_differences(1, tau, c, gamma, xi[: m + 1])
    r = np.ones(n)
    p, ok = Nw.newton_phi_fixed(op, r, d, xi, c, gamma, 1e-10, m, Nw.Stats())
    x = (lam - c) / gamma
    np.testing.assert_allclose(p, L.newton_eval(d, xi[: m + 1], x)[m], rtol=1e-12, atol=1e-14)
    exact = np.array([L.phi_scalar(1, tau * t) for t in lam])
    assert np.abs(p - exact).max() <= 1e-9


def test_no_restart_driver_agrees_with_plain(xi):
    """At the plain rule's s the no-restart driver converges with the same
    degrees and the same result; at s/2 of a case that needs s it reports
    no convergence instead of restarting."""
    op, *_ = _op2d(16, (0, 0, 1, 0))
    v = np.random.default_rng(2).standard_normal(op.shape)
    h, tol = 0.2, 1e-10
    st = Nw.Stats()
    ref = Nw.h_phi1_substeps(op, h, v, tol, st, xi=xi)
    assert st.s >= 2 and st.restarts == 0
    y, degs, conv = Nw.h_phi1_at(op, h, v, tol, st.s, xi=xi)
    assert conv and degs == list(st.degrees)
    np.testing.assert_array_equal(y, ref)
    _, degs2, conv2 = Nw.h_phi1_at(op, h, v, tol, st.s // 2, m_max=max(st.degrees), xi=xi)
    assert not conv2


def test_decision_rule_truth_table():
    meta = Lr.Meta(z_min=0.0, rho_m=0.05, delta_m=2.0, m_max=100, q_max=3)
    # q=0 rejected by the classifier, q=1 by the degree; q=2 (m 44, cost
    # 4*45-1 = 179) and q=3 (m 13, cost 8*14-1 = 111) accepted: q=3 is cheaper
    outs = [(0.2, -1.0), (0.97, 3.0), (0.40, 0.5), (0.1, 5.0)]
    assert Lr.decide(outs, meta) == (8, 13)
    # with q=3 at m 30 (cost 247) q=2 is the cheaper
    outs[3] = (0.27, 5.0)
    assert Lr.decide(outs, meta) == (4, 44)
    # equal cost: the smaller q (q=0: m 19, cost 19; q=1: m 9, cost 19)
    tie = [((19 - 2) / 105, 1.0), ((9 - 2) / 105, 1.0)]
    assert Lr.decide(tie, Lr.Meta(rho_m=0.05, delta_m=2.0, q_max=1)) == (1, 19)
    assert Lr.decide([(0.1, -0.1)] * 4, meta) is None
    # the degree is clamped to [1, m_max]
    assert Lr.decide([(-0.5, 1.0)], meta) == (1, 1)
    # need = 100*o*1.05 + 2 <= 100 exactly at o = 98/105
    assert Lr.decide([(98 / 105 - 1e-12, 1.0)], meta) == (1, 100)
    assert Lr.decide([(98 / 105 + 1e-9, 1.0)], meta) is None


def test_features_closed_form():
    """The 64^2 advection-diffusion problem: Gershgorin interval [-3380, 0]
    (c = -1690, gamma = 845), constant D = 0.1 and b = (-1, -0.5) give the
    Peclet number |b_x| dx / (2 D) = 5/65 and coefficient ratio 1."""
    n = 64
    dx = 1.0 / 65
    ratio, pe = Lr.stencil_stats(np.full((n, n), 0.1), [np.full((n, n), -1.0),
                                                        np.full((n, n), -0.5)], (dx, dx))
    assert ratio == pytest.approx(1.0, rel=1e-15) and pe == pytest.approx(1.0 * dx / 0.2, rel=1e-15)
    f = Lr.features(2, 1e-3, -3380.0, 0.0, 1e-10, 1, Lr.KIND_STENCIL, 2, n * n, ratio, pe,
                    math.sqrt(n * n) * 0.5)
    assert f[0] == pytest.approx(math.log10(1e-3 / 4 * 845.0), rel=1e-15)
    assert f[1] == -0.5 and f[2] == -1.0 and f[3] == 0.2
    assert f[4] == pytest.approx(math.log10(3.38) / 3, rel=1e-15)
    assert f[6] == 0.0 and f[7] == pytest.approx(2 / 3)
    assert f[10] == pytest.approx(math.log10(0.5) / 10, rel=1e-15)
    assert f[11] == pytest.approx(math.log10(4096) / 8, rel=1e-15)
    r2, pe2 = Lr.csr_stats(np.array([-2.0, -4.0, -6.0]))
    assert r2 == pytest.approx(4.0 / 6.0) and pe2 == 0.0


def _constant_network(o0, o1, sizes=M.SIZES):
    """A network whose output is (o0, o1) for every input: zero weights, the
    output layer's biases only."""
    theta = np.zeros(M.n_params(sizes))
    theta[-2:] = [o0, o1]
    return theta


def test_learned_phi1_fixed_count_accepts_and_falls_back(xi):
    op, D, b, dx = _op2d()
    ratio, pe = Lr.stencil_stats(D, b, dx)
    v = np.random.default_rng(3).standard_normal(op.shape)
    h, tol = 2e-3, 1e-10
    ref = h * Dn.phi_dense(op.dense(), 1, h, v.ravel()).reshape(op.shape)
    meta = Lr.Meta(rho_m=0.0, delta_m=0.0)
    # outputs exactly representable in FP32, so the degree is exact
    # proposal (s = 1, m = 50): enough; accepted without the plain method
    y, ls = Lr.phi1_learned(op, h, v, tol, _constant_network(0.5, 1.0), meta,
                            Lr.KIND_STENCIL, 2, ratio, pe, xi, fixed=True)
    assert ls.proposed and ls.accepted and (ls.s, ls.m) == (1, 50) and ls.plain is None
    assert np.linalg.norm(y - ref) <= 1e-9 * np.linalg.norm(ref)
    # proposal (s = 1, m = 4): its check fails; the plain result is returned
    y2, ls2 = Lr.phi1_learned(op, h, v, tol, _constant_network(1.0 / 32, 1.0), meta,
                              Lr.KIND_STENCIL, 2, ratio, pe, xi, fixed=True)
    assert ls2.proposed and not ls2.accepted and ls2.plain is not None
    st = Nw.Stats()
    np.testing.assert_array_equal(y2, Nw.h_phi1_substeps(op, h, v, tol, st, xi=xi))
    # no q accepted: plain
    _, ls3 = Lr.phi1_learned(op, h, v, tol, _constant_network(0.5, -1.0), meta,
                             Lr.KIND_STENCIL, 2, ratio, pe, xi)
    assert not ls3.proposed and ls3.plain is not None


def test_learned_phi1_adaptive(xi):
    """Adaptive mode: the proposal's s with the plain method's per-substep
    stop, so an accepted call equals the plain method at that s exactly; a
    substep that reaches m_max sends the call to the plain method."""
    op, D, b, dx = _op2d()
    ratio, pe = Lr.stencil_stats(D, b, dx)
    v = np.random.default_rng(3).standard_normal(op.shape)
    meta = Lr.Meta(rho_m=0.0, delta_m=0.0)
    tol = 1e-10
    # h = 0.1: the plain rule takes s = 1 (degree 58); the proposal s = 1, m = 4
    # is accepted and its m only batches the launches
    st = Nw.Stats()
    ref = Nw.h_phi1_substeps(op, 0.1, v, tol, st, xi=xi)
    assert st.s == 1
    y, ls = Lr.phi1_learned(op, 0.1, v, tol, _constant_network(1.0 / 32, 1.0), meta,
                            Lr.KIND_STENCIL, 2, ratio, pe, xi)
    assert ls.accepted and ls.s == 1 and ls.degrees == list(st.degrees)
    np.testing.assert_array_equal(y, ref)
    # h = 0.4: s = 1 reaches m_max (the plain rule needs s = 2): fallback
    st = Nw.Stats()
    ref = Nw.h_phi1_substeps(op, 0.4, v, tol, st, xi=xi)
    assert st.s == 2
    y, ls = Lr.phi1_learned(op, 0.4, v, tol, _constant_network(0.5, 1.0), meta,
                            Lr.KIND_STENCIL, 2, ratio, pe, xi)
    assert ls.proposed and not ls.accepted and ls.degrees == [100]
    np.testing.assert_array_equal(y, ref)
