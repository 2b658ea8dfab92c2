"""The combustion nonlinearity of the oracle (Sec. III-C) pinned to closed
forms: values at u = 1 and 2, the derivative against a complex-step
derivative of g (exact to rounding, independent of the hand-written g'),
the maximum of g at the root of g', the cut against IEEE underflow, and the
two exponential steps on A = 0, where each reduces to a scalar formula per
point."""
import math

import numpy as np
import pytest

from oracle import leja as L
from oracle import newton as Nw
from oracle import operators as O


def test_values():
    g, dg = Nw.combustion(np.array([1.0, 2.0, 1.5]))
    assert g[0] == 0.25 and g[1] == 0.0 and dg[0] == 0.25 * 19.0
    assert g[2] == pytest.approx(0.125 * math.exp(20.0 * (1 - 1 / 1.5)), rel=1e-15)


def test_derivative_complex_step():
    u = np.array([0.05, 0.3, 0.9, 1.0, 1.3, 1.8, 2.0, 2.7])
    hstep = 1e-30

    def g_complex(z):  # g written again for complex arguments, no cut
        return 0.25 * (2.0 - z) * np.exp(20.0 * (1.0 - 1.0 / z))

    ref = np.imag(g_complex(u + 1j * hstep)) / hstep
    _, dg = Nw.combustion(u)
    np.testing.assert_allclose(dg, ref, rtol=1e-13, atol=1e-300)


def test_maximum_at_root_of_derivative():
    # g'(u) = 0  <=>  u^2 + 20 u - 40 = 0  ->  u* = sqrt(140) - 10
    us = math.sqrt(140.0) - 10.0
    g, dg = Nw.combustion(np.array([us]))
    assert abs(dg[0]) < 1e-14 * 20.0 * g[0]  # the bracket's rounding, scaled
    grid = np.linspace(1.0, 2.0, 10001)
    gg, _ = Nw.combustion(grid)
    assert g[0] >= gg.max() - 1e-15 and abs(grid[np.argmax(gg)] - us) < 2e-4


def test_cut_matches_underflow():
    u = np.array([-1.0, 0.0, 0.01, Nw.COMBUSTION_CUT, 0.026, 0.04])
    g, dg = Nw.combustion(u)
    assert (g[:4] == 0).all() and (dg[:4] == 0).all()
    # just above the cut the FP64 exponential already underflows to 0 ...
    assert math.exp(20.0 * (1.0 - 1.0 / 0.026)) == 0.0 and g[4] == 0.0
    # ... while further up it is a (tiny) positive number
    assert 0.0 < g[5] < 1e-200 and dg[5] > 0.0


def test_steps_on_zero_operator_reduce_to_scalar_formulas():
    """A = 0 (a CSR operator with no entries): exponential Euler gives
    u + h g(u); Rosenbrock-Euler gives u + h phi_1(h g'(u)) g(u) pointwise,
    with phi_1(z) = (e^z - 1)/z."""
    n = 7
    op = O.CsrOperator(n, np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32),
                       np.zeros(0))
    u0 = np.array([0.02, 0.5, 1.0, 1.2, 1.5, 1.83, 2.0])
    h = 1e-3  # h g'(u) of order 1 at every point
    g, dg = Nw.combustion(u0)
    xi = L.leja_points(100)
    ue, _ = Nw.exp_euler_step(op, u0, h, 1e-12, nonlin=Nw.NONLIN_COMBUSTION, xi=xi)
    np.testing.assert_allclose(ue, u0 + h * g, rtol=1e-14, atol=0)
    ur, st = Nw.exp_rosenbrock_step(op, u0, h, 1e-12, nonlin=Nw.NONLIN_COMBUSTION, xi=xi)
    z = h * dg
    phi1 = np.where(z == 0.0, 1.0, np.expm1(z) / np.where(z == 0.0, 1.0, z))
    ref = u0 + h * phi1 * g
    # the stop test is relative to the whole increment's norm
    assert np.linalg.norm(ur - ref) <= 1e-11 * np.linalg.norm(ref - u0)
    assert st.alpha == dg.min() and st.beta == dg.max()
