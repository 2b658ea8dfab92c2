"""Pins for the oracle's Leja points, scalar phi_k and divided differences.

Each check is tied to mathematics, not to the oracle's own code: closed forms,
brute force on tiny inputs, a library routine (scipy expm via Opitz's
theorem) and bounds from the mean-value theorem for divided differences.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import leja as L


@pytest.fixture(scope="module")
def xi():
    return L.leja_points(L.M_MAX)


def test_leja_first_points_closed_form(xi):
    # xi_0 = 2 (convention); xi_1 = -2; xi_2 = 0; xi_3 = +2/sqrt(3) (tie to the larger)
    assert xi[0] == 2.0
    assert xi[1] == -2.0
    assert abs(xi[2]) <= 1e-15
    assert abs(xi[3] - 2.0 / math.sqrt(3.0)) <= 1e-15
    assert len(set(np.round(xi, 14))) == len(xi)          # distinct
    assert np.all(np.abs(xi) <= 2.0)


def test_leja_brute_force_grid(xi):
    # brute force: argmax of prod|x - xi_i| over a fine grid agrees with the refined point
    grid = np.linspace(-2.0, 2.0, 400001)
    spacing = grid[1] - grid[0]
    logp = np.zeros_like(grid)
    for j in range(1, 25):
        with np.errstate(divide="ignore"):
            logp = logp + np.log(np.abs(grid - xi[j - 1]))
        if j == 3:
            continue   # exact symmetric tie, pinned in closed form above
        k = int(np.argmax(logp))
        assert abs(grid[k] - xi[j]) <= 2 * spacing, (j, grid[k], xi[j])


def test_leja_capacity_one(xi):
    # [-2, 2] has logarithmic capacity 1: (prod_{i<j}|xi_j - xi_i|)^(1/j) -> 1
    vals = []
    for j in range(60, 101):
        vals.append(math.exp(sum(math.log(abs(xi[j] - xi[i])) for i in range(j)) / j))
    assert 0.9 < min(vals) and max(vals) < 1.2


@pytest.mark.parametrize("z", [-300.0, -37.5, -3.0, -1.0, -0.3, -1e-6, 0.0, 1e-9, 0.7, 2.5])
def test_phi_scalar_closed_forms(z):
    assert L.phi_scalar(0, z) == pytest.approx(math.exp(z), rel=1e-15)
    e1 = 1.0 if z == 0.0 else math.expm1(z) / z
    assert L.phi_scalar(1, z) == pytest.approx(e1, rel=1e-14)
    if abs(z) > 0.5:
        e2 = (math.exp(z) - 1.0 - z) / (z * z)
        assert L.phi_scalar(2, z) == pytest.approx(e2, rel=1e-12)
    else:
        e2 = sum(z ** i / math.factorial(i + 2) for i in range(30))
        assert L.phi_scalar(2, z) == pytest.approx(e2, rel=1e-14)


def test_dd_two_points_exp(xi):
    # k = 0 on two points: f[x0, x1] = (e^{a} - e^{b}) / (x0 - x1)
    tau, c, gamma = 0.37, -3.1, 1.3
    d = L.divided_differences(0, tau, c, gamma, xi[:2])
    za, zb = tau * c + tau * gamma * xi[0], tau * c + tau * gamma * xi[1]
    assert d[0] == pytest.approx(math.exp(za), rel=1e-15)
    assert d[1] == pytest.approx((math.exp(za) - math.exp(zb)) / (xi[0] - xi[1]), rel=1e-13)


def test_dd_small_gamma_limit(xi):
    # gamma -> 0: d_j -> (tau gamma)^j e^{tau c} / j!   (k = 0)
    tau, c, gamma = 1.0, -0.8, 1e-7
    d = L.divided_differences(0, tau, c, gamma, xi[:8])
    for j in range(8):
        ref = (tau * gamma) ** j * math.exp(tau * c) / math.factorial(j)
        assert d[j] == pytest.approx(ref, rel=1e-5)


@pytest.mark.parametrize("k", [0, 1, 2])
@pytest.mark.parametrize("tg", [0.05, 1.0, 6.0])
def test_dd_opitz_scipy_expm(xi, k, tg):
    # Opitz: f(Z) e_1 holds the divided differences, Z lower bidiagonal with
    # diagonal xi and unit subdiagonal; f(Z) via scipy expm of an augmented matrix.
    m = 30
    tau, c, gamma = 1.0, -2.0 * tg, tg        # beta = 0, alpha = -4 tau gamma
    L_ = np.diag(xi[: m + 1]) + np.diag(np.ones(m), -1)
    Z = tau * c * np.eye(m + 1) + tau * gamma * L_
    n = m + 1
    M = np.zeros((n + k, n + k)) if k > 0 else None
    if k == 0:
        col = scipy.linalg.expm(Z)[:, 0]
    else:
        M[:n, :n] = Z
        M[0, n] = 1.0
        for i in range(k - 1):
            M[n + i, n + i + 1] = 1.0
        col = scipy.linalg.expm(M)[:n, n + k - 1]
    d = L.divided_differences(k, tau, c, gamma, xi[: m + 1])
    big = np.abs(d) > 1e-10 * np.abs(d).max()
    assert np.allclose(d[big], col[big], rtol=1e-9, atol=0)
    assert np.allclose(d, col, rtol=0, atol=1e-15 * np.abs(d).max())


@pytest.mark.parametrize("tg", [0.3, 4.0, 25.0])
def test_dd_mean_value_bounds(xi, tg):
    # phi_1^{(j)}(z) = int_0^1 th^j e^{th z} dth lies in (0, 1/(j+1)] for z <= 0,
    # so with beta = 0:  0 < d_j = (tau gamma)^j phi_1^{(j)}(eta)/j! <= (tau gamma)^j/(j+1)!
    d = L.divided_differences(1, 1.0, -2.0 * tg, tg, xi[:60])
    for j in range(60):
        ub = math.exp(j * math.log(tg) - math.lgamma(j + 2))
        assert 0.0 < d[j] <= ub * (1 + 1e-12)


def test_newton_interpolates_nodes(xi):
    # the Newton polynomial through the divided differences matches f at its nodes
    tau, c, gamma, m = 0.5, -20.0, 10.0, 40
    d = L.divided_differences(1, tau, c, gamma, xi[: m + 1])
    p = L.newton_eval(d, xi, xi[: m + 1])[m]
    f = np.array([L.phi_scalar(1, tau * c + tau * gamma * x) for x in xi[: m + 1]])
    assert np.allclose(p, f, rtol=1e-12, atol=1e-14)


def test_schedule_monotone_and_ranges(xi):
    # C1 operator (alpha=-3380, beta=0), h = 1e-3, tol 1e-10: one substep
    s, m, _ = L.plain_schedule(1, 1e-3, -1690.0, 845.0, 1e-10, xi)
    assert s == 1 and 5 <= m <= 30
    # s never decreases as h grows
    prev = 1
    for h in [1e-4, 1e-3, 1e-2, 1e-1]:
        s, m, _ = L.plain_schedule(1, h, -2.0e5, 1.0e5, 1e-10, xi)
        assert s >= prev and m <= L.M_MAX
        prev = s
    assert prev > 1


def _golden(name):
    import os
    vals = {}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_schedule_paper_range(xi):
    # Sec. III-D, Table 4 (tests/golden/paper_table4_step.txt): one step of the
    # 256^3 Dirichlet problem with tol = 1e-4, h = 1e-4 used 40 matrix-vector
    # products.  The a-priori degree for that interval must be of that order:
    # within a factor of 2.5 either way (a range check, not parity: the paper
    # does not give its schedule).
    g = _golden("paper_table4_step.txt")
    dx = 1.0 / (g["grid_points_per_axis"] + 1)
    rho = 12.0 / dx ** 2
    s, m, _ = L.plain_schedule(1, g["h"], -rho / 2, rho / 4, g["tol"], xi)
    mv = g["matvecs_per_step"]
    assert s == 1 and mv / 2.5 <= m <= mv * 2.5


def _bary_errors(xi, f_of, m_top):
    """max over the 2001-point grid G of |f - p_m| for m = 0..m_top, where p_m is
    the degree-m interpolant of f at xi_0..xi_m evaluated in the barycentric
    (second) form of Lagrange interpolation: no divided differences involved.
    Returns the errors and max_G |f|."""
    g = np.linspace(-2.0, 2.0, 2001)
    fg = f_of(g)
    errs = np.empty(m_top + 1)
    for m in range(m_top + 1):
        nodes = xi[: m + 1]
        fn = f_of(nodes)
        diff = nodes[:, None] - nodes[None, :]
        np.fill_diagonal(diff, 1.0)
        w = 1.0 / np.prod(diff, axis=1)
        dx = g[:, None] - nodes[None, :]
        hit = dx == 0.0
        dx[hit] = 1.0
        t = w[None, :] / dx
        p = (t @ fn) / t.sum(axis=1)
        rows, cols = np.nonzero(hit)
        p[rows] = fn[cols]
        errs[m] = np.max(np.abs(p - fg))
    return errs, float(np.max(np.abs(fg)))


def _phi_np(k):
    # phi_0 = exp, phi_1 = expm1(z)/z with phi_1(0) = 1 (numpy, independent of the oracle)
    if k == 0:
        return np.exp
    def phi1(z):
        z = np.asarray(z, dtype=np.float64)
        out = np.ones_like(z)
        nz = z != 0.0
        out[nz] = np.expm1(z[nz]) / z[nz]
        return out
    return phi1


@pytest.mark.parametrize("k,h,c,gamma,tol", [
    (1, 1e-3, -1690.0, 845.0, 1e-10),      # the 64^2 advection-diffusion interval
    (1, 2e-3, -5.0e3, 2.5e3, 1e-8),        # h gamma = 5: one substep, a middle degree
    (1, 1.0, -60.0, 30.0, 1e-10),          # h gamma = 30: close to the single-substep limit
    (1, 1.0, -400.0, 200.0, 1e-10),        # h gamma = 200: several substeps
    (0, 1.0, -150.0, 75.0, 1e-6),          # exp, h gamma = 75
    (1, 1.0, -35.0, 40.0, 1e-8),           # interval reaching into Re z > 0
    (1, 1.0, -2000.0, 1000.0, 1e-10),      # h gamma = 1000: s = 8, degree near m_max
    (0, 1.0, -3000.0, 1500.0, 1e-6),       # exp, h gamma = 1500: s = 16
])
def test_schedule_meets_its_definition(xi, k, h, c, gamma, tol):
    # The a-priori rule by its definition, checked with interpolants built
    # without divided differences: at the returned (s, m) the degree-m
    # interpolant at the Leja points meets max_G|f - p_m| <= tol max_G|f| for
    # f(x) = phi_k(tau c + tau gamma x), tau = h/s; degree m-1 does not; and at
    # s/2 no degree <= 100 does.  Thresholds carry a 1e-6 relative slack for the
    # two evaluation orders' rounding.
    s, m, _ = L.plain_schedule(k, h, c, gamma, tol, xi)
    phi = _phi_np(k)
    tau = h / s
    errs, fmax = _bary_errors(xi, lambda x: phi(tau * c + tau * gamma * x), m)
    assert errs[m] <= tol * fmax * (1 + 1e-6)
    if m > 0:
        assert errs[m - 1] > tol * fmax * (1 - 1e-6)
    if s > 1:
        tau2 = 2.0 * tau
        errs2, fmax2 = _bary_errors(xi, lambda x: phi(tau2 * c + tau2 * gamma * x), L.M_MAX)
        assert errs2.min() > tol * fmax2 * (1 - 1e-6)
