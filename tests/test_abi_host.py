"""The C ABI library on the CPU: it loads, exports every symbol include/ei.h
declares, and its host-side pieces (Leja points, divided differences, the
a-priori schedule) agree with the oracle.  No device compute is called."""
import os
import re

import numpy as np
import pytest

from oracle import leja as L
from oracle import skew as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ei():
    from paper_1309_4616_gb300 import build
    build.build()
    from paper_1309_4616_gb300 import ei as mod
    return mod


def test_header_symbols_exported(ei):
    hdr = open(os.path.join(ROOT, "include", "ei.h")).read()
    declared = set(re.findall(r"\b(ei_[a-z_0-9]+)\s*\(", hdr)) - {"ei_ctx"}
    assert declared == set(ei.EXPORTS)
    L_ = ei.lib()
    for name in declared:
        assert hasattr(L_, name), name


def test_status_strings(ei):
    assert ei.status_string(0) == "ok"
    assert "not converged" in ei.status_string(3)


def test_leja_points_match_oracle(ei):
    xi = ei.leja_points(100)
    xo = L.leja_points(100)
    assert np.abs(xi - xo).max() <= 1e-14


@pytest.mark.parametrize("k,tau,c,gamma", [
    (1, 1e-3, -1690.0, 845.0),          # the 64^2 advection-diffusion interval
    (1, 1e-4, -5.9e5, 2.95e5),           # the 256^3 interval, h = 1e-4
    (0, 0.37, -3.1, 1.3),
    (2, 0.5, -20.0, 10.0),
    (1, 1.0, -60.0, 30.0),
    (1, 1e-2, -2.0e4, 1.0e4),
])
def test_divided_differences_match_oracle(ei, k, tau, c, gamma):
    xi = L.leja_points(100)
    d = ei.divided_differences(k, tau, c, gamma, 100)
    do = L.divided_differences(k, tau, c, gamma, xi)
    big = np.abs(do) > 1e-300
    rel = np.abs(d[big] - do[big]) / np.abs(do[big])
    assert rel.max() <= 1e-13


@pytest.mark.parametrize("k,h,c,gamma,tol", [
    (1, 1e-3, -1690.0, 845.0, 1e-10),
    (1, 1e-4, -5.9e5, 2.95e5, 1e-10),
    (1, 5e-5, -2.4e6, 1.2e6, 1e-6),
    (1, 1e-2, -4 * 513 ** 2, 2 * 513 ** 2, 1e-10),
    (0, 0.5, -30.0, 15.0, 1e-12),
])
def test_schedule_matches_oracle(ei, k, h, c, gamma, tol):
    xi = L.leja_points(100)
    assert ei.schedule(k, h, c, gamma, tol) == L.plain_schedule(k, h, c, gamma, tol, xi)[:2]


def test_invalid_arguments(ei):
    with pytest.raises(ei.EIError) as e:
        ei.divided_differences(1, -1.0, 0.0, 1.0)
    assert e.value.status == ei.ERR_INVALID_ARG
    with pytest.raises(ei.EIError):
        ei.leja_points(101)


@pytest.mark.parametrize("k,tau,c,gamma", [
    (0, 1.0, 0.0, 0.5),
    (0, 2.0, 3.0, 4.0),
    (0, 0.3, -50.0, 20.0),
    (0, 0.35, 0.4, 22.0),                # a substep of the 21-spin bath interval
    (1, 5.0, 1.0, 2.0),
    (3, 0.3, -50.0, 20.0),
])
def test_divided_differences_imag_match_oracle(ei, k, tau, c, gamma):
    """The complex Opitz exponential: entries are bounded by about 1, and the
    library's double-precision scaling and squaring holds them to ~1e-14 in
    absolute terms against the oracle's decimal divided differences."""
    xi = L.leja_points(100)
    d = ei.divided_differences_imag(k, tau, c, gamma, 100)
    do = S.divided_differences_imag(k, tau, c, gamma, xi)
    assert np.abs(d - do).max() <= 1e-13 * max(1.0, np.abs(do).max())


@pytest.mark.parametrize("k,h,c,gamma,tol", [
    (0, 20.0, 0.0, 0.5, 1e-10),
    (0, 200.0, 0.0, 0.5, 1e-10),
    (0, 7.0, 3.0, 2.0, 1e-5),
    (1, 3.0, 1.0, 1.0, 1e-10),
    (2, 1.0, 5.0, 2.0, 1e-8),
])
def test_schedule_imag_matches_oracle(ei, k, h, c, gamma, tol):
    xi = L.leja_points(100)
    assert ei.schedule_imag(k, h, c, gamma, tol) == S.schedule_imag(k, h, c, gamma, tol, xi)


def test_imag_host_entries_invalid_arguments(ei):
    """ei_divided_differences_imag / ei_schedule_imag refuse what the header
    rules out: k outside 0..8, m or m_max outside range, non-positive tau, h
    or tol, gamma <= 0 for the schedule, non-finite c."""
    bad_dd = [(9, 1.0, 0.0, 1.0, 10), (-1, 1.0, 0.0, 1.0, 10), (0, 0.0, 0.0, 1.0, 10),
              (0, 1.0, float("nan"), 1.0, 10), (0, 1.0, 0.0, -1.0, 10), (0, 1.0, 0.0, 1.0, 101)]
    for k, tau, c, g, m in bad_dd:
        with pytest.raises(ei.EIError) as e:
            ei.divided_differences_imag(k, tau, c, g, m)
        assert e.value.status == ei.ERR_INVALID_ARG
    bad_s = [(0, -1.0, 0.0, 1.0, 1e-8), (0, 1.0, 0.0, 0.0, 1e-8), (0, 1.0, 0.0, 1.0, 0.0),
             (9, 1.0, 0.0, 1.0, 1e-8), (0, 1.0, float("inf"), 1.0, 1e-8)]
    for k, h, c, g, tol in bad_s:
        with pytest.raises(ei.EIError) as e:
            ei.schedule_imag(k, h, c, g, tol)
        assert e.value.status == ei.ERR_INVALID_ARG
    with pytest.raises(ei.EIError) as e:
        ei.schedule_imag(0, 1.0, 0.0, 1.0, 1e-8, m_max=0)
    assert e.value.status == ei.ERR_INVALID_ARG
    # gamma = 0 is a valid degenerate interval for the divided differences:
    # f is constant in xi, so d_0 = phi_k(-i tau c) and the rest vanish
    d = ei.divided_differences_imag(0, 2.0, 0.7, 0.0, 5)
    assert d[0] == pytest.approx(np.exp(-1j * 1.4), abs=1e-15)
    assert np.abs(d[1:]).max() == 0.0
