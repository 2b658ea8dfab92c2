"""The Schroedinger-type path of the oracle (oracle/skew.py: phi_k(-i h H) v
for a real symmetric H, complex products of Eq. (3) with K = C), pinned to
facts independent of it: the interpolation property of the complex divided
differences at the nodes, scipy's expm of the complex matrix -ihH, the unitarity
of e^{-ihH}, the augmented-matrix phi_1, and a diagonal H in closed form."""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import leja as L
from oracle import operators as O
from oracle import skew as S


@pytest.fixture(scope="module")
def xi():
    return L.leja_points(100)


def _chain(n, seed):
    """A real symmetric H: the negative Laplacian of a weighted path graph plus
    a random potential (a tight-binding Hamiltonian)."""
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.5, 1.5, n - 1)
    rowptr, col, val = [0], [], []
    for i in range(n):
        for j, x in ((i - 1, w[i - 1] if i > 0 else 0), (i + 1, w[i] if i < n - 1 else 0)):
            if 0 <= j < n:
                col.append(j)
                val.append(-x)
        rowptr.append(len(col))
    deg = np.zeros(n)
    for i in range(n):
        deg[i] = -sum(val[rowptr[i]:rowptr[i + 1]])
    pot = rng.uniform(-1, 1, n)
    op = O.CsrOperator(n, np.array(rowptr), np.array(col, dtype=np.int32), np.array(val),
                       deg + pot)
    return op


def test_divided_differences_interpolate_at_nodes(xi):
    k, tau, c, gamma = 0, 0.7, 1.3, 2.1
    d = S.divided_differences_imag(k, tau, c, gamma, xi[:31])
    nodes = xi[:31]
    p = S.newton_eval_c(d, xi, nodes)[-1]
    f = S.f_grid(k, tau, c, gamma, nodes)
    np.testing.assert_allclose(p, f, rtol=0, atol=1e-13)
    # phi_0(-i y): |f| = 1
    np.testing.assert_allclose(np.abs(f), 1.0, rtol=0, atol=1e-15)


def test_propagator_against_expm_and_unitary(xi):
    op = _chain(60, 1)
    H = op.dense()
    v = np.random.default_rng(2).standard_normal(60) + 1j * np.random.default_rng(3).standard_normal(60)
    h = 2.0
    y, s, degs = S.phi_apply_imag(op, 0, h, v, 1e-12, xi=xi)
    ex = scipy.linalg.expm(-1j * h * H) @ v
    assert np.linalg.norm(y - ex) / np.linalg.norm(ex) <= 1e-10
    assert abs(np.linalg.norm(y) - np.linalg.norm(v)) <= 1e-10 * np.linalg.norm(v)


def test_propagator_substeps(xi):
    """A long time: the schedule takes s > 1 and the powers of e^{-i tau H}
    still match the full propagator."""
    op = _chain(40, 4)
    v = np.random.default_rng(5).standard_normal(40).astype(complex)
    h = 40.0
    y, s, _ = S.phi_apply_imag(op, 0, h, v, 1e-10, xi=xi)
    assert s > 1
    ex = scipy.linalg.expm(-1j * h * op.dense()) @ v
    assert np.linalg.norm(y - ex) / np.linalg.norm(ex) <= 1e-8


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_phik_against_augmented_matrix(xi, k):
    """phi_k(-ihH)v is the top-right column of exp([[-ihH, v e_1^T], [0, J_k]]),
    J_k the k x k shift (ones above the diagonal)."""
    op = _chain(30, 6)
    n = 30
    v = np.random.default_rng(7).standard_normal(n) + 0.5j
    h = 0.8
    y, s, _ = S.phi_apply_imag(op, k, h, v, 1e-12, xi=xi)
    M = np.zeros((n + k, n + k), dtype=complex)
    M[:n, :n] = -1j * h * op.dense()
    M[:n, n] = v
    for i in range(k - 1):
        M[n + i, n + i + 1] = 1.0
    ex = scipy.linalg.expm(M)[:n, n + k - 1]
    assert s == 1 and np.linalg.norm(y - ex) / np.linalg.norm(ex) <= 1e-10


def test_diagonal_closed_form(xi):
    n = 25
    lam = np.linspace(-3.0, 5.0, n)
    op = O.CsrOperator(n, np.zeros(n + 1, dtype=np.int64), np.zeros(0, np.int32),
                       np.zeros(0), lam)
    v = np.ones(n, dtype=complex)
    for k in (0, 2):
        y, _, _ = S.phi_apply_imag(op, k, 0.9, v, 1e-13, xi=xi)
        z = -1j * 0.9 * lam
        if k == 0:
            ex = np.exp(z)
        else:  # (e^z - 1 - z)/z^2, 1/2 at z = 0
            zs = np.where(z == 0, 1.0, z)
            ex = np.where(z == 0, 0.5, (np.exp(zs) - 1 - zs) / zs ** 2)
        np.testing.assert_allclose(y, ex, rtol=1e-10, atol=1e-12)


def test_spin_bath_hamiltonian_against_kronecker():
    """The synthetic spin-bath matrix (the input of the Schroedinger workload)
    equals sum_bonds Jx X_i X_j + Jy Y_i Y_j + Jz Z_i Z_j built from 2x2 Pauli
    matrices by Kronecker products (spin i = bit i), and is real symmetric."""
    from paper_1309_4616_gb300 import workloads as W
    g = W.spin_bath(7)
    M = O.CsrOperator(g.n, g.rowptr, g.col, g.val, g.diag).dense()
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    Y = np.array([[0, -1j], [1j, 0]])
    Z = np.diag([1.0, -1.0]).astype(complex)

    def site(P, i, N):
        out = np.ones((1, 1), dtype=complex)
        for q in range(N - 1, -1, -1):
            out = np.kron(out, P if q == i else np.eye(2))
        return out

    H = np.zeros((g.n, g.n), dtype=complex)
    for i, j, jx, jy, jz in g.bonds:
        for P, J in ((X, jx), (Y, jy), (Z, jz)):
            H += J * site(P, i, 7) @ site(P, j, 7)
    assert np.abs(H.imag).max() == 0.0
    np.testing.assert_allclose(M, H.real, rtol=0, atol=1e-14)
    assert len(g.bonds) == 2 * 7 - 3 and len(g.col) == g.n * len(g.bonds)
