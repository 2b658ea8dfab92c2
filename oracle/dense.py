"""phi_k(hA)v by definition, for small dense A.

ORACLE — test infrastructure only (see oracle/__init__.py).

phi_0 = exp and phi_k(z) = sum_{i>=0} z^i/(i+k)! (the entire functions of
Eq. (2)).  For k >= 1 the augmented matrix
    M = [[hA, v, 0, .., 0], [0, J_k]],   J_k the k x k upper shift,
satisfies  expm(M)[:n, n+k-1] = phi_k(hA) v  (Saad 1992; Al-Mohy & Higham
2011), so phi_k(hA)v is one call of scipy's scaling-and-squaring expm.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def phi_dense(A: np.ndarray, k: int, h: float, v: np.ndarray) -> np.ndarray:
    n = A.shape[0]
    v = np.asarray(v, dtype=np.float64).ravel()
    if k == 0:
        return scipy.linalg.expm(h * A) @ v
    M = np.zeros((n + k, n + k))
    M[:n, :n] = h * A
    M[:n, n] = v
    for i in range(k - 1):
        M[n + i, n + i + 1] = 1.0
    return scipy.linalg.expm(M)[:n, n + k - 1]
