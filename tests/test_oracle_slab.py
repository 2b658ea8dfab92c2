"""The all-core oracle step (oracle/slab.py) against the serial oracle.

The slab version must reproduce newton.exp_rosenbrock_step: the same interval,
substep count and per-substep degrees, and the same state up to the norms'
summation order (1e-13 relative on the increment)."""
import numpy as np
import pytest

from oracle import newton as Nw
from oracle import operators as O
from oracle import slab as S


@pytest.mark.parametrize("parts", [1, 3, 7])
@pytest.mark.parametrize("bc,h", [((1,) * 6, 3e-3), ((0, 1, 1, 0, 0, 1), 1e-1)])
def test_slab_step_equals_serial(parts, bc, h):
    rng = np.random.default_rng(5)
    n = (19, 14, 13)
    shape = (13, 14, 19)
    dx = (1 / 19, 1 / 19, 1 / 19)
    D = rng.uniform(0.5, 1.5, shape)
    b = tuple(rng.uniform(-2, 2, shape) for _ in range(3))
    u0 = rng.uniform(0, 1, shape)
    tol = 1e-10
    ref, st = Nw.exp_rosenbrock_step(O.StencilOperator(n, dx, D, b, bc=bc), u0, h, tol)
    sop = S.SlabStencil(n, dx, D, b, bc=bc, parts=parts)
    got, st2 = S.exp_rosenbrock_step(sop, u0, h, tol)
    sop.close()
    assert (st2.alpha, st2.beta) == (st.alpha, st.beta)
    assert st2.s == st.s and st2.degrees == st.degrees and st2.matvecs == st.matvecs
    inc, inc2 = ref - u0, got - u0
    assert np.linalg.norm(inc2 - inc) <= 1e-13 * np.linalg.norm(inc)


def test_slab_euler_step_equals_serial():
    rng = np.random.default_rng(6)
    n = (17, 15, 12)
    shape = (12, 15, 17)
    dx = (1 / 17, 1 / 17, 1 / 17)
    D = rng.uniform(0.5, 1.5, shape)
    b = tuple(rng.uniform(-2, 2, shape) for _ in range(3))
    u0 = rng.uniform(0, 1, shape)
    h, tol = 2e-2, 1e-8
    op = O.StencilOperator(n, dx, D, b, bc=(1,) * 6)
    ref, st = Nw.exp_euler_step(op, u0, h, tol, Nw.NONLIN_LOGISTIC)
    sop = S.SlabStencil(n, dx, D, b, bc=(1,) * 6, parts=4)
    got, st2 = S.exp_euler_step(sop, u0, h, tol)
    sop.close()
    assert (st2.alpha, st2.beta) == (st.alpha, st.beta)
    assert st2.s == st.s and st2.degrees == st.degrees
    inc, inc2 = ref - u0, got - u0
    assert np.linalg.norm(inc2 - inc) <= 1e-13 * np.linalg.norm(inc)
