"""A constant-coefficient stencil operator by the faces its rows touch (oracle).

With D, b and c constant, Sec. III-A's seven-point rows differ only where a
boundary condition is folded in, so every row is fixed by which of the six
faces its point lies on: a neighbour coefficient is the interior value
D/dx^2 + s b/(2 dx) or 0 where that neighbour is a ghost, and the diagonal
is the interior one plus, for each Neumann ghost, that same interior
neighbour value (Dirichlet ghosts leave the interior diagonal as it is).
The float-float library reads such an operator from a 70-entry table built
on exactly this; here the oracle's assembled rows are checked against it on
grids with extents 1, 2 and more, 2D and 3D, every face code.  No GPU.
"""
import itertools

import numpy as np
import pytest

from oracle import operators as O

CASES = [
    ((7, 5, 4), (1, 0, 1, 1, 0, 1), 0.8, (0.5, -0.3, 0.2), -0.7),
    ((6, 2, 3), (0, 1, 1, 0, 1, 0), 0.3, (-1.0, 0.4, 0.6), 0.2),
    ((1, 4, 5), (1, 1, 0, 1, 0, 0), 0.5, (0.3, 0.2, -0.1), 0.0),
    ((9, 6), (1, 0, 0, 1), 0.6, (0.7, -0.2), -0.3),
    ((2, 1), (0, 0, 1, 1), 1.1, (0.0, 0.4), 0.5),
]


def _face_class(i, n):
    return (1 if i == 0 else 0) | (2 if i == n - 1 else 0)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_rows_follow_face_class(case):
    n, bc, D, b, c = CASES[case]
    dim = len(n)
    dx = tuple(1.0 / (v + 1) for v in n)
    shape = tuple(reversed(n))
    op = O.StencilOperator(n, dx, np.full(shape, D), tuple(np.full(shape, x) for x in b),
                           c=np.full(shape, c), bc=bc)
    # the interior neighbour values, the interior diagonal
    nb = {(ax, sgn): D / dx[ax] ** 2 + sgn * b[ax] / (2.0 * dx[ax])
          for ax in range(dim) for sgn in (-1, 1)}
    d_int = c - sum(2.0 * D / dx[ax] ** 2 for ax in range(dim))
    seen = {}
    for idx in itertools.product(*(range(v) for v in shape)):
        crd = tuple(reversed(idx))  # (x, y[, z])
        cls = tuple(_face_class(crd[ax], n[ax]) for ax in range(dim))
        row = (tuple(op.off[(ax, sgn)][idx] for ax in range(dim) for sgn in (-1, 1)),
               op.diag[idx])
        # every row of one class is the same row
        if cls in seen:
            assert row == seen[cls], (crd, cls)
        else:
            seen[cls] = row
        # and it is the interior row with the class's faces folded in
        diag = d_int
        for ax in range(dim):
            for side, sgn in ((0, -1), (1, 1)):
                ghost = cls[ax] & (1 << side)
                want = 0.0 if ghost else nb[(ax, sgn)]
                assert op.off[(ax, sgn)][idx] == pytest.approx(want, rel=1e-14, abs=1e-12)
                if ghost and bc[2 * ax + side] == O.NEUMANN0:
                    diag += nb[(ax, sgn)]
        assert op.diag[idx] == pytest.approx(diag, rel=1e-13, abs=1e-10)
