"""The allocation-free spectral-interval entry point.

ei_estimate_spectrum_stencil_noalloc serves callers that must not allocate
device memory: real-time or budgeted code that reserves all of it up front,
and hosts whose framework owns the GPU's memory through its own pool.  Its
reduction scratch lives in a fixed array inside the library.  Here it is
called through the C ABI twice in a row on two different operators (FP64 and
FP32 coefficients), and each result must equal, bit for bit, the interval that
ei_set_operator_stencil + ei_estimate_spectrum report for the same operator:
both evaluate the same rows and take an exact min/max.  After a warm-up call,
repeated calls must leave the device's free memory unchanged.  The file is
collected last so that a failure here does not hide the other tests' results.
"""
import ctypes as C

import numpy as np
import pytest

from gpu_helpers import dev, require_gpu

pytestmark = pytest.mark.gpu


def _noalloc(ei, torch, n, dx, D, b, c, bc, prec=0):
    dim = len(n)
    n3 = (C.c_int64 * 3)(*(list(n) + [1] * (3 - dim)))
    dx3 = (C.c_double * 3)(*(list(dx) + [1.0] * (3 - dim)))
    bc6 = (C.c_int * 6)(*(list(bc) + [1] * (6 - len(bc))))
    bptr = (C.c_void_p * 3)()
    bcst = (C.c_double * 3)()
    for e in range(dim):
        bptr[e] = b[e].data_ptr()
    alpha, beta = C.c_double(), C.c_double()
    stream = torch.cuda.current_stream()
    st = ei.lib().ei_estimate_spectrum_stencil_noalloc(
        0, C.c_void_p(stream.cuda_stream), dim, n3, dx3, C.c_void_p(D.data_ptr()), 0.0, bptr,
        bcst, C.c_void_p(c.data_ptr()) if c is not None else None, 0.0, bc6, prec,
        C.byref(alpha), C.byref(beta))
    return st, alpha.value, beta.value


def _operator(torch, seed, n, dtype):
    rng = np.random.default_rng(seed)
    shape = tuple(reversed(n))
    D = dev(torch, rng.uniform(0.5, 1.5, shape), dtype)
    b = [dev(torch, rng.uniform(-2, 2, shape), dtype) for _ in n]
    c = dev(torch, rng.uniform(-1, 1, shape), dtype)
    return D, b, c


CASES = [((37, 29, 21), (1 / 37, 1 / 30, 1 / 22), (1, 0, 1, 1, 0, 1), 1),
         ((301, 77), (0.01, 0.02), (0, 1, 1, 0), 2)]


@pytest.mark.parametrize("prec", [0, 1], ids=["f64", "f32"])
def test_noalloc_spectrum_equals_context_twice(prec):
    torch, ei = require_gpu()
    dtype = torch.float64 if prec == 0 else torch.float32
    for n, dx, bc, seed in CASES:
        D, b, c = _operator(torch, seed, n, dtype)
        ctx = ei.Context()
        ctx.set_operator_stencil(n, dx, D, b, c, bc, prec)
        ref = ctx.estimate_spectrum()
        ctx.close()
        for _ in range(2):  # the shared scratch keeps the last call's contents
            st, a, bb = _noalloc(ei, torch, n, dx, D, b, c, bc, prec)
            assert st == ei.OK, ei.status_string(st)
            assert (a, bb) == ref


def test_noalloc_allocates_nothing():
    torch, ei = require_gpu()
    n, dx, bc, seed = CASES[0]
    D, b, c = _operator(torch, seed, n, torch.float64)
    torch.cuda.synchronize()
    st, a0, b0 = _noalloc(ei, torch, n, dx, D, b, c, bc)  # first call on the device: set-up
    assert st == ei.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(20):
        st, a, bb = _noalloc(ei, torch, n, dx, D, b, c, bc)
        assert st == ei.OK and (a, bb) == (a0, b0)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_single_nan_coefficient():
    torch, ei = require_gpu()
    n, dx, bc, seed = CASES[0]
    D, b, c = _operator(torch, seed, n, torch.float64)
    D[3, 5, 7] = float("nan")
    st, _, _ = _noalloc(ei, torch, n, dx, D, b, c, bc)
    assert st == ei.ERR_NONFINITE
    ctx = ei.Context()
    with pytest.raises(ei.EIError):
        ctx.set_operator_stencil(n, dx, D, b, c, bc, ei.PREC_F64)
    ctx.close()


def test_noalloc_rejects_too_many_points():
    torch, ei = require_gpu()
    D, b, c = _operator(torch, 3, (4, 4, 4), torch.float64)
    st, _, _ = _noalloc(ei, torch, (1024, 1024, 129), (1.0, 1.0, 1.0), D, b, c, (1,) * 6)
    assert st == ei.ERR_INVALID_ARG
