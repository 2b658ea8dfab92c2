"""Shared helpers of the GPU parity tests: build the library, move numpy
inputs to the device, and run the oracle beside the CUDA path."""
import numpy as np
import pytest


def require_gpu():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1309_4616_gb300 import build
    build.build()
    from paper_1309_4616_gb300 import ei
    return torch, ei


def dev(torch, a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def stencil_context(torch, ei, n, dx, D, b, c=0.0, bc=None, prec=0):
    """A Context holding the stencil operator; array coefficients go to the device."""
    dt = torch.float64 if prec == 0 else torch.float32
    ctx = ei.Context()
    to = (lambda x: x if isinstance(x, (int, float)) else dev(torch, x, dt))
    ctx.set_operator_stencil(n, dx, to(D), [to(x) for x in b], to(c), bc, prec)
    return ctx
