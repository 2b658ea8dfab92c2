"""The batched form: many independent 2D problems in one persistent launch.

Every problem's phi_1(h A) v is compared with the oracle (FP64: 1e-9 relative
2-norm, identical substep count and summed Leja degree; FP32: 1e-5).  The
full 1024-problem workload is checked on a sample of problems the oracle
finishes quickly, plus finiteness of all results and graph replay being
bit-identical.
"""
import math

import numpy as np
import pytest

from oracle import leja as L
from oracle import newton as Nw
from oracle import operators as O
from paper_1309_4616_gb300 import workloads as W

from gpu_helpers import rel_err, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return require_gpu()


@pytest.fixture(scope="module")
def xi():
    return L.leja_points(100)


def _oracle(p, xi, tol, m_max=100):
    op = O.StencilOperator(p.n, p.dx, p.D, p.b, bc=p.bc)
    return Nw.phi_apply(op, 1, p.h, p.v, tol, m_max=m_max, xi=xi)


def _small_batch(seed, count, nmax=48):
    probs = W.batch_2d(count=count, seed=seed, nmin=4, nmax=nmax)
    # include degenerate shapes
    probs[0].n = (1, 1)
    probs[0].v = np.array([[0.7]])
    probs[1].n = (5, 1)
    probs[1].v = np.linspace(1, 2, 5).reshape(1, 5)
    for p in probs[:2]:
        p.dx = (1.0 / (p.n[0] + 1), 1.0 / (p.n[1] + 1))
    return probs


def _pack(torch, probs, dtype):
    flat = np.concatenate([p.v.ravel() for p in probs])
    return torch.from_numpy(flat).to("cuda", dtype)


def _unpack(out, offsets, i):
    return out[offsets[i]:offsets[i + 1]]


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_vs_oracle(env, xi, prec):
    torch, ei = env
    probs = _small_batch(11 + prec, 48)
    tol = 1e-10 if prec == 0 else 1e-6
    b = ei.Batch(probs, prec=prec, tol=tol)
    dt = torch.float64 if prec == 0 else torch.float32
    v = _pack(torch, probs, dt)
    out = torch.empty_like(v)
    st = b.phi1(v, out)
    got = out.cpu().numpy().astype(np.float64)
    for i, p in enumerate(probs):
        ref, ost = _oracle(p, xi, tol)
        g = _unpack(got, b.offsets, i)
        if prec == 0:
            assert rel_err(g, ref) <= 1e-9, (i, p.n, rel_err(g, ref))
            assert st[i].s == ost.s and st[i].degree_sum == sum(ost.degrees), \
                (i, st[i].s, ost.s, st[i].degree_sum, ost.degrees)
            assert st[i].alpha == pytest.approx(ost.alpha, rel=1e-13, abs=1e-9)
        else:
            assert rel_err(g, ref) <= 1e-5, (i, p.n, rel_err(g, ref))
    b.close()


def test_batch_restarts_and_replay(env, xi):
    # a small m_max forces some problems to double s and rerun alone
    torch, ei = env
    probs = _small_batch(5, 24, nmax=40)
    for p in probs:
        p.h *= 20.0
    b = ei.Batch(probs, prec=0, tol=1e-10, options={"m_max": 12})
    v = _pack(torch, probs, torch.float64)
    out = torch.empty_like(v)
    st = b.phi1(v, out)
    got = out.cpu().numpy()
    assert any(s.restarts > 0 for s in st)
    for i, p in enumerate(probs):
        ref, ost = _oracle(p, xi, 1e-10, m_max=12)
        assert rel_err(_unpack(got, b.offsets, i), ref) <= 1e-9
        assert st[i].s == ost.s and st[i].restarts == ost.restarts
    out2 = torch.empty_like(v)
    b.phi1(v, out2)
    assert torch.equal(out, out2)
    b.close()


def test_batch_full_workload_sampled(env, xi):
    torch, ei = env
    probs = W.batch_2d()
    assert len(probs) == 1024
    b = ei.Batch(probs, prec=0, tol=1e-10)
    v = _pack(torch, probs, torch.float64)
    out = torch.empty_like(v)
    st = b.phi1(v, out)
    out2 = torch.empty_like(v)
    b.phi1(v, out2)
    assert torch.equal(out, out2)          # graph replay is bit-identical
    got = out.cpu().numpy()
    assert np.isfinite(got).all()
    # the problems the oracle finishes fastest (work ~ N^2 * total degree)
    work = [p.n[0] * p.n[1] * max(1, s.degree_sum) for p, s in zip(probs, st)]
    sample = list(np.argsort(work)[:12]) + list(np.argsort(work)[500:503])
    for i in sample:
        p = probs[i]
        ref, ost = _oracle(p, xi, 1e-10)
        assert rel_err(_unpack(got, b.offsets, i), ref) <= 1e-9
        assert st[i].s == ost.s and st[i].degree_sum == sum(ost.degrees)
    b.close()
