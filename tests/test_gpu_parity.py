"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar: FP64 results within 1e-9 relative 2-norm of the oracle, Leja degree per
substep and substep count identical, Gershgorin interval within 1e-13
relative; the FP32 form within 1e-5.  Grid sizes span several kernel tiles
(32 x 8 x 16 points) with ragged tails in every axis.
"""
import numpy as np
import pytest

from oracle import leja as L
from oracle import newton as Nw
from oracle import operators as O
from paper_1309_4616_gb300 import workloads as W

from gpu_helpers import dev, rel_err, require_gpu, stencil_context

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    return require_gpu()


@pytest.fixture(scope="module")
def xi():
    return L.leja_points(100)


def _check_stats(st, ost):
    assert st.s == ost.s, (st.s, ost.s)
    assert st.degree_list() == list(ost.degrees)[: len(st.degree_list())], \
        (st.degree_list(), ost.degrees)
    assert st.alpha == pytest.approx(ost.alpha, rel=1e-13, abs=1e-9)
    assert st.beta == pytest.approx(ost.beta, rel=1e-13, abs=1e-9)


# --------------------------------------------------------------------------
# 2D advection-diffusion on 64 x 64, the small configuration in full
# --------------------------------------------------------------------------
@pytest.mark.parametrize("arith", [0, 1])
@pytest.mark.parametrize("single", [0, 1, 2])
def test_adv_diff_2d_phi1(env, xi, arith, single):
    torch, ei = env
    w = W.adv_diff_2d()
    op = O.StencilOperator(w.n, w.dx, w.D, w.b, bc=w.bc)
    ref, ost = Nw.phi_apply(op, 1, w.h, w.v, w.tol, xi=xi)
    ctx = stencil_context(torch, ei, w.n, w.dx, w.D, w.b, 0.0, w.bc)
    a, b = ctx.estimate_spectrum()
    assert a == pytest.approx(-3380.0, rel=1e-13) and abs(b) < 1e-9
    v = dev(torch, w.v)
    out = torch.empty_like(v)
    st = ctx.phi_apply(1, w.h, v, out, w.tol, {"arith": arith, "single_iter": single})
    assert rel_err(out.cpu().numpy(), ref) <= FP64_TOL
    _check_stats(st, ost)


# --------------------------------------------------------------------------
# 3D variable coefficients, ragged tiles
# --------------------------------------------------------------------------
def _fields_3d(rng, n):
    nx, ny, nz = n
    D = rng.uniform(0.5, 1.5, (nz, ny, nx))
    b = tuple(rng.uniform(-2, 2, (nz, ny, nx)) for _ in range(3))
    return D, b


@pytest.mark.parametrize("single", [0, 1, 2])
@pytest.mark.parametrize("arith", [0, 1])
def test_rosenbrock_3d_neumann(env, xi, single, arith):
    torch, ei = env
    rng = np.random.default_rng(21)
    n = (37, 29, 21)
    dx = (1 / 37, 1 / 37, 1 / 37)
    D, b = _fields_3d(rng, n)
    u0 = rng.uniform(0, 1, (21, 29, 37))
    op = O.StencilOperator(n, dx, D, b, bc=(O.NEUMANN0,) * 6)
    h, tol = 2e-4, 1e-10
    ref, ost = Nw.exp_rosenbrock_step(op, u0, h, tol, xi=xi)
    ctx = stencil_context(torch, ei, n, dx, D, b, 0.0, (1,) * 6)
    u = dev(torch, u0)
    st = ctx.step(ei.EXP_ROSENBROCK, h, u, ei.NONLIN_LOGISTIC, tol,
                  {"arith": arith, "single_iter": single})
    got = u.cpu().numpy()
    assert rel_err(got - u0, ref - u0) <= FP64_TOL
    assert rel_err(got, ref) <= FP64_TOL
    _check_stats(st, ost)


@pytest.mark.parametrize("rosenbrock", [False, True])
@pytest.mark.parametrize("arith", [0, 1])
def test_step_3d_mixed_bc_with_c(env, xi, arith, rosenbrock):
    # native FP64 runs F (and J's diagonal and interval) in one TMA pass
    torch, ei = env
    rng = np.random.default_rng(22)
    n = (45, 17, 33)
    dx = (0.02, 0.025, 0.03)
    D, b = _fields_3d(rng, n)
    c = rng.uniform(-3, 1, (33, 17, 45))
    bc = (0, 1, 1, 0, 0, 1)
    u0 = rng.uniform(0, 1, (33, 17, 45))
    op = O.StencilOperator(n, dx, D, b, c=c, bc=bc)
    h, tol = 1e-4, 1e-10
    if rosenbrock:
        ref, ost = Nw.exp_rosenbrock_step(op, u0, h, tol, xi=xi)
    else:
        ref, ost = Nw.exp_euler_step(op, u0, h, tol, Nw.NONLIN_LOGISTIC, xi=xi)
    ctx = stencil_context(torch, ei, n, dx, D, b, c, bc)
    u = dev(torch, u0)
    st = ctx.step(ei.EXP_ROSENBROCK if rosenbrock else ei.EXP_EULER, h, u, ei.NONLIN_LOGISTIC,
                  tol, {"arith": arith})
    got = u.cpu().numpy()
    assert rel_err(got - u0, ref - u0) <= FP64_TOL
    _check_stats(st, ost)


@pytest.mark.parametrize("m_max", [100, 15])
def test_substeps_2d_mixed(env, xi, m_max):
    # a large h makes the a-priori rule ask for several substeps
    torch, ei = env
    rng = np.random.default_rng(23)
    n = (70, 43)
    dx = (1 / 71, 1 / 44)
    D = rng.uniform(0.2, 1.0, (43, 70))
    b = (rng.uniform(-1, 1, (43, 70)), rng.uniform(-1, 1, (43, 70)))
    bc = (1, 0, 0, 1)
    v0 = rng.standard_normal((43, 70))
    op = O.StencilOperator(n, dx, D, b, bc=bc)
    h, tol = 0.02, 1e-10
    ref, ost = Nw.phi_apply(op, 1, h, v0, tol, m_max=m_max, xi=xi)
    assert ost.s > 1
    ctx = stencil_context(torch, ei, n, dx, D, b, 0.0, bc)
    v = dev(torch, v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply(1, h, v, out, tol, {"m_max": m_max})
    assert rel_err(out.cpu().numpy(), ref) <= FP64_TOL
    _check_stats(st, ost)


@pytest.mark.parametrize("k", [0, 2])
def test_phi_k_other_orders(env, xi, k):
    torch, ei = env
    rng = np.random.default_rng(30 + k)
    n = (33, 9)
    dx = (1 / 34, 1 / 10)
    D = rng.uniform(0.1, 0.3, (9, 33))
    b = (rng.uniform(-1, 1, (9, 33)), rng.uniform(-1, 1, (9, 33)))
    v0 = rng.standard_normal((9, 33))
    op = O.StencilOperator(n, dx, D, b)
    h, tol = (2e-3 if k == 0 else 2e-4), 1e-11
    ref, ost = Nw.phi_apply(op, k, h, v0, tol, xi=xi)
    ctx = stencil_context(torch, ei, n, dx, D, b)
    v = dev(torch, v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply(k, h, v, out, tol)
    assert rel_err(out.cpu().numpy(), ref) <= FP64_TOL
    _check_stats(st, ost)


def test_fp32_form(env, xi):
    # FP32 vectors and matvec; FP64-class divided differences, interval and sum
    torch, ei = env
    rng = np.random.default_rng(24)
    n = (40, 24, 20)
    dx = (1 / 40,) * 3
    D, b = _fields_3d(rng, n)
    D32 = D.astype(np.float32)
    b32 = tuple(x.astype(np.float32) for x in b)
    u0 = rng.uniform(0, 1, (20, 24, 40)).astype(np.float32)
    # the oracle runs in FP64 on the same (FP32-representable) inputs
    op = O.StencilOperator(n, dx, D32.astype(np.float64), [x.astype(np.float64) for x in b32],
                           bc=(1,) * 6)
    h, tol = 5e-5, 1e-6
    ref, ost = Nw.exp_euler_step(op, u0.astype(np.float64), h, tol, Nw.NONLIN_LOGISTIC, xi=xi)
    ctx = stencil_context(torch, ei, n, dx, D32, b32, 0.0, (1,) * 6, prec=1)
    u = dev(torch, u0)
    ctx.step(ei.EXP_EULER, h, u, ei.NONLIN_LOGISTIC, tol)
    got = u.cpu().numpy().astype(np.float64)
    assert rel_err(got, ref) <= FP32_TOL
    assert rel_err(got - u0, ref - u0) <= 1e-4


# --------------------------------------------------------------------------
# CSR
# --------------------------------------------------------------------------
def _graph(n, seed):
    g = W.rgg_graph(n=n, mean_degree=12.0, seed=seed)
    return g


@pytest.mark.parametrize("order", ["morton", "random"])
def test_csr_graph_phi1(env, xi, order):
    torch, ei = env
    g = W.rgg_graph(n=3000, mean_degree=12.0, seed=77, order=order)
    op = O.CsrOperator(g.n, g.rowptr, g.col, g.val, -g.deg_w)
    v0 = W.random_vector(g.n, 5)
    h = 40.0 / (2 * g.deg_w.max())
    ref, ost = Nw.phi_apply(op, 1, h, v0, 1e-10, xi=xi)
    ctx = ei.Context()
    ctx.set_operator_csr(g.n, dev(torch, g.rowptr), dev(torch, g.col), dev(torch, g.val),
                         dev(torch, -g.deg_w))
    a, b = ctx.estimate_spectrum()
    assert a == pytest.approx(-2 * g.deg_w.max(), rel=1e-13)
    v = dev(torch, v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply(1, h, v, out, 1e-10)
    assert rel_err(out.cpu().numpy(), ref) <= FP64_TOL
    _check_stats(st, ost)


def test_csr_rosenbrock(env, xi):
    torch, ei = env
    g = W.rgg_graph(n=2000, mean_degree=12.0, seed=78)
    op = O.CsrOperator(g.n, g.rowptr, g.col, g.val, -g.deg_w)
    u0 = np.random.default_rng(3).uniform(0, 1, g.n)
    h = 0.5
    ref, ost = Nw.exp_rosenbrock_step(op, u0, h, 1e-10, xi=xi)
    ctx = ei.Context()
    ctx.set_operator_csr(g.n, dev(torch, g.rowptr), dev(torch, g.col), dev(torch, g.val),
                         dev(torch, -g.deg_w))
    u = dev(torch, u0)
    st = ctx.step(ei.EXP_ROSENBROCK, h, u, ei.NONLIN_LOGISTIC, 1e-10)
    got = u.cpu().numpy()
    assert rel_err(got - u0, ref - u0) <= FP64_TOL
    _check_stats(st, ost)


def _irregular_graph(n, seed, hub_degree):
    """Symmetric weighted graph with isolated nodes (empty rows), a hub whose
    row is longer than a warp's 256-entry chunk, and ragged degrees."""
    rng = np.random.default_rng(seed)
    edges = set()
    for i in range(n):
        for j in rng.integers(0, n, size=rng.integers(0, 9)):
            if i != j:
                edges.add((min(i, j), max(int(j), i)))
    hub = n // 3
    for j in rng.choice(n, size=min(hub_degree, n - 1), replace=False):
        if j != hub:
            edges.add((min(hub, int(j)), max(hub, int(j))))
    iso = set(range(5, n, 97))  # isolated nodes
    edges = {(a, b) for a, b in edges if a not in iso and b not in iso}
    w = {e: rng.uniform(0.5, 2.0) for e in edges}
    rows = [[] for _ in range(n)]
    for (a, b), x in w.items():
        rows[a].append((b, x))
        rows[b].append((a, x))
    rowptr = np.zeros(n + 1, dtype=np.int64)
    col, val = [], []
    for i in range(n):
        rows[i].sort()
        rowptr[i + 1] = rowptr[i] + len(rows[i])
        col += [c for c, _ in rows[i]]
        val += [x for _, x in rows[i]]
    col = np.array(col, dtype=np.int32)
    val = np.array(val)
    deg = np.bincount(np.repeat(np.arange(n), np.diff(rowptr)), val, minlength=n)
    return rowptr, col, val, deg


@pytest.mark.parametrize("lanes", [0, 1, 2, 4, 32])
@pytest.mark.parametrize("n,hub", [(1000, 700), (20, 19), (33, 5)])
def test_csr_irregular_rows(env, xi, n, hub, lanes):
    """Empty rows, a row longer than a chunk, warps whose entries span several
    chunks, n below and not a multiple of 32; the sliced kernel (0, the
    default: the hub pads its slice, empty rows end their windows) and the 1-,
    2-, 4- and 32-lane kernels on the CSR arrays."""
    torch, ei = env
    rowptr, col, val, deg = _irregular_graph(n, 5 + n, hub)
    assert (np.diff(rowptr) == 0).any()
    if hub > 256:
        assert np.diff(rowptr).max() > 256
    op = O.CsrOperator(n, rowptr, col, val, -deg)
    v0 = W.random_vector(n, 9)
    h = 30.0 / (2 * deg.max())
    ref, ost = Nw.phi_apply(op, 1, h, v0, 1e-10, xi=xi)
    ctx = ei.Context()
    ctx.set_operator_csr(n, dev(torch, rowptr), dev(torch, col), dev(torch, val), dev(torch, -deg))
    v = dev(torch, v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply(1, h, v, out, 1e-10, {"csr_lanes": lanes})
    assert rel_err(out.cpu().numpy(), ref) <= FP64_TOL
    _check_stats(st, ost)
    if lanes in (0, 4):  # the native FP64 form of the same kernel
        st = ctx.phi_apply(1, h, v, out, 1e-10,
                           {"csr_lanes": lanes, "arith": ei.ARITH_NATIVE_F64})
        assert rel_err(out.cpu().numpy(), ref) <= FP64_TOL
        _check_stats(st, ost)


@pytest.mark.parametrize("defect", ["col_high", "col_negative", "rowptr_start", "rowptr_end",
                                    "rowptr_decreasing"])
def test_csr_invalid_structure_rejected(env, defect):
    """A structure the kernels could not read safely is refused before use
    (the check reads only the stated n + 1 and nnz entries); the context stays
    usable."""
    torch, ei = env
    g = W.rgg_graph(n=500, seed=3)
    rowptr, col = g.rowptr.copy(), g.col.copy()
    if defect == "col_high":
        col[17] = g.n
    elif defect == "col_negative":
        col[-1] = -1
    elif defect == "rowptr_start":
        rowptr[0] = 1
    elif defect == "rowptr_end":
        rowptr[-1] -= 1
    else:
        rowptr[200] = rowptr[202] + 1
    ctx = ei.Context()
    with pytest.raises(ei.EIError) as e:
        ctx.set_operator_csr(g.n, dev(torch, rowptr), dev(torch, col), dev(torch, g.val),
                             dev(torch, -g.deg_w))
    assert e.value.status == ei.ERR_INVALID_ARG
    ctx.set_operator_csr(g.n, dev(torch, g.rowptr), dev(torch, g.col), dev(torch, g.val),
                         dev(torch, -g.deg_w))
    assert ctx.estimate_spectrum()[0] == pytest.approx(-2 * g.deg_w.max(), rel=1e-13)
    ctx.close()


# --------------------------------------------------------------------------
# edge cases
# --------------------------------------------------------------------------
def test_zero_vector_and_scalar_operator(env, xi):
    torch, ei = env
    ctx = stencil_context(torch, ei, (19, 5, 3), (0.1, 0.1, 0.1), 1.0, (0.0, 0.0, 0.0), 0.0,
                          (1,) * 6)
    z = torch.zeros(3 * 5 * 19, dtype=torch.float64, device="cuda")
    out = torch.full_like(z, 7.0)
    st = ctx.phi_apply(1, 0.01, z, out, 1e-10)
    assert not out.any().item() and st.degree_sum == 0
    # A = cI: D = 0, b = 0, Neumann everywhere, c = -3 -> gamma = 0
    ctx2 = stencil_context(torch, ei, (11, 4), (0.1, 0.1), 0.0, (0.0, 0.0), -3.0, (1,) * 4)
    assert ctx2.estimate_spectrum() == (-3.0, -3.0)
    v0 = np.random.default_rng(1).standard_normal(44)
    v = dev(torch, v0)
    out = torch.empty_like(v)
    for k in (0, 1, 2):
        ctx2.phi_apply(k, 0.1, v, out, 1e-10)
        assert np.allclose(out.cpu().numpy(), L.phi_scalar(k, -0.3) * v0, rtol=1e-14)


def test_single_point_and_thin_grids(env, xi):
    torch, ei = env
    for n, bc in [((1, 1, 1), (0,) * 6), ((1, 7, 1), (0, 1, 1, 0, 0, 1)), ((65, 1), (0, 0, 1, 1))]:
        dim = len(n)
        rng = np.random.default_rng(sum(n))
        shape = tuple(reversed(n))
        D = rng.uniform(0.5, 1.5, shape)
        b = tuple(rng.uniform(-1, 1, shape) for _ in range(dim))
        dx = tuple([0.1] * dim)
        v0 = rng.standard_normal(shape)
        op = O.StencilOperator(n, dx, D, b, bc=bc)
        ref, ost = Nw.phi_apply(op, 1, 1e-3, v0, 1e-10, xi=xi)
        ctx = stencil_context(torch, ei, n, dx, D, b, 0.0, bc)
        v = dev(torch, v0)
        out = torch.empty_like(v)
        st = ctx.phi_apply(1, 1e-3, v, out, 1e-10)
        assert rel_err(out.cpu().numpy(), ref) <= FP64_TOL
        _check_stats(st, ost)


def test_errors_leave_outputs_untouched(env):
    torch, ei = env
    ctx = ei.Context()
    v = torch.ones(8, dtype=torch.float64, device="cuda")
    out = torch.full_like(v, 5.0)
    with pytest.raises(ei.EIError) as e:
        ctx.phi_apply(1, 0.1, v, out, 1e-10)
    assert e.value.status == ei.ERR_STATE
    ctx = stencil_context(torch, ei, (4, 2), (0.1, 0.1), 1.0, (0.0, 0.0), 0.0)
    for args in [(-1, 0.1, 1e-10), (1, 0.0, 1e-10), (1, 0.1, 0.0), (1, float("nan"), 1e-10)]:
        with pytest.raises(ei.EIError) as e:
            ctx.phi_apply(args[0], args[1], v, out, args[2])
        assert e.value.status == ei.ERR_INVALID_ARG
    bad = v.clone()
    bad[3] = float("nan")
    with pytest.raises(ei.EIError) as e:
        ctx.phi_apply(1, 0.1, bad, out, 1e-10)
    assert e.value.status == ei.ERR_NONFINITE
    assert (out == 5.0).all().item()
    u = bad.clone()
    with pytest.raises(ei.EIError) as e:
        ctx.step(ei.EXP_EULER, 0.1, u, ei.NONLIN_LOGISTIC, 1e-10)
    assert e.value.status == ei.ERR_NONFINITE
    assert torch.equal(torch.isnan(u), torch.isnan(bad))
    # the Rosenbrock interval of J = A + diag(g'(u)) with a NaN of either sign
    # or an infinity in u, in both arithmetics
    for arith in (ei.ARITH_NATIVE_F64, ei.ARITH_DF):
        for val in (float("nan"), -float("nan"), float("inf"), -float("inf")):
            u = v.clone()
            u[3] = val
            with pytest.raises(ei.EIError) as e:
                ctx.step(ei.EXP_ROSENBROCK, 0.1, u, ei.NONLIN_LOGISTIC, 1e-10, {"arith": arith})
            assert e.value.status == ei.ERR_NONFINITE
    with pytest.raises(ei.EIError) as e:
        ctx.step(7, 0.1, u, ei.NONLIN_LOGISTIC, 1e-10)
    assert e.value.status == ei.ERR_INVALID_ARG


def test_step_host_equals_step(env, xi):
    torch, ei = env
    rng = np.random.default_rng(40)
    n = (20, 12, 9)
    D, b = _fields_3d(rng, n)
    u0 = rng.uniform(0, 1, (9, 12, 20))
    ctx = stencil_context(torch, ei, n, (0.05,) * 3, D, b, 0.0, (1,) * 6)
    ud = dev(torch, u0)
    ctx.step(ei.EXP_ROSENBROCK, 1e-4, ud, ei.NONLIN_LOGISTIC, 1e-10)
    uh = torch.from_numpy(u0.copy()).pin_memory()
    ctx.step_host(ei.EXP_ROSENBROCK, 1e-4, uh, ei.NONLIN_LOGISTIC, 1e-10)
    assert torch.equal(uh, ud.cpu())


def test_context_reuse_across_operator_kinds(env, xi):
    """One context takes a 3D stencil, a CSR graph, then a constant-coefficient
    2D stencil that needs several substeps; every call matches the oracle
    (nothing of one operator's layout carries over to the next)."""
    torch, ei = env
    ctx = ei.Context()
    w = W.adr_3d(n=18, h=2e-3)
    op = O.StencilOperator(w.n, w.dx, w.D, w.b, bc=w.bc)
    ref, ost = Nw.exp_rosenbrock_step(op, w.u0, w.h, w.tol, xi=xi)
    ctx.set_operator_stencil(w.n, w.dx, dev(torch, w.D), [dev(torch, x) for x in w.b], 0.0,
                             list(w.bc), ei.PREC_F64)
    u = dev(torch, w.u0)
    st = ctx.step(ei.EXP_ROSENBROCK, w.h, u, ei.NONLIN_LOGISTIC, w.tol)
    assert rel_err(u.cpu().numpy() - w.u0, ref - w.u0) <= FP64_TOL
    _check_stats(st, ost)

    g = W.rgg_graph(n=3000, seed=8)
    gop = O.CsrOperator(g.n, g.rowptr, g.col, g.val, -g.deg_w)
    h = 30.0 / (2.0 * g.deg_w.max())
    v0 = W.random_vector(g.n, 2)
    ref, ost = Nw.phi_apply(gop, 1, h, v0, 1e-10, xi=xi)
    ctx.set_operator_csr(g.n, dev(torch, g.rowptr), dev(torch, g.col), dev(torch, g.val),
                         dev(torch, -g.deg_w))
    v = dev(torch, v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply(1, h, v, out, 1e-10)
    assert rel_err(out.cpu().numpy(), ref) <= FP64_TOL
    _check_stats(st, ost)

    n, dx = (48, 48), (1 / 49, 1 / 49)
    sop = O.StencilOperator(n, dx, 0.2, (0.4, 0.9), bc=(0, 0, 0, 0))
    v0 = np.random.default_rng(4).standard_normal((48, 48))
    ref, ost = Nw.phi_apply(sop, 1, 0.25, v0, 1e-8, xi=xi)
    assert ost.s > 1
    ctx.set_operator_stencil(n, dx, 0.2, [0.4, 0.9], 0.0, [0, 0, 0, 0], ei.PREC_F64)
    v = dev(torch, v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply(1, 0.25, v, out, 1e-8)
    assert rel_err(out.cpu().numpy(), ref) <= FP64_TOL
    _check_stats(st, ost)
    ctx.close()


@pytest.mark.parametrize("method", ["euler", "rosenbrock"])
def test_step_host_paths_match_device(env, method):
    """ei_step_host on pinned (mapped: read and written by the kernels) and on
    pageable host memory (copied) gives the device step's result bit for bit."""
    torch, ei = env
    rng = np.random.default_rng(61)
    n = (41, 23, 17)
    dx = (1 / 41, 1 / 41, 1 / 41)
    D, b = _fields_3d(rng, n)
    u0 = rng.uniform(0, 1, (17, 23, 41))
    m = ei.EXP_EULER if method == "euler" else ei.EXP_ROSENBROCK
    ctx = stencil_context(torch, ei, n, dx, D, b, 0.0, (1,) * 6)
    ud = dev(torch, u0)
    ctx.step(m, 3e-4, ud, ei.NONLIN_LOGISTIC, 1e-10)
    ref = ud.cpu().numpy()
    pinned = torch.from_numpy(u0.copy()).pin_memory()
    ctx.step_host(m, 3e-4, pinned, ei.NONLIN_LOGISTIC, 1e-10)
    pageable = torch.from_numpy(u0.copy())
    ctx.step_host(m, 3e-4, pageable, ei.NONLIN_LOGISTIC, 1e-10)
    assert np.array_equal(pinned.numpy(), ref) and np.array_equal(pageable.numpy(), ref)
    ctx.close()


def _smooth_case():
    n = (37, 29, 21)
    shape = (21, 29, 37)
    dx = (1 / 37,) * 3
    z, y, x = np.meshgrid(*(np.arange(k) + 0.5 for k in shape), indexing="ij")
    D = 1 + 0.3 * np.sin(np.pi * x / 37) * np.cos(np.pi * y / 29)
    v0 = np.cos(np.pi * x / 37) * np.cos(np.pi * y / 29) + 0.5 * np.cos(np.pi * z / 21)
    return n, dx, D, v0


def _bracket_tol(op, v0, h, xi, side):
    """A tol 1e-7 (relative) above (side 1) or below (side -1) the oracle's
    estimate ratio |d_m| ||w_m|| / ||p_m|| at a degree m of the Newton loop on
    v0 (s = 1, tau = h), and the degree the oracle then stops at.  The ratios
    are not monotone: m is the last degree below the tol-1e-10 one whose ratio
    is a new minimum by 1 %, with the next lower one 1 % below it and none
    within 1 % of it in between."""
    _, ost0 = Nw.phi_apply(op, 1, h, v0, 1e-10, xi=xi)
    assert ost0.s == 1
    alpha, beta = op.gershgorin()
    c, gamma = 0.5 * (alpha + beta), 0.25 * (beta - alpha)
    d = L.divided_differences(1, h, c, gamma, xi[:101])
    w = np.array(v0, dtype=np.float64).reshape(op.shape)
    p = d[0] * w
    ratios = []
    for j in range(ost0.degrees[0] + 20):
        w = op.matvec(w) / gamma - (c / gamma + xi[j]) * w
        p = p + d[j + 1] * w
        ratios.append(abs(d[j + 1]) * np.linalg.norm(w) / np.linalg.norm(p))

    def first_pass(t):
        return next(i + 1 for i, r in enumerate(ratios) if r <= t)

    def clear(k):
        t = ratios[k - 1]
        if k < 3 or not min(ratios[:k - 1]) > 1.01 * t:
            return False
        nxt = first_pass(0.99 * t)
        return all(not (0.99 * t <= r <= 1.01 * t) for r in ratios[k:nxt - 1])

    m = max(k for k in range(3, ost0.degrees[0]) if clear(k))
    tol = ratios[m - 1] * (1.0 + side * 1e-7)
    return tol, (m if side > 0 else first_pass(tol))


@pytest.mark.parametrize("side", [1, -1])
def test_native_bracket_rechecks(env, xi, side):
    """Native FP64 stencil steps after the first bracket ||w|| and ||p|| in FP32
    and take the stop test from the brackets.  A tol 1e-7 from the oracle's
    estimate ratio at a degree m (_bracket_tol) leaves the brackets (about 1e-6
    wide on this grid) undecided there, so the host forms both norms and takes
    the test: converged at m (side 1), or not, going on with the norms formed
    (side -1).  The result, the degree and the substep count must be the
    oracle's."""
    torch, ei = env
    n, dx, D, v0 = _smooth_case()
    op = O.StencilOperator(n, dx, D, (0.0, 0.0, 0.0), bc=(O.NEUMANN0,) * 6)
    h = 1e-2
    tol, expect = _bracket_tol(op, v0, h, xi, side)
    ref, ost = Nw.phi_apply(op, 1, h, v0, tol, xi=xi)
    assert ost.s == 1 and ost.degrees == [expect]
    ctx = stencil_context(torch, ei, n, dx, D, (0.0, 0.0, 0.0), 0.0, (1,) * 6)
    v = dev(torch, v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply(1, h, v, out, tol, {"arith": ei.ARITH_NATIVE_F64})
    assert st.p_rechecks == 1 and st.arith_used == ei.ARITH_NATIVE_F64
    assert rel_err(out.cpu().numpy(), ref) <= FP64_TOL
    _check_stats(st, ost)
    # the same call in float-float forms its norms in every step
    st = ctx.phi_apply(1, h, v, out, tol, {"arith": ei.ARITH_DF})
    assert st.p_rechecks == 0
    assert rel_err(out.cpu().numpy(), ref) <= FP64_TOL
    _check_stats(st, ost)
    ctx.close()


def test_native_brackets_decide(env, xi):
    """At an ordinary tol the brackets decide every test: no recheck, and the
    oracle's result and degree."""
    torch, ei = env
    n, dx, D, v0 = _smooth_case()
    op = O.StencilOperator(n, dx, D, (0.0, 0.0, 0.0), bc=(O.NEUMANN0,) * 6)
    h, tol = 1e-2, 1e-10
    ref, ost = Nw.phi_apply(op, 1, h, v0, tol, xi=xi)
    ctx = stencil_context(torch, ei, n, dx, D, (0.0, 0.0, 0.0), 0.0, (1,) * 6)
    v = dev(torch, v0)
    out = torch.empty_like(v)
    st = ctx.phi_apply(1, h, v, out, tol, {"arith": ei.ARITH_NATIVE_F64, "profile": 1})
    assert st.p_rechecks == 0
    assert st.newton_bounded == st.newton_timed - 1  # all but the first step
    assert rel_err(out.cpu().numpy(), ref) <= FP64_TOL
    _check_stats(st, ost)
    ctx.close()


@pytest.mark.parametrize("arith", [0, 1])
def test_successive_steps_rescaled_operator(env, xi, arith):
    """Successive Rosenbrock steps on one context, native FP64 (one iteration a
    launch) and float-float (two).  The first step
    writes the scaled operator (J - cI)/gamma0; a later step whose gamma stays
    within gamma0 (1 +- 1/8) rewrites only its diagonal and runs the Newton
    loop in the basis w_j / r^j, r = gamma0/gamma; a step outside that range
    rewrites all of it.  States u0 * (1, 1.05, 1.1, 3, 3.1, 1) give r = 1, 0.991,
    0.982, then 1 (rewritten), 0.987, then 1 again.  Each step must give the
    oracle's result, degree and substep count."""
    torch, ei = env
    n = (23, 19, 17)
    shape = tuple(reversed(n))
    dx = (1 / 23,) * 3
    rng = np.random.default_rng(41)
    D = rng.uniform(0.5, 1.5, shape) * 1e-3
    b = tuple(rng.uniform(-1, 1, shape) * 1e-2 for _ in range(3))
    op = O.StencilOperator(n, dx, D, b, bc=(1,) * 6)
    u0 = rng.uniform(0, 1, shape)
    ctx = stencil_context(torch, ei, n, dx, D, b, 0.0, (1,) * 6)
    h, tol = 2.0, 1e-10
    for scale in (1.0, 1.05, 1.1, 3.0, 3.1, 1.0):
        uin = u0 * scale
        ref, ost = Nw.exp_rosenbrock_step(op, uin, h, tol, xi=xi)
        u = dev(torch, uin)
        st = ctx.step(ei.EXP_ROSENBROCK, h, u, ei.NONLIN_LOGISTIC, tol, {"arith": arith})
        got = u.cpu().numpy()
        assert st.arith_used == (ei.ARITH_NATIVE_F64 if arith else ei.ARITH_DF)
        assert rel_err(got - uin, ref - uin) <= FP64_TOL, scale
        _check_stats(st, ost)
    ctx.close()


@pytest.mark.parametrize("method", ["euler", "rosenbrock"])
def test_native_step_reads_u_in_place(env, xi, method):
    """A native FP64 step on a grid whose rows are a multiple of 4 elements
    reads a 16-byte aligned u in place instead of importing it; a u one
    element into a larger buffer (8-byte aligned) is imported.  Both give
    the same bits, and the oracle's step."""
    torch, ei = env
    rng = np.random.default_rng(43)
    n = (40, 24, 20)
    dx = (1 / 40,) * 3
    D, b = _fields_3d(rng, n)
    u0 = rng.uniform(0, 1, (20, 24, 40))
    op = O.StencilOperator(n, dx, D, b, bc=(1,) * 6)
    h, tol = 2e-4, 1e-10
    rosen = method == "rosenbrock"
    if rosen:
        ref, ost = Nw.exp_rosenbrock_step(op, u0, h, tol, xi=xi)
    else:
        ref, ost = Nw.exp_euler_step(op, u0, h, tol, Nw.NONLIN_LOGISTIC, xi=xi)
    ctx = stencil_context(torch, ei, n, dx, D, b, 0.0, (1,) * 6)
    m = ei.EXP_ROSENBROCK if rosen else ei.EXP_EULER
    opts = {"arith": ei.ARITH_NATIVE_F64}
    ctx.step(m, h, dev(torch, u0), ei.NONLIN_LOGISTIC, tol, opts)  # the scaled operator made
    ua = dev(torch, u0)
    assert ua.data_ptr() % 16 == 0
    sa = ctx.step(m, h, ua, ei.NONLIN_LOGISTIC, tol, opts)
    buf = torch.zeros(u0.size + 1, dtype=torch.float64, device=ua.device)
    ub = buf[1:].view(u0.shape)
    ub.copy_(dev(torch, u0))
    assert ub.data_ptr() % 16 == 8
    sb = ctx.step(m, h, ub, ei.NONLIN_LOGISTIC, tol, opts)
    assert torch.equal(ua, ub)
    assert sa.launches == sb.launches - 1  # the import
    got = ua.cpu().numpy()
    assert rel_err(got - u0, ref - u0) <= FP64_TOL
    _check_stats(sa, ost)
    ctx.close()
