"""Benchmark: exponential Rosenbrock-Euler steps of the 3D
advection-diffusion-reaction problem on 256^3 cells (FP64, Neumann,
D(x) = 1 + 0.5 sin sin sin, smooth random b with max |b| = 2, g = u(1-u),
h = 1e-4, Leja tol 1e-10), through the library's C ABI.

A "step" is one call of ei_step: the F = A u + g(u) evaluation, the
Gershgorin interval of J = A + diag(g'(u)), the a-priori schedule and
divided differences on the host, the Newton/Leja loop (one fused kernel per
degree) and the update u += h phi_1(hJ) F.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one rank per GPU) each rank integrates its own replica:
the method has no exchange step on one problem, so the ranks share nothing
but the barrier and the max-over-ranks time ("weak" scaling).
--impl reference times the CPU oracle (the plain numpy/decimal restatement of
the method) on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "adr3d_256_fp64_rosenbrock"
METRIC = "phi1(hA)v steps/s at stated rel err vs FP64 oracle; matvec HBM GB/s vs peak"
N_SIDE = 256
# Newton launch (float-float, explicit coefficients), j > 0, per grid point:
# w read 8 + w' write 8 + p read 8 + p write 8 + 7 coefficients x 8.  The
# two-iteration kernel moves the same 88 bytes per launch for two iterations.
BYTES_PER_POINT = 88
# DRAM bytes per grid point of one launch of the two-iteration float-float
# kernel, from ncu dram__bytes_read.sum + dram__bytes_write.sum on 192^3
# (profiles/launches_adr3d_256_rosenbrock.md, taken on the current kernel);
# traffic scales with the points.
# Valid for the kernel as captured: retake it when the kernel changes.
PAIR_DRAM_BYTES_PER_POINT = 86.9
# DRAM bytes of one launch of the float-float 2-lane complex CSR kernel on the
# 21-spin operator (profiles/k_csr_newton_cg_spin_bath_21.md, the current kernel)
SPIN_DRAM_BYTES_PER_LAUNCH = 1.242e9
# the same for the float-float 2-lane real CSR kernel on the 2^20-node graph
# (profiles/k_csr_newton_g_rgg_2e20.md)
RGG_DRAM_BYTES_PER_LAUNCH = 195.8e6
FLOPS_PER_POINT_PAPER = 10  # the paper's count for (alpha A + beta I)x, Sec. III-A


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    # problem size (grid side, nodes or problem count); --n is kept as an alias
    # (torchrun reads an abbreviated --n as one of its own options: use --size there)
    ap.add_argument("--size", "--n", dest="n", type=int, default=None, help=argparse.SUPPRESS)
    # batch workloads: fixed tile height instead of the autotuner (profiling)
    ap.add_argument("--tile-rows", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--workload", default="adr3d",
                    choices=["adr3d", "adr3d_fp32", "rgg_csr", "batch", "batch_fp32",
                             "adr3d_learned", "adr3d_fp32_learned", "rgg_csr_learned",
                             "batch_learned_fp32", "batch_plain_fp64_loop", "combustion",
                             "combustion_fast", "combustion_nonlin", "heat_dirichlet_data",
                             "heat_dirichlet_hom", "phi2_adr3d", "spin_bath", "spin_bath_fp32"],
                    help="adr3d (default, the headline): 256^3 FP64 Rosenbrock-Euler; "
                         "adr3d_fp32: 512^3 FP32 exponential Euler; rgg_csr: 2^20-node CSR phi_1")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline sample")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------
# CPU oracle: a bounded sample of one step, extrapolated to a full step
# --------------------------------------------------------------------------
def oracle_setup(w):
    from oracle import leja as L
    from oracle import operators as O
    return O.StencilOperator(w.n, w.dx, w.D, w.b, bc=w.bc), L.leja_points(100)


def oracle_step_sample(w, u, op, xi, n_iter=3):
    """Times the oracle's parts of one exponential Rosenbrock-Euler step at the
    full size: F = A u + g(u), the Gershgorin interval of J, the a-priori
    schedule and divided differences, and n_iter Newton iterations.  A full step
    is the setup plus m_sched iterations (the a-priori degree).  Returns
    (seconds per full step, description)."""
    from oracle import leja as L
    from oracle import newton as Nw
    from oracle import operators as O

    t0 = time.perf_counter()
    g, dg = Nw.nonlinearity(u, Nw.NONLIN_LOGISTIC)
    F = op.matvec(u) + g
    J = O.ShiftedOperator(op, dg)
    alpha, beta = J.gershgorin()
    c, gamma = 0.5 * (alpha + beta), 0.25 * (beta - alpha)
    s, m_sched, _ = L.plain_schedule(1, w.h, c, gamma, w.tol, xi)
    d = L.divided_differences(1, w.h / s, c, gamma, xi)
    t1 = time.perf_counter()
    stats = Nw.Stats()
    wv = F.copy()
    p = d[0] * wv
    for j in range(n_iter):
        wv = J.matvec(wv) / gamma - (c / gamma + xi[j]) * wv
        stats.matvecs += 1
        p = p + d[j + 1] * wv
        abs(d[j + 1]) * float(np.sqrt(np.sum(wv * wv))) <= w.tol * float(np.sqrt(np.sum(p * p)))
    t2 = time.perf_counter()
    t_iter = (t2 - t1) / n_iter
    per_step = (t1 - t0) + s * m_sched * t_iter
    desc = (f"oracle (numpy/decimal, 1 thread) at {w.n[0]}^3: F + Gershgorin + schedule + "
            f"divided differences timed in full ({t1 - t0:.2f} s), {n_iter} Newton iterations "
            f"timed ({t_iter:.2f} s each) and scaled to the a-priori count s*m = {s}*{m_sched}")
    return per_step, desc


def run_reference(args):
    """The CPU oracle on bounded samples of the same workload (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1309_4616_gb300 import workloads as W
    w = W.adr_3d(n=args.n if args.n is not None else N_SIDE)
    u = w.u0.copy()
    op, xi = oracle_setup(w)
    for _ in range(args.warmup):
        oracle_step_sample(w, u, op, xi, n_iter=1)
    times = []
    desc = ""
    t_start = time.perf_counter()
    for _ in range(args.steps):
        per_step, desc = oracle_step_sample(w, u, op, xi, n_iter=1)
        times.append(per_step)
    wall = time.perf_counter() - t_start
    est = statistics.mean(times)
    value = 1.0 / est
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": est * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": list(w.n), "h": w.h, "tol": w.tol,
                   "bc": "neumann", "sample_wall_s": wall},
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": 1, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# --------------------------------------------------------------------------
# the GPU arm
# --------------------------------------------------------------------------
class Workload:
    """One benchmark configuration: set-up, one step, its bytes per point."""
    name = ""
    method = ""
    dtype = ""

    def state_reset(self):
        self.state.copy_(self.state0)


class Adr3d(Workload):
    """256^3 (or --n) FP64 exponential Rosenbrock-Euler, Neumann, logistic g."""

    def __init__(self, torch, ei, W, dev, ctx, n):
        self.name, self.method = WORKLOAD, "exp_rosenbrock_euler"
        self.dtype = "f64 (float-float pairs on the FP32 pipes)"
        self.ei, self.w = ei, W.adr_3d(n=n)
        w = self.w
        self.npts = n ** 3
        self.keep = [torch.from_numpy(w.D).to(dev)] + [torch.from_numpy(x).to(dev) for x in w.b]
        ctx.set_operator_stencil(w.n, w.dx, self.keep[0], self.keep[1:], 0.0, list(w.bc),
                                 ei.PREC_F64)
        self.state0 = torch.from_numpy(w.u0).to(dev)
        self.state = self.state0.clone()
        self.host0 = w.u0
        self.bytes_per_point = BYTES_PER_POINT
        self.config = {"grid": [n] * 3, "h": w.h, "tol": w.tol, "bc": "neumann",
                       "method": self.method}

    def step(self, ctx, opts=None):
        return ctx.step(self.ei.EXP_ROSENBROCK, self.w.h, self.state, self.ei.NONLIN_LOGISTIC,
                        self.w.tol, opts)

    def step_host(self, ctx, host, opts=None):
        return ctx.step_host(self.ei.EXP_ROSENBROCK, self.w.h, host, self.ei.NONLIN_LOGISTIC,
                             self.w.tol, opts)

    def kernel(self, fused):
        return ("k_newton2_tma<float-float> (two Newton iterations per launch)"
                if fused == 2 else "k_newton_tma<float-float>")


class Adr3dFp32(Adr3d):
    """512^3 reduced-precision form: FP32 vectors and stencil, exponential Euler."""

    def __init__(self, torch, ei, W, dev, ctx, n):
        self.name, self.method = f"adr3d_{n}_fp32_exp_euler", "exp_euler"
        self.dtype = "f32 (float-float Newton sum)"
        self.ei, self.w = ei, W.adr_3d_fp32(n=n)
        w = self.w
        self.npts = n ** 3
        f32 = torch.float32
        self.keep = [torch.from_numpy(w.D).to(dev, f32)] + \
            [torch.from_numpy(x).to(dev, f32) for x in w.b]
        ctx.set_operator_stencil(w.n, w.dx, self.keep[0], self.keep[1:], 0.0, list(w.bc),
                                 ei.PREC_F32)
        self.state0 = torch.from_numpy(w.u0).to(dev, f32)
        self.state = self.state0.clone()
        self.host0 = w.u0.astype(np.float32)
        # w 4 + w' 4 + p 8+8 + 7 coefficients x 4
        self.bytes_per_point = 52
        self.config = {"grid": [n] * 3, "h": w.h, "tol": w.tol, "bc": "neumann",
                       "method": self.method}

    def step(self, ctx, opts=None):
        return ctx.step(self.ei.EXP_EULER, self.w.h, self.state, self.ei.NONLIN_LOGISTIC,
                        self.w.tol, opts)

    def step_host(self, ctx, host, opts=None):
        return ctx.step_host(self.ei.EXP_EULER, self.w.h, host, self.ei.NONLIN_LOGISTIC,
                             self.w.tol, opts)

    def kernel(self, fused):
        return ("k_newton2_tma<float> (two Newton iterations per launch)"
                if fused == 2 else "k_newton_tma<float>")


class Combustion3d(Adr3d):
    """The combustion model of Sec. III-C with the step of Table 4: 256^3
    interior points, Laplacian, homogeneous Dirichlet, u0 = 1, h = tol = 1e-4;
    exponential Euler (Eq. (2)) with the combustion term fused into the F
    kernel, at full precision (float-float) or with FP32 fast math."""

    fast = False

    def __init__(self, torch, ei, W, dev, ctx, n):
        kind = "fast" if self.fast else "full"
        self.name, self.method = f"combustion_{n}_fp64_exp_euler_{kind}", "exp_euler"
        self.dtype = "f64 (float-float pairs on the FP32 pipes)"
        self.ei, self.w = ei, W.combustion_3d(n=n)
        w = self.w
        self.npts = n ** 3
        self.keep = []
        ctx.set_operator_stencil(w.n, w.dx, w.D, list(w.b), 0.0, list(w.bc), ei.PREC_F64)
        self.state0 = torch.from_numpy(w.u0).to(dev)
        self.state = self.state0.clone()
        self.host0 = w.u0
        self.bytes_per_point = BYTES_PER_POINT
        self.nonlin = ei.NONLIN_COMBUSTION_FAST if self.fast else ei.NONLIN_COMBUSTION
        self.config = {"grid": [n] * 3, "h": w.h, "tol": w.tol, "bc": "dirichlet0",
                       "method": self.method, "u0": 1.0,
                       "nonlinearity": "combustion (2-u) e^{20(1-1/u)}/4, " +
                       ("FP32 __expf/__fdividef" if self.fast else "float-float")}

    def step(self, ctx, opts=None):
        return ctx.step(self.ei.EXP_EULER, self.w.h, self.state, self.nonlin, self.w.tol, opts)

    def step_host(self, ctx, host, opts=None):
        return ctx.step_host(self.ei.EXP_EULER, self.w.h, host, self.nonlin, self.w.tol, opts)


class Combustion3dFast(Combustion3d):
    fast = True


class HeatDirichlet(Adr3d):
    """The boundary conditions of Sec. III-A on the Table 4 grid: u_t = Laplace(u)
    on 256^3 interior points (dx = 1/257), Dirichlet faces,
    u0 = sin(pi x) sin(pi y) sin(pi z), one exponential Euler step
    (h = tol = 1e-4).  With data: the paper's boundary
    function sin(pi z) exp(-xy) on all six faces (ei_set_dirichlet_values);
    without: homogeneous."""

    data = True

    def __init__(self, torch, ei, W, dev, ctx, n):
        kind = "sin(pi z)exp(-xy)" if self.data else "homogeneous"
        self.name = f"heat_{n}_dirichlet_{'data' if self.data else 'hom'}_exp_euler"
        self.method = "exp_euler"
        self.dtype = "f64 (float-float pairs on the FP32 pipes)"
        self.ei, self.w = ei, W.combustion_3d(n=n)
        w = self.w
        self.npts = n ** 3
        self.keep = []
        ctx.set_operator_stencil(w.n, w.dx, 1.0, [0.0, 0.0, 0.0], 0.0, list(w.bc), ei.PREC_F64)
        if self.data:
            ax = np.arange(1, n + 1) / (n + 1)
            P, Q = np.meshgrid(ax, ax, indexing="ij")  # [slow, fast]
            f = lambda x, y, z: np.sin(np.pi * z) * np.exp(-x * y)
            faces = [f(0 * P, Q, P), f(1 + 0 * P, Q, P), f(Q, 0 * P, P), f(Q, 1 + 0 * P, P),
                     f(Q, P, 0 * P), f(Q, P, 1 + 0 * P)]
            self.keep = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in faces]
            ctx.set_dirichlet_values(self.keep)
        s1 = np.sin(np.pi * np.arange(1, n + 1) / (n + 1))
        u0 = s1[:, None, None] * s1[None, :, None] * s1[None, None, :]
        self.state0 = torch.from_numpy(u0).to(dev)
        self.state = self.state0.clone()
        self.host0 = u0
        self.bytes_per_point = BYTES_PER_POINT
        self.config = {"grid": [n] * 3, "h": w.h, "tol": w.tol, "bc": "dirichlet",
                       "boundary_data": kind, "method": self.method,
                       "u0": "sin(pi x) sin(pi y) sin(pi z)"}

    def step(self, ctx, opts=None):
        return ctx.step(self.ei.EXP_EULER, self.w.h, self.state, self.ei.NONLIN_NONE, self.w.tol,
                        opts)

    def step_host(self, ctx, host, opts=None):
        return ctx.step_host(self.ei.EXP_EULER, self.w.h, host, self.ei.NONLIN_NONE, self.w.tol,
                             opts)


class HeatDirichletHom(HeatDirichlet):
    data = False


class NonlinStats:
    """ei_stats-like record of one pointwise evaluation."""

    def __init__(self, ms=0.0, timed=0):
        self.launches = 1
        self.matvecs = 0
        self.newton_ms = ms
        self.newton_timed = timed
        self.newton_fused = 1

    def degree_list(self):
        return []


class NonlinEval(Workload):
    """Table 3 of the paper: one evaluation of the combustion term g(u) of
    Sec. III-C at every point of an n^3 grid (u ~ U[1, 2]), FP64 arrays
    evaluated in float-float (ei_nonlinearity).  The other variants (native
    FP64, FP32, and FP32 fast math on FP64 and FP32 arrays) are timed once at
    set-up and listed in the config."""

    def __init__(self, torch, ei, W, dev, ctx, n):
        self.name, self.method = f"combustion_nonlinearity_{n}", "g(u) pointwise"
        self.dtype = "f64 (float-float on the FP32 pipes)"
        self.ei, self.torch = ei, torch
        u = W.combustion_field(n)
        self.npts = n ** 3
        self.host0 = u
        self.state0 = torch.from_numpy(u).to(dev)
        self.state = self.state0.clone()
        self.g = torch.empty_like(self.state)
        self.stream = ctx.stream
        # read u 8 + write g 8
        self.bytes_per_point = 16
        u32 = self.state.to(torch.float32)
        g32 = torch.empty_like(u32)
        variants = {
            "f64_float_float": (ei.NONLIN_COMBUSTION, self.state, self.g, ei.ARITH_DF),
            "f64_native": (ei.NONLIN_COMBUSTION, self.state, self.g, ei.ARITH_NATIVE_F64),
            "f64_fast_math": (ei.NONLIN_COMBUSTION_FAST, self.state, self.g, ei.ARITH_DF),
            "f32_full": (ei.NONLIN_COMBUSTION, u32, g32, ei.ARITH_DF),
            "f32_fast_math": (ei.NONLIN_COMBUSTION_FAST, u32, g32, ei.ARITH_DF),
        }
        ms = {}
        for name, (kind, uu, gg, ar) in variants.items():
            ms[name] = round(self._time(kind, uu, gg, ar), 4)
        self.config = {"grid": [n] * 3, "u": "uniform [1, 2]", "variants_ms": ms,
                       "l2_note": "one evaluation reads u and writes g once"}

    def _run(self, kind, u, g, arith):
        self.ei.nonlinearity(kind, u, g, None, arith=arith, stream=self.stream)

    def _time(self, kind, u, g, arith, reps=10):
        torch = self.torch
        for _ in range(3):
            self._run(kind, u, g, arith)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        for _ in range(reps):
            self._run(kind, u, g, arith)
        e1.record(self.stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    def step(self, ctx, opts=None):
        if opts and opts.get("profile"):
            return NonlinStats(self._time(self.ei.NONLIN_COMBUSTION, self.state, self.g,
                                          self.ei.ARITH_DF, reps=1), 1)
        self._run(self.ei.NONLIN_COMBUSTION, self.state, self.g, self.ei.ARITH_DF)
        return NonlinStats()

    def step_host(self, ctx, host, opts=None):
        d = host.to(self.state.device, non_blocking=True)
        self._run(self.ei.NONLIN_COMBUSTION, d, self.g, self.ei.ARITH_DF)
        pinned_like(self, host).copy_(self.g, non_blocking=False)
        return NonlinStats()

    def kernel(self, fused):
        return "k_nonlin_eval<float-float> (combustion g(u), Table 3)"


class RggCsr(Workload):
    """phi_1(hA)v for A = -(graph Laplacian) of the 2^20-node random geometric
    graph, h*rho(A) = 100, tol 1e-10, FP64."""

    def __init__(self, torch, ei, W, dev, ctx, n):
        self.name, self.method = "rgg_2^20_csr_phi1", "phi1"
        self.dtype = "f64 (float-float pairs on the FP32 pipes)"
        self.ei = ei
        g = W.rgg_graph(n=n)
        self.npts = g.n
        self.keep = [torch.from_numpy(g.rowptr).to(dev), torch.from_numpy(g.col).to(dev),
                     torch.from_numpy(g.val).to(dev), torch.from_numpy(-g.deg_w).to(dev)]
        ctx.set_operator_csr(g.n, *self.keep)
        self.h = 100.0 / (2.0 * g.deg_w.max())
        self.tol = 1e-10
        v = W.random_vector(g.n, 5)
        self.host0 = v
        self.state0 = torch.from_numpy(v).to(dev)
        self.state = self.state0.clone()
        self.out = torch.empty_like(self.state)
        nnz = g.col.size
        # val 8 + col 4 per entry, rowptr 8 + diag 8 + w 8 + w' 8 + p 16 per row
        self.bytes_per_point = 12.0 * nnz / g.n + 48.0
        self.config = {"nodes": g.n, "nnz": int(nnz), "mean_degree": nnz / g.n,
                       "h_rho": 100.0, "tol": self.tol, "method": self.method}
        self.traffic_per_launch = RGG_DRAM_BYTES_PER_LAUNCH if n == 1 << 20 else None

    def step(self, ctx, opts=None):
        return ctx.phi_apply(1, self.h, self.state, self.out, self.tol, opts)

    def step_host(self, ctx, host, opts=None):
        # phi_1(hA)v of the same v every call: the result goes to its own buffer
        d = host.to(self.state.device, non_blocking=True)
        st = ctx.phi_apply(1, self.h, d, self.out, self.tol, opts)
        pinned_like(self, host).copy_(self.out, non_blocking=False)
        return st

    def kernel(self, fused):
        return "k_csr_newton_g<float-float, 2 lanes a row> (32 rows a warp in 2 rounds)"


class PhiKAdr3d(Adr3d):
    """phi_2(hA)v on the 256^3 advection-diffusion operator of the headline
    workload, h = 5e-4 (h rho ~ 600: the a-priori rule takes several substeps,
    each an e^{tau A} run on the state and a psi run on v), tol 1e-10, FP64."""

    k = 2

    def __init__(self, torch, ei, W, dev, ctx, n):
        Adr3d.__init__(self, torch, ei, W, dev, ctx, n)
        self.name, self.method = f"adr3d_{n}_phi{self.k}_substeps", f"phi_{self.k}(hA)v"
        self.h = 5e-4
        self.out = torch.empty_like(self.state)
        self.config = {"grid": [n] * 3, "h": self.h, "tol": self.w.tol, "k": self.k,
                       "bc": "neumann", "method": self.method}

    def step(self, ctx, opts=None):
        return ctx.phi_apply(self.k, self.h, self.state, self.out, self.w.tol, opts)

    def step_host(self, ctx, host, opts=None):
        d = host.to(self.state.device, non_blocking=True)
        st = ctx.phi_apply(self.k, self.h, d, self.out, self.w.tol, opts)
        pinned_like(self, host).copy_(self.out, non_blocking=False)
        return st


class SpinBath(Workload):
    """e^{-i t H} psi for the spin-bath Hamiltonian of Sec. III-D (two central
    spins and a bath, 21 spins: 2^21 complex states, 40 entries a row),
    t = 10, tol 1e-5: Table 5's integration as one propagation call, FP64."""
    prec = 0

    def __init__(self, torch, ei, W, dev, ctx, n):
        single = self.prec == 1
        self.name = f"spin_bath_{n}_propagator" + ("_fp32" if single else "")
        self.method = "exp(-i t H) psi"
        self.dtype = ("f32 (Newton sum float-float)" if single
                      else "f64 (float-float pairs on the FP32 pipes)")
        g = W.spin_bath(n)
        self.npts = g.n
        dt = torch.float32 if single else torch.float64
        self.keep = [torch.from_numpy(g.rowptr).to(dev), torch.from_numpy(g.col).to(dev),
                     torch.from_numpy(g.val).to(dt).to(dev), torch.from_numpy(g.diag).to(dt).to(dev)]
        ctx.set_operator_csr(g.n, *self.keep, prec=self.prec)
        self.h, self.tol = 10.0, 1e-5
        v = W.spin_state(g.n, 5)
        if single:
            v = v.astype(np.complex64)
        self.host0 = v
        self.state0 = torch.from_numpy(v).to(dev)
        self.state = self.state0.clone()
        self.out = torch.empty_like(self.state)
        nnz = g.col.size
        # per row: val + col per entry, rowptr 8, diagonal, w in + w out, p read + write
        ev = 4 if single else 8
        self.bytes_per_point = (ev + 4.0) * nnz / g.n + 8 + ev + 4 * ev + 32
        self.config = {"spins": n, "states": g.n, "nnz_offdiag": int(nnz),
                       "entries_per_row": nnz / g.n + 1, "t": self.h, "tol": self.tol,
                       "method": self.method}

        self.traffic_per_launch = SPIN_DRAM_BYTES_PER_LAUNCH if (n == 21 and not single) else None

    def step(self, ctx, opts=None):
        return ctx.phi_apply_imag(0, self.h, self.state, self.out, self.tol, opts)

    def step_host(self, ctx, host, opts=None):
        d = host.to(self.state.device, non_blocking=True)
        st = ctx.phi_apply_imag(0, self.h, d, self.out, self.tol, opts)
        pinned_like(self, host).copy_(self.out, non_blocking=False)
        return st

    def kernel(self, fused):
        fmt = "float" if self.prec == 1 else "float-float"
        return (f"k_csr_newton_cg<{fmt}, 2 lanes a row> (complex w and p interleaved, "
                f"real H)")


class SpinBathFp32(SpinBath):
    prec = 1


TILE_ROWS = 0


def pinned_like(wl, host):
    """A pinned host buffer shaped like `host`, kept on the workload: where a
    pass maps v to a separate output, the e2e read-back lands there."""
    buf = getattr(wl, "_host_out", None)
    if buf is None or buf.shape != host.shape or buf.dtype != host.dtype:
        import torch
        buf = torch.empty(host.shape, dtype=host.dtype).pin_memory()
        wl._host_out = buf
    return buf


class Batch2d(Workload):
    """1024 independent 2D advection-diffusion problems (sides log-uniform in
    [32, 512], per-side Dirichlet/Neumann, constant D, b, h), all phi_1(h A) v in
    one persistent launch replayed from a CUDA graph.  A step is one pass of the
    whole batch."""

    prec = 0

    def __init__(self, torch, ei, W, dev, ctx, n, learned_opt=False):
        self.name = "batch_1024_2d" + ("_fp32" if self.prec else "_fp64")
        self.method = "phi1 (batched, persistent kernel)"
        self.dtype = "f32 (float-float Newton sum)" if self.prec else \
            "f64 (float-float pairs on the FP32 pipes)"
        self.ei = ei
        probs = W.batch_2d(count=n)
        self.tol = 1e-6 if self.prec else 1e-10
        t0 = time.perf_counter()
        opts = {"tile_rows": TILE_ROWS} if TILE_ROWS else {}
        if learned_opt:
            opts["learned"] = 1  # plans come from the network at each pass
        self.batch = ei.Batch(probs, prec=self.prec, tol=self.tol, options=opts or None)
        self.setup_s = time.perf_counter() - t0
        dt = torch.float32 if self.prec else torch.float64
        flat = np.concatenate([p.v.ravel() for p in probs])
        self.host0 = flat.astype(np.float32) if self.prec else flat
        self.state0 = torch.from_numpy(self.host0).to(dev)
        self.state = self.state0.clone()
        self.out = torch.empty_like(self.state)
        self.npts = int(flat.size)
        self.probs = probs
        self.bytes_per_point = 32  # per point-iteration: w 8 + w' 8 + p 8+8 (constant coefficients)
        self.config = {"problems": len(probs), "points": self.npts, "tol": self.tol,
                       "method": self.method, "setup_s": self.setup_s}

    def step(self, ctx, opts=None):
        st = self.batch.phi1(self.state, self.out)
        if "strip_rows" not in self.config:
            self.config["strip_rows"] = sorted({int(x.tile_rows) for x in st})
        return BatchStepStats(st, self.probs)

    def step_host(self, ctx, host):
        # phi_1(hA)v of the same v every pass: the result goes to its own
        # pinned buffer, not back into the input
        d = host.to(self.state.device, non_blocking=True)
        st = self.batch.phi1(d, self.out)
        pinned_like(self, host).copy_(self.out, non_blocking=False)
        return BatchStepStats(st, self.probs)

    def kernel(self, fused):
        return "k_batch (persistent, device work queue)"


class Batch2dFp32(Batch2d):
    prec = 1


class Batch2dLearnedFp32(Batch2d):
    """The learned + FP32 + batched form: the 1024 problems in FP32 (tol 1e-6),
    one persistent launch per pass, every problem's substep count from the
    committed schedule network (adaptive; the a-priori rule where a proposal
    reaches m_max).  The plan is made inside every pass."""

    prec = 1

    def __init__(self, torch, ei, W, dev, ctx, n):
        from paper_1309_4616_gb300 import learned
        self.model = learned.load()
        Batch2d.__init__(self, torch, ei, W, dev, ctx, n, learned_opt=True)
        self.batch.set_schedule_model(self.model)
        self.name = "batch_1024_2d_fp32_learned"
        self.method = "phi1 (batched, persistent kernel, learned schedule)"
        self.config["schedule"] = "learned (network proposal, a posteriori stop)"


class Batch2dPlainLoop(Workload):
    """The plain FP64 GPU method on the same 1024 problems: one context per
    problem, ei_phi_apply with the a-priori schedule, one problem after the
    other (tol 1e-6, the accuracy the FP32 form states).  A step is one pass
    over all problems."""

    def __init__(self, torch, ei, W, dev, ctx, n):
        self.name = "batch_1024_2d_fp64_plain_loop"
        self.method = "phi1 (one ei_phi_apply per problem, a-priori schedule)"
        self.dtype = "f64 (float-float pairs on the FP32 pipes)"
        self.ei = ei
        probs = W.batch_2d(count=n)
        self.tol = 1e-6
        t0 = time.perf_counter()
        self.ctxs = []
        for p in probs:
            c = ei.Context(ctx.device, ctx.stream)
            c.set_operator_stencil(p.n, p.dx, float(p.D), [float(x) for x in p.b], 0.0,
                                   list(p.bc), ei.PREC_F64)
            self.ctxs.append(c)
        self.setup_s = time.perf_counter() - t0
        flat = np.concatenate([p.v.ravel() for p in probs])
        self.offsets = np.concatenate([[0], np.cumsum([p.v.size for p in probs])])
        self.host0 = flat
        self.state0 = torch.from_numpy(flat).to(dev)
        self.state = self.state0.clone()
        self.out = torch.empty_like(self.state)
        self.npts = int(flat.size)
        self.probs = probs
        self.bytes_per_point = 72  # 2D explicit coefficients: w 8 + w' 8 + p 16 + 5 x 8
        self.config = {"problems": len(probs), "points": self.npts, "tol": self.tol,
                       "method": self.method, "setup_s": self.setup_s}

    def _run(self, v, opts):
        agg = LoopStepStats()
        for i, (c, p) in enumerate(zip(self.ctxs, self.probs)):
            a, b = int(self.offsets[i]), int(self.offsets[i + 1])
            st = c.phi_apply(1, p.h, v[a:b], self.out[a:b], self.tol, opts)
            agg.add(st, self.bytes_per_point * (b - a))
        return agg

    def step(self, ctx, opts=None):
        return self._run(self.state, opts)

    def step_host(self, ctx, host, opts=None):
        d = host.to(self.state.device, non_blocking=True)
        st = self._run(d, opts)
        pinned_like(self, host).copy_(self.out, non_blocking=False)
        return st

    def kernel(self, fused):
        return "k_newton2_tma<float-float> (per-problem launches)"


class LoopStepStats:
    """ei_stats-like sum over the calls of one pass."""

    def __init__(self):
        self.launches = self.matvecs = self.newton_timed = 0
        self.newton_ms = 0.0
        self.newton_fused = 1
        self.timed_bytes = 0.0
        self._degs = []

    def add(self, st, bytes_per_iteration_sweep):
        self.launches += st.launches
        self.matvecs += st.matvecs
        self.newton_timed += st.newton_timed
        self.newton_ms += st.newton_ms
        self.newton_fused = st.newton_fused or 1
        self.timed_bytes += bytes_per_iteration_sweep * st.newton_fused * st.newton_timed
        if len(self._degs) < 3:
            self._degs.append(int(st.degree_sum))

    def degree_list(self):
        return self._degs


class BatchStepStats:
    """ei_stats-like view of a batch pass."""

    def __init__(self, st, probs):
        self.launches = 5
        self.matvecs = int(sum(s.degree_sum + s.s - 1 for s in st))
        self.point_iters = int(sum((s.degree_sum + s.s) * p.n[0] * p.n[1]
                                   for s, p in zip(st, probs)))
        self.newton_ms = 0.0
        self.newton_timed = 0
        self.newton_fused = 1
        self.learned = 1 if any(s.learned == 1 for s in st) else 0
        self.learned_kept = sum(1 for s in st if s.learned == 1)
        self._st = st

    def degree_list(self):
        return [int(s.degree_sum) for s in self._st[:3]]


class Learned:
    """The same workload with phi_1 under the learned schedule: the committed
    network (paper_1309_4616_gb300/schedule_mlp.npz) proposes s and m, the a
    posteriori estimate accepts or rejects, the plain method is the fallback."""

    def setup_learned(self, ctx):
        from paper_1309_4616_gb300 import learned
        self.model = learned.load()
        ctx.set_schedule_model(self.model)
        self.name += "_learned"
        self.method += " (learned schedule)"
        self.config["schedule"] = "learned (network proposal, a posteriori check)"

    @staticmethod
    def _opts(opts):
        o = {"learned": 1}
        o.update(opts or {})
        return o

    def step(self, ctx, opts=None):
        return super().step(ctx, self._opts(opts))

    def step_host(self, ctx, host, opts=None):
        return super().step_host(ctx, host, self._opts(opts))


class Adr3dLearned(Learned, Adr3d):
    def __init__(self, torch, ei, W, dev, ctx, n):
        Adr3d.__init__(self, torch, ei, W, dev, ctx, n)
        self.setup_learned(ctx)


class Adr3dFp32Learned(Learned, Adr3dFp32):
    def __init__(self, torch, ei, W, dev, ctx, n):
        Adr3dFp32.__init__(self, torch, ei, W, dev, ctx, n)
        self.setup_learned(ctx)


class RggCsrLearned(Learned, RggCsr):
    def __init__(self, torch, ei, W, dev, ctx, n):
        RggCsr.__init__(self, torch, ei, W, dev, ctx, n)
        self.setup_learned(ctx)


WORKLOADS = {"adr3d": Adr3d, "adr3d_fp32": Adr3dFp32, "rgg_csr": RggCsr, "batch": Batch2d,
             "batch_fp32": Batch2dFp32, "adr3d_learned": Adr3dLearned,
             "adr3d_fp32_learned": Adr3dFp32Learned, "rgg_csr_learned": RggCsrLearned,
             "batch_learned_fp32": Batch2dLearnedFp32, "batch_plain_fp64_loop": Batch2dPlainLoop,
             "combustion": Combustion3d, "combustion_fast": Combustion3dFast,
             "combustion_nonlin": NonlinEval, "heat_dirichlet_data": HeatDirichlet,
             "heat_dirichlet_hom": HeatDirichletHom, "phi2_adr3d": PhiKAdr3d,
             "spin_bath": SpinBath, "spin_bath_fp32": SpinBathFp32}
DEFAULT_N = {"adr3d": N_SIDE, "adr3d_fp32": 512, "rgg_csr": 1 << 20, "batch": 1024,
             "batch_fp32": 1024, "adr3d_learned": N_SIDE, "adr3d_fp32_learned": 512,
             "rgg_csr_learned": 1 << 20, "batch_learned_fp32": 1024,
             "batch_plain_fp64_loop": 1024, "combustion": N_SIDE, "combustion_fast": N_SIDE,
             "combustion_nonlin": N_SIDE, "heat_dirichlet_data": N_SIDE,
             "heat_dirichlet_hom": N_SIDE, "phi2_adr3d": N_SIDE, "spin_bath": 21,
             "spin_bath_fp32": 21}


def replica_group(world, backend):
    """The process group of N replicas (None for one process).  Ranks share no
    data: only a barrier and the slowest replica's times."""
    if world <= 1:
        return None
    import torch.distributed as dist
    dist.init_process_group(backend)
    return dist


def max_over_ranks(value, dist, device):
    """The largest value over all ranks (every rank receives it)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args):
    import torch
    from paper_1309_4616_gb300 import build, ei
    from paper_1309_4616_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = replica_group(world, "nccl")
    if rank == 0 or world == 1:
        build.build()
    if dist is not None:
        dist.barrier()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    ctx = ei.Context(local, stream)
    global TILE_ROWS
    TILE_ROWS = args.tile_rows
    n = args.n if args.n is not None else DEFAULT_N[args.workload]
    wl = WORKLOADS[args.workload](torch, ei, W, dev, ctx, n)
    npts = wl.npts

    # warm-up on a copy, then the timed steps from the initial state
    for _ in range(args.warmup):
        wl.step(ctx)
    wl.state_reset()
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches = 0
    matvecs = []
    degrees = []
    learned_flags = []
    learned_kept = None
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(args.steps):
        st = wl.step(ctx)
        launches += st.launches
        matvecs.append(st.matvecs)
        degrees.append(st.degree_list())
        learned_flags.append(int(getattr(st, "learned", 0)))
        if hasattr(st, "learned_kept"):
            learned_kept = st.learned_kept
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    if dist is not None:
        dist.barrier()

    # roofline of the dominant kernel: per-launch CUDA events around every Newton
    # launch of two further steps (profile option), same stream, same sizes
    wl.state_reset()
    prof_ms, prof_n, fused, prof_bytes = 0.0, 0, 1, 0.0
    for _ in range(2):
        st = wl.step(ctx, {"profile": 1})
        prof_ms += st.newton_ms
        prof_n += st.newton_timed
        fused = st.newton_fused
        prof_bytes += getattr(st, "timed_bytes", 0.0)
    hbm, peak_kind = peaks()
    if prof_n == 0 and hasattr(st, "point_iters"):
        # batched pass: one persistent launch; algorithmic bytes of all its sweeps
        # over the measured time per pass
        avg_launch_s = ms * 1e-3 / args.steps
        achieved = wl.bytes_per_point * st.point_iters / avg_launch_s / 1e9
    elif hasattr(st, "timed_bytes"):
        # many problems, one launch sequence each: bytes of all timed launches
        # over their summed time
        avg_launch_s = prof_ms / max(prof_n, 1) * 1e-3
        achieved = prof_bytes / max(prof_ms * 1e-3, 1e-12) / 1e9
    else:
        # unit: one point-iteration; a two-iteration launch processes two per point
        # (its DRAM traffic is about half of that: w_{j+1} stays on chip)
        avg_launch_s = prof_ms / max(prof_n, 1) * 1e-3
        achieved = wl.bytes_per_point * npts * fused / avg_launch_s / 1e9

    # e2e through the public API with host buffers: H2D of the state, the step, D2H
    u_host = torch.from_numpy(np.ascontiguousarray(wl.host0).copy()).pin_memory()
    k_e2e = max(1, min(args.steps, 10))
    wl.step_host(ctx, u_host)  # warm
    u_host.copy_(torch.from_numpy(np.ascontiguousarray(wl.host0)))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        wl.step_host(ctx, u_host)
    torch.cuda.synchronize(dev)
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)

    cpu = None
    if rank == 0 and not args.no_cpu and args.workload == "adr3d":
        op, xi = oracle_setup(wl.w)
        per_step, desc = oracle_step_sample(wl.w, wl.w.u0.copy(), op, xi)
        cpu = {"value": 1.0 / per_step, "unit": "steps/s", "cores": 1, "kind": "oracle",
               "sample": desc}

    if rank == 0:
        steps_total = args.steps * world
        value = steps_total / (ms * 1e-3)
        esz = u_host.element_size()
        config = {"workload": wl.name, **wl.config, "parallelism": f"replicas x{world}",
                  "l2": "inputs larger than L2 (each vector >= 8 MB and the step's working "
                        "set >= 0.3 GB; 256^3: 134 MB per vector)",
                  "matvecs_per_step": matvecs, "degrees": degrees[:3]}
        if learned_kept is not None and getattr(wl, "model", None) is not None:
            config["learned_problems_kept_per_pass"] = learned_kept
        elif any(learned_flags):
            config["learned_accepted_steps"] = sum(1 for f in learned_flags if f == 1)
        line = {
            "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": wl.dtype, "data": "synthetic", "config": config,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm,
                         "traffic": (PAIR_DRAM_BYTES_PER_POINT * npts
                                     if isinstance(wl, Adr3d) and fused == 2
                                     else getattr(wl, "traffic_per_launch", None)),
                         "kernel": wl.kernel(fused),
                         "bytes_per_launch": (prof_bytes / max(prof_n, 1)) if prof_bytes
                         else wl.bytes_per_point * npts * fused,
                         "avg_launch_us": avg_launch_s * 1e6, "launches_timed": prof_n,
                         "iterations_per_launch": fused,
                         "us_per_iteration": avg_launch_s * 1e6 / fused,
                         "peak_kind": peak_kind,
                         "paper_gflops": FLOPS_PER_POINT_PAPER * npts * fused / avg_launch_s / 1e9},
            "cpu_baseline": cpu,
            "e2e": {"value": k_e2e * world / e2e_s, "unit": "steps/s",
                    "h2d_bytes_per_step": npts * esz, "d2h_bytes_per_step": npts * esz},
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line))
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
