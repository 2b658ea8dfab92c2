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
DTYPE_FF = "float-float (FP32 pairs: 48-bit significand, FP32 exponent range)"
# Newton launch (explicit coefficients, 8-byte formats), j > 0, per grid point
# as stored: w read 8 + w' write 8 + p read 8 + p write 8 + 7 coefficients x 8.
# The two-iteration kernel moves the same 88 bytes per launch for two iterations.
BYTES_PER_POINT = 88
# Algorithmic bytes per point-iteration of the 256^3 workload as its scope
# table counts them: w read 8, w' write 8, p read and write 16, and the operator
# as its inputs (D 8, b 24, u_n for g' 8).  The library stores the seven
# coefficients instead (BYTES_PER_POINT).
ALG_BYTES_PER_POINT = 72
# the same for a constant-coefficient operator (w 8, w' 8, p 16)
CONST_BYTES_PER_POINT = 32
# FP64 flops of one Newton iteration per grid point (a fused multiply-add counts
# two), on the scaled operator (A - cI)/gamma the native kernel iterates with:
# the 7-point product (7 multiplies, 6 adds), the shift -xi_j w (1 multiply, 1
# add), the Newton sum (1 multiply, 1 add) and the two squared norms
# (2 multiplies, 2 adds).
FP64_FLOPS_PER_POINT = 21
# the same for an iteration in bracket mode (every step after the first of a
# native loop): both squared norms bracketed by FP32 arithmetic on integer-cut
# values instead of formed in FP64
FP64_FLOPS_PER_POINT_BOUNDED = 17
# GB300's FP64 peak from unit counts and clocks: the nominal 1.25 TFLOP/s over
# 152 SMs at 2070 MHz is 4 FP64 flops (two FMA lanes) per SM and clock.
SMS, FP64_FLOPS_PER_SM_CLK = 152, 4
# DRAM bytes per grid point of one launch of the two-iteration float-float
# kernel on the scaled operator, from ncu dram__bytes_read.sum +
# dram__bytes_write.sum over every working launch of the 256^3 bench step
# (profiles/dram_bytes_newton_kernels_256cube.md).
# Valid for the kernel as captured: retake it when the kernel changes.
PAIR_DRAM_BYTES_PER_POINT = 87.6
# the same for one launch of the native-FP64 one-iteration kernel on the scaled
# operator (a bracket step), from the same capture
NATIVE_DRAM_BYTES_PER_POINT = 96.1
# the float-float pair kernel on a constant operator's coefficient table (no
# coefficient arrays), per point and launch: ncu dram__bytes_read.sum +
# dram__bytes_write.sum over the 49 working launches of the 256^3 combustion
# step (profiles/k_newton2_tma_table_combustion_192cube.md; 28.6 B a launch
# that reads p, 20.5 a loop's first, part of w and p staying in L2)
TABLE_PAIR_DRAM_BYTES_PER_POINT = 27.8
# DRAM bytes of one launch of the float-float sliced complex CSR kernel on the
# 21-spin operator (profiles/k_csr_newton_sell_c_spin_bath_21.md)
SPIN_DRAM_BYTES_PER_LAUNCH = 1.237e9
# the same for the sliced real CSR kernel on the 2^20-node graph, float-float
# and native FP64 (profiles/k_csr_newton_sell_rgg_2e20.md)
RGG_DRAM_BYTES_PER_LAUNCH = 228.2e6
RGG_DRAM_BYTES_PER_LAUNCH_F64 = 227.7e6
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
                    choices=["adr3d", "adr3d_ff", "adr3d_fp32", "rgg_csr", "adv_diff_2d", "batch",
                             "batch_ff", "batch_fp32",
                             "adr3d_learned", "adr3d_fp32_learned", "rgg_csr_learned",
                             "batch_learned_fp32", "batch_plain_fp64_loop", "combustion",
                             "combustion_fast", "combustion_nonlin", "heat_dirichlet_data",
                             "heat_dirichlet_hom", "phi2_adr3d", "spin_bath", "spin_bath_fp32",
                             "batch_vs_plain_loop"],
                    help="adr3d (default, the headline): 256^3 FP64 Rosenbrock-Euler; "
                         "adr3d_fp32: 512^3 FP32 exponential Euler; rgg_csr: 2^20-node CSR phi_1")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline sample")
    return ap.parse_args()


def peaks_sm_mhz():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"])
    except Exception:
        return 2070.0


# GB300's nominal HBM3e bandwidth (GB/s), reported beside the measured copy rate
HBM_NOMINAL_GBS = 7900.0


def with_nominal(d):
    """An HBM roofline object with its fraction of the nominal bandwidth added."""
    if d.get("unit") == "GB/s":
        d["nominal_peak"] = HBM_NOMINAL_GBS
        d["frac_nominal"] = d["achieved"] / HBM_NOMINAL_GBS
    return d


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
# the reference arm: the oracle on the host cores
# --------------------------------------------------------------------------
REF_BUDGET_S = 150.0   # timed whole steps of the reference arm stop here


def run_reference(args):
    """The CPU oracle (rank 0 only) on the same workload and trajectory: whole
    exponential Rosenbrock-Euler steps from u0 with the oracle's step split
    over all host cores (oracle/slab.py; equal to the serial oracle up to the
    norms' summation order).  One untimed warm-up step; then K timed whole
    steps, or as many as fit in REF_BUDGET_S (at least one), stated in the
    line."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import leja as L
    from oracle import slab as S
    from paper_1309_4616_gb300 import workloads as W
    w = W.adr_3d(n=args.n if args.n is not None else N_SIDE)
    xi = L.leja_points(100)
    sop = S.SlabStencil(w.n, w.dx, w.D, w.b, bc=w.bc)
    u = w.u0.copy()
    t_warm = 0.0
    if args.warmup > 0:
        t0 = time.perf_counter()
        S.exp_rosenbrock_step(sop, u, w.h, w.tol, xi=xi)
        t_warm = time.perf_counter() - t0
    times = []
    t_start = time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        u, st = S.exp_rosenbrock_step(sop, u, w.h, w.tol, xi=xi)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start + statistics.mean(times) > REF_BUDGET_S:
            break
    wall = time.perf_counter() - t_start
    sop.close()
    k = len(times)
    per_step = sum(times) / k
    value = 1.0 / per_step
    cores = S.host_threads()
    desc = (f"{k} whole steps of the {w.n[0]}^3 exponential Rosenbrock-Euler trajectory from "
            f"u0 timed in full ({sum(times):.1f} s), oracle split in z-slabs over {cores} host "
            f"threads; 1 untimed warm-up step ({t_warm:.1f} s)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s",
        "n_gpus": args.gpus, "steps": k, "warmup": min(args.warmup, 1),
        "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": list(w.n), "h": w.h, "tol": w.tol,
                   "bc": "neumann", "steps_requested": args.steps,
                   "warmup_requested": args.warmup, "timed_wall_s": wall,
                   "nproc": os.cpu_count()},
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": cores, "kind": "oracle",
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
    """256^3 (or --n) FP64 exponential Rosenbrock-Euler, Neumann, logistic g, in
    native IEEE double arithmetic (arith = 1).  arith = 0 runs the same step in
    the float-float format on the FP32 pipes."""

    arith = 1

    def __init__(self, torch, ei, W, dev, ctx, n):
        self.name, self.method = WORKLOAD, "exp_rosenbrock_euler"
        self.ei, self.w = ei, W.adr_3d(n=n)
        w = self.w
        self.npts = n ** 3
        self.keep = [torch.from_numpy(w.D).to(dev)] + [torch.from_numpy(x).to(dev) for x in w.b]
        ctx.set_operator_stencil(w.n, w.dx, self.keep[0], self.keep[1:], 0.0, list(w.bc),
                                 ei.PREC_F64)
        self.state0 = torch.from_numpy(w.u0).to(dev)
        self.state = self.state0.clone()
        self.host0 = w.u0
        self.set_arith(self.arith)
        self.config = {"grid": [n] * 3, "h": w.h, "tol": w.tol, "bc": "neumann",
                       "method": self.method}

    def set_arith(self, arith):
        self.arith = arith
        self.dtype = "f64" if arith else DTYPE_FF
        self.bytes_per_point = BYTES_PER_POINT

    def _o(self, opts):
        o = {"arith": self.arith}
        o.update(opts or {})
        return o

    def step(self, ctx, opts=None):
        return ctx.step(self.ei.EXP_ROSENBROCK, self.w.h, self.state, self.ei.NONLIN_LOGISTIC,
                        self.w.tol, self._o(opts))

    def step_host(self, ctx, host, opts=None):
        return ctx.step_host(self.ei.EXP_ROSENBROCK, self.w.h, host, self.ei.NONLIN_LOGISTIC,
                             self.w.tol, self._o(opts))

    def kernel(self, fused):
        fmt = "double" if self.arith else "float-float"
        return (f"k_newton2_tma<{fmt}> (two Newton iterations per launch)"
                if fused == 2 else f"k_newton_tma<{fmt}> (one Newton iteration per launch)")


class Adr3dFF(Adr3d):
    """The headline step in the float-float format (FP32 pipes)."""

    arith = 0

    def __init__(self, torch, ei, W, dev, ctx, n):
        Adr3d.__init__(self, torch, ei, W, dev, ctx, n)
        self.name = WORKLOAD + "_float_float"


class Adr3dFp32(Adr3d):
    """512^3 reduced-precision form: FP32 vectors and stencil, exponential Euler."""

    arith = 0

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
        # per point-iteration as the scope counts it: w 4 + w' 4 + p 16 + the
        # operator as its inputs (D 4 + b 12); the library stores the seven
        # coefficients instead (52 B: bytes_per_point_stored)
        self.bytes_per_point = 40
        self.bytes_per_point_stored = 52
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
    arith = 0

    def __init__(self, torch, ei, W, dev, ctx, n):
        kind = "fast" if self.fast else "full"
        self.name, self.method = f"combustion_{n}_fp64_exp_euler_{kind}", "exp_euler"
        self.dtype = DTYPE_FF
        self.ei, self.w = ei, W.combustion_3d(n=n)
        w = self.w
        self.npts = n ** 3
        self.keep = []
        ctx.set_operator_stencil(w.n, w.dx, w.D, list(w.b), 0.0, list(w.bc), ei.PREC_F64)
        self.state0 = torch.from_numpy(w.u0).to(dev)
        self.state = self.state0.clone()
        self.host0 = w.u0
        # constant coefficients: the scope's count is w 8 + w' 8 + p 16; the
        # pair kernel reads the operator from its coefficient table (as stored:
        # 32 bytes; 88 with the seven coefficient arrays)
        self.bytes_per_point = CONST_BYTES_PER_POINT
        self.bytes_per_point_stored = BYTES_PER_POINT
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
    arith = 0

    def __init__(self, torch, ei, W, dev, ctx, n):
        kind = "sin(pi z)exp(-xy)" if self.data else "homogeneous"
        self.name = f"heat_{n}_dirichlet_{'data' if self.data else 'hom'}_exp_euler"
        self.method = "exp_euler"
        self.dtype = DTYPE_FF
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
        self.bytes_per_point = CONST_BYTES_PER_POINT
        self.bytes_per_point_stored = BYTES_PER_POINT
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
        self.dtype = DTYPE_FF
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
    graph, h*rho(A) = 100, tol 1e-10, in native FP64 (arith = 1; 0: the
    float-float form)."""

    arith = 1

    def __init__(self, torch, ei, W, dev, ctx, n):
        self.name, self.method = "rgg_2^20_csr_phi1", "phi1"
        self.ei = ei
        self.set_arith(self.arith)
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
        self.n_full = n == 1 << 20

    @property
    def traffic_per_launch(self):
        if not self.n_full:
            return None
        return RGG_DRAM_BYTES_PER_LAUNCH_F64 if self.arith else RGG_DRAM_BYTES_PER_LAUNCH

    def set_arith(self, arith):
        self.arith = arith
        self.dtype = "f64" if arith else DTYPE_FF

    def _o(self, opts):
        o = {"arith": self.arith}
        o.update(opts or {})
        return o

    def step(self, ctx, opts=None):
        return ctx.phi_apply(1, self.h, self.state, self.out, self.tol, self._o(opts))

    def step_host(self, ctx, host, opts=None):
        # phi_1(hA)v of the same v every call: the result goes to its own buffer
        d = host.to(self.state.device, non_blocking=True)
        st = ctx.phi_apply(1, self.h, d, self.out, self.tol, self._o(opts))
        pinned_like(self, host).copy_(self.out, non_blocking=False)
        return st

    def kernel(self, fused):
        fmt = "double" if self.arith else "float-float"
        return f"k_csr_newton_sell<{fmt}> (slices of 32 rows, a lane a row)"


class AdvDiff2d(Workload):
    """phi_1(hA)v on the 64 x 64 advection-diffusion operator (homogeneous
    Dirichlet, D = 0.1, b = (-1, -0.5), h = 1e-3, tol 1e-10), the small
    configuration, in native FP64 (arith = 1; 0: the float-float form).  A call
    moves 131 KB: it is bound by launch and synchronisation latency."""

    arith = 1

    def __init__(self, torch, ei, W, dev, ctx, n):
        self.name, self.method = f"adv_diff_2d_{n}_phi1", "phi1"
        self.ei = ei
        self.set_arith(self.arith)
        w = W.adv_diff_2d(n=n)
        self.w = w
        self.npts = n * n
        ctx.set_operator_stencil(w.n, w.dx, w.D, [w.b[0], w.b[1]], 0.0, list(w.bc),
                                 ei.PREC_F64)
        self.h, self.tol = w.h, w.tol
        self.host0 = w.v
        self.state0 = torch.from_numpy(w.v).to(dev)
        self.state = self.state0.clone()
        self.out = torch.empty_like(self.state)
        self.bytes_per_point = 32.0  # w 8 + w' 8 + p 16 (constant coefficients)
        self.config = {"grid": [n, n], "h": self.h, "tol": self.tol, "bc": "dirichlet",
                       "method": self.method}

    traffic_per_launch = None
    l2_note = ("inputs fit in L2 (32 KB a vector) and L2 is not flushed: the call is "
               "bound by launch and synchronisation latency, not by memory")

    def set_arith(self, arith):
        self.arith = arith
        self.dtype = "f64" if arith else DTYPE_FF

    def _o(self, opts):
        o = {"arith": self.arith}
        o.update(opts or {})
        return o

    def step(self, ctx, opts=None):
        return ctx.phi_apply(1, self.h, self.state, self.out, self.tol, self._o(opts))

    def step_host(self, ctx, host, opts=None):
        d = host.to(self.state.device, non_blocking=True)
        st = ctx.phi_apply(1, self.h, d, self.out, self.tol, self._o(opts))
        pinned_like(self, host).copy_(self.out, non_blocking=False)
        return st

    def kernel(self, fused):
        fmt = "double" if self.arith else "float-float"
        return f"k_newton_tma<{fmt}> / k_newton2_tma (64 x 64, latency-bound)"


class PhiKAdr3d(Adr3d):
    """phi_2(hA)v on the 256^3 advection-diffusion operator of the headline
    workload, h = 5e-4 (h rho ~ 600: the a-priori rule takes several substeps,
    each an e^{tau A} run on the state and a psi run on v), tol 1e-10, FP64."""

    k = 2
    arith = 0

    def __init__(self, torch, ei, W, dev, ctx, n):
        Adr3d.__init__(self, torch, ei, W, dev, ctx, n)
        self.name, self.method = f"adr3d_{n}_phi{self.k}_substeps", f"phi_{self.k}(hA)v"
        self.h = 5e-4
        self.out = torch.empty_like(self.state)
        self.bytes_per_point = ALG_BYTES_PER_POINT
        self.bytes_per_point_stored = BYTES_PER_POINT
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
                      else DTYPE_FF)
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
        return (f"k_csr_newton_sell_c<{fmt}> (slices of 32 rows, complex w and p "
                f"interleaved, real H)")


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
    arith = 1  # FP64 batches: native FP64 (0: float-float)

    def __init__(self, torch, ei, W, dev, ctx, n, learned_opt=False):
        self.name = "batch_1024_2d" + ("_fp32" if self.prec else
                                       "_fp64" if self.arith else "_float_float")
        self.method = "phi1 (batched, persistent kernel)"
        self.dtype = ("f32 (float-float Newton sum)" if self.prec else
                      "f64" if self.arith else DTYPE_FF)
        self.ei = ei
        probs = W.batch_2d(count=n)
        self.tol = 1e-6 if self.prec else 1e-10
        t0 = time.perf_counter()
        opts = {"tile_rows": TILE_ROWS} if TILE_ROWS else {}
        if not self.prec and self.arith:
            opts["arith"] = 1
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


class Batch2dFF(Batch2d):
    arith = 0


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
    problem, ei_phi_apply in native FP64 with the a-priori schedule, one problem
    after the other (tol 1e-6, the accuracy the FP32 form states).  A step is
    one pass over all problems."""

    arith = 1

    def __init__(self, torch, ei, W, dev, ctx, n):
        self.name = "batch_1024_2d_fp64_plain_loop"
        self.method = "phi1 (one ei_phi_apply per problem, a-priori schedule)"
        self.dtype = "f64" if self.arith else DTYPE_FF
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
            o = {"arith": self.arith}
            o.update(opts or {})
            st = c.phi_apply(1, p.h, v[a:b], self.out[a:b], self.tol, o)
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
        return ("k_newton_tma<double> (per-problem launches)" if self.arith
                else "k_newton2_tma<float-float> (per-problem launches)")


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


WORKLOADS = {"adr3d": Adr3d, "adr3d_ff": Adr3dFF, "adr3d_fp32": Adr3dFp32, "rgg_csr": RggCsr,
             "adv_diff_2d": AdvDiff2d, "batch": Batch2d, "batch_ff": Batch2dFF,
             "batch_fp32": Batch2dFp32, "adr3d_learned": Adr3dLearned,
             "adr3d_fp32_learned": Adr3dFp32Learned, "rgg_csr_learned": RggCsrLearned,
             "batch_learned_fp32": Batch2dLearnedFp32, "batch_plain_fp64_loop": Batch2dPlainLoop,
             "combustion": Combustion3d, "combustion_fast": Combustion3dFast,
             "combustion_nonlin": NonlinEval, "heat_dirichlet_data": HeatDirichlet,
             "heat_dirichlet_hom": HeatDirichletHom, "phi2_adr3d": PhiKAdr3d,
             "spin_bath": SpinBath, "spin_bath_fp32": SpinBathFp32}
DEFAULT_N = {"adr3d": N_SIDE, "adr3d_ff": N_SIDE, "adr3d_fp32": 512, "rgg_csr": 1 << 20,
             "adv_diff_2d": 64, "batch": 1024, "batch_ff": 1024,
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


def timed_steps(wl, ctx, args, torch, dev, stream, dist, local):
    """W untimed warm-up steps on a copy, then K steps from the initial state
    between CUDA events on the library's stream, with the clocks sampled
    during the timed region."""
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
    r = {"launches": 0, "matvecs": [], "degrees": [], "learned_flags": [], "learned_kept": None}
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(args.steps):
        st = wl.step(ctx)
        r["launches"] += st.launches
        r["matvecs"].append(st.matvecs)
        r["degrees"].append(st.degree_list())
        r["learned_flags"].append(int(getattr(st, "learned", 0)))
        if hasattr(st, "learned_kept"):
            r["learned_kept"] = st.learned_kept
    e1.record(stream)
    torch.cuda.synchronize(dev)
    r["clocks"] = sampler.stop()
    r["ms"] = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    if dist is not None:
        dist.barrier()
    # the dominant kernel: per-launch CUDA events around every Newton launch of
    # two further steps (profile option), same stream, same sizes
    wl.state_reset()
    prof_ms, prof_n, fused, prof_bytes, prof_nb = 0.0, 0, 1, 0.0, 0
    for _ in range(2):
        st = wl.step(ctx, {"profile": 1})
        prof_ms += st.newton_ms
        prof_n += st.newton_timed
        prof_nb += getattr(st, "newton_bounded", 0)
        fused = st.newton_fused
        prof_bytes += getattr(st, "timed_bytes", 0.0)
    r.update(prof_ms=prof_ms, prof_n=prof_n, fused=fused, prof_bytes=prof_bytes, last=st,
             prof_bounded=prof_nb)
    return r


def roofline(wl, r, args, npts):
    """The roofline object of the dominant kernel from the profiled launches."""
    hbm, peak_kind = peaks()
    prof_ms, prof_n, fused, prof_bytes, st = (r["prof_ms"], r["prof_n"], r["fused"],
                                              r["prof_bytes"], r["last"])
    if prof_n == 0 and hasattr(st, "point_iters"):
        # batched pass: one persistent launch; algorithmic bytes of all its sweeps
        # over the measured time per pass
        avg_launch_s = r["ms"] * 1e-3 / args.steps
        achieved = wl.bytes_per_point * st.point_iters / avg_launch_s / 1e9
    elif hasattr(st, "timed_bytes"):
        # many problems, one launch sequence each: bytes of all timed launches
        # over their summed time
        avg_launch_s = prof_ms / max(prof_n, 1) * 1e-3
        achieved = prof_bytes / max(prof_ms * 1e-3, 1e-12) / 1e9
    else:
        avg_launch_s = prof_ms / max(prof_n, 1) * 1e-3
        achieved = wl.bytes_per_point * npts * fused / avg_launch_s / 1e9
    traffic = getattr(wl, "traffic_per_launch", None)
    # a constant operator (D, b and c constants): the pair kernel reads the
    # coefficient table instead of the seven arrays
    table = getattr(st, "coef_table", 0) > 0
    if isinstance(wl, Adr3d) and wl.dtype == DTYPE_FF and fused == 2:
        # the float-float pair kernel (ncu)
        per_pt = TABLE_PAIR_DRAM_BYTES_PER_POINT if table else PAIR_DRAM_BYTES_PER_POINT
        traffic = per_pt * npts if per_pt else None
    out = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
           "frac": achieved / hbm,
           "traffic": traffic,
           "kernel": wl.kernel(fused) + (", the operator as its coefficient table"
                                         if table else ""),
           "bytes_per_launch": (prof_bytes / max(prof_n, 1)) if prof_bytes
           else wl.bytes_per_point * npts * fused,
           "avg_launch_us": avg_launch_s * 1e6, "launches_timed": prof_n,
           "iterations_per_launch": fused,
           "us_per_iteration": avg_launch_s * 1e6 / fused,
           "peak_kind": peak_kind,
           "paper_gflops": FLOPS_PER_POINT_PAPER * npts * fused / avg_launch_s / 1e9}
    stored = getattr(wl, "bytes_per_point_stored", None)
    if table:
        stored = CONST_BYTES_PER_POINT  # w, w' and p only
    if stored:
        out["bytes_per_point"] = wl.bytes_per_point
        out["bytes_per_point_stored"] = stored
        out["frac_stored"] = stored * npts / avg_launch_s / 1e9 / hbm
    if type(wl).__name__ in ("RggCsr", "RggCsrLearned") and wl.arith:
        # native FP64: the HBM bound and the FP64-pipe bound (2 flops an entry,
        # 12 a row: the update, the Newton sum and two squared norms) are close;
        # report against the larger
        sm_mhz = peaks_sm_mhz()
        fpk = SMS * FP64_FLOPS_PER_SM_CLK * sm_mhz * 1e6 / 1e12
        flops = 2.0 * wl.config["nnz"] + 12.0 * npts
        t_alu = flops / (fpk * 1e12)
        t_hbm = wl.bytes_per_point * npts / (hbm * 1e9)
        out.update({"t_alu_us": t_alu * 1e6, "t_hbm_us": t_hbm * 1e6,
                    "fp64_tflops": flops / avg_launch_s / 1e12, "fp64_peak": fpk,
                    "fp64_frac": flops / avg_launch_s / 1e12 / fpk})
        if t_alu > t_hbm:
            out.update({"bound": "alu", "achieved": flops / avg_launch_s / 1e12, "peak": fpk,
                        "unit": "TFLOP/s", "frac": flops / avg_launch_s / 1e12 / fpk,
                        "peak_kind": f"derived: {SMS} SMs x {FP64_FLOPS_PER_SM_CLK} FP64 "
                                     f"flop/clk x {sm_mhz:.0f} MHz"})
    if type(wl).__name__ in ("Adr3d", "Adr3dFF", "Adr3dLearned"):
        # the scope's algorithmic bytes (72 per point-iteration: the operator as
        # its inputs D, b, u_n) against measured HBM; the stored-coefficient
        # count (88) kept beside it; DRAM bytes from ncu where captured
        alg = ALG_BYTES_PER_POINT * npts * fused / avg_launch_s / 1e9
        dram = (PAIR_DRAM_BYTES_PER_POINT if (not wl.arith and fused == 2)
                else NATIVE_DRAM_BYTES_PER_POINT if (wl.arith and fused == 1) else None)
        traffic = dram * npts if dram is not None else None
        hb = {"bound": "hbm", "achieved": alg, "peak": hbm, "unit": "GB/s", "frac": alg / hbm,
              "traffic": traffic, "bytes_per_point": ALG_BYTES_PER_POINT,
              "bytes_per_launch": ALG_BYTES_PER_POINT * npts * fused,
              "bytes_per_launch_stored": BYTES_PER_POINT * npts,
              "frac_stored": BYTES_PER_POINT * npts / avg_launch_s / 1e9 / hbm,
              "dram_frac": (traffic / avg_launch_s / 1e9 / hbm) if traffic else None,
              "peak_kind": peak_kind}
        if wl.arith:
            # native FP64: bound by the FP64 pipe (min of the two rooflines)
            sm_mhz = peaks_sm_mhz()
            fpk = SMS * FP64_FLOPS_PER_SM_CLK * sm_mhz * 1e6 / 1e12
            # launches in the p-norm bound mode skip the squared norm of p
            nb = r.get("prof_bounded", 0)
            fpp = (FP64_FLOPS_PER_POINT * (prof_n - nb)
                   + FP64_FLOPS_PER_POINT_BOUNDED * nb) / max(prof_n, 1)
            tf = fpp * npts * fused / avg_launch_s / 1e12
            t_alu = fpp * npts * fused / (fpk * 1e12)
            t_hbm = ALG_BYTES_PER_POINT * npts * fused / (hbm * 1e9)
            out.update({"bound": "alu" if t_alu >= t_hbm else "hbm", "achieved": tf,
                        "peak": fpk, "unit": "TFLOP/s", "frac": tf / fpk, "traffic": traffic,
                        "alu": "FP64 pipe", "flops_per_point": fpp,
                        "launches_bounded": nb,
                        "peak_kind": f"derived: {SMS} SMs x {FP64_FLOPS_PER_SM_CLK} FP64 "
                                     f"flop/clk x {sm_mhz:.0f} MHz",
                        "t_alu_us": t_alu * 1e6, "t_hbm_us": t_hbm * 1e6, "hbm": hb})
        else:
            out.update(hb)
            out["kernel"] = wl.kernel(fused)
            out.update({"avg_launch_us": avg_launch_s * 1e6, "launches_timed": prof_n,
                        "iterations_per_launch": fused,
                        "us_per_iteration": avg_launch_s * 1e6 / fused})
    if isinstance(out.get("hbm"), dict):
        with_nominal(out["hbm"])
    return with_nominal(out)


def first_step_state(wl, ctx, torch):
    """u_1 of one step from u_0 (the first timed step's result) on the host, and
    the step's stats."""
    wl.state_reset()
    st = wl.step(ctx)
    torch.cuda.synchronize()
    return wl.state.double().cpu().numpy().reshape(wl.w.u0.shape), st


def rel_errors(u1, ref, u0):
    inc = np.linalg.norm((u1 - u0) - (ref - u0)) / np.linalg.norm(ref - u0)
    state = np.linalg.norm(u1 - ref) / np.linalg.norm(ref)
    return float(inc), float(state)


def cpu_leg(w, gpu_states, gpu_stats):
    """The oracle on the host (rank 0, N = 1): one whole step from u_0 with the
    serial oracle (the cpu_baseline), one with the all-core slab oracle, and the
    relative error of each GPU form's first step against the serial result."""
    from oracle import leja as L
    from oracle import newton as Nw
    from oracle import operators as O
    from oracle import slab as S

    xi = L.leja_points(100)
    op = O.StencilOperator(w.n, w.dx, w.D, w.b, bc=w.bc)
    t0 = time.perf_counter()
    ref, ost = Nw.exp_rosenbrock_step(op, w.u0, w.h, w.tol, xi=xi)
    t_serial = time.perf_counter() - t0
    del op
    sop = S.SlabStencil(w.n, w.dx, w.D, w.b, bc=w.bc)
    t0 = time.perf_counter()
    ref_s, sst = S.exp_rosenbrock_step(sop, w.u0, w.h, w.tol, xi=xi)
    t_all = time.perf_counter() - t0
    sop.close()
    errs = {}
    for name, u1 in gpu_states.items():
        inc, state = rel_errors(u1, ref, w.u0)
        gst = gpu_stats[name]
        errs[name] = {"value": inc, "state": state,
                      "of": "first step from u0, full field: ||du_gpu - du_oracle|| / "
                            "||du_oracle|| with du = u1 - u0 (state: ||u1 - u1_oracle|| / "
                            "||u1_oracle||), FP64 oracle",
                      "bound": 1e-9,
                      "s_and_degrees_match_oracle": bool(gst.s == ost.s and
                                                         gst.degree_list() == list(ost.degrees))}
    slab_agree, _ = rel_errors(ref_s, ref, w.u0)
    cores = S.host_threads()
    cpu = {"value": 1.0 / t_serial, "unit": "steps/s", "cores": 1, "kind": "oracle",
           "sample": (f"one whole exponential Rosenbrock-Euler step of the {w.n[0]}^3 workload "
                      f"from u0 with the serial oracle (numpy/decimal, 1 thread): {t_serial:.1f} s, "
                      f"s = {ost.s}, degrees {list(ost.degrees)}"),
           "nproc": os.cpu_count(),
           "all_cores": {"value": 1.0 / t_all, "unit": "steps/s", "cores": cores,
                         "kind": "oracle (z-slabs on host threads, oracle/slab.py)",
                         "sample": f"the same whole step: {t_all:.1f} s; increment within "
                                   f"{slab_agree:.1e} of the serial oracle"}}
    return cpu, errs


def cpu_leg_phi(wl, gpu_out, gpu_stats):
    """The oracle on the host for a phi_1(hA)v workload (graph or 2D stencil):
    the whole call with the serial oracle (the cpu_baseline, calls/s), and the
    relative error of each GPU form's result against it (full vector)."""
    from oracle import leja as L
    from oracle import newton as Nw
    from oracle import operators as O
    from paper_1309_4616_gb300 import workloads as W

    xi = L.leja_points(100)
    if isinstance(wl, RggCsr):
        g = W.rgg_graph(n=wl.npts)
        op = O.CsrOperator(g.n, g.rowptr, g.col, g.val, -g.deg_w)
        what = f"one phi_1(hA)v call on the {g.n}-node graph"
    else:
        w = wl.w
        op = O.StencilOperator(w.n, w.dx, w.D, w.b, bc=w.bc)
        what = f"one phi_1(hA)v call on the {w.n[0]} x {w.n[1]} grid"
    t0 = time.perf_counter()
    ref, ost = Nw.phi_apply(op, 1, wl.h, wl.host0, wl.tol, xi=xi)
    t_serial = time.perf_counter() - t0
    ref = np.asarray(ref).ravel()
    errs = {}
    for name, got in gpu_out.items():
        gst = gpu_stats[name]
        errs[name] = {"value": float(np.linalg.norm(got.ravel() - ref) / np.linalg.norm(ref)),
                      "of": "||out_gpu - out_oracle|| / ||out_oracle||, full vector, FP64 oracle",
                      "bound": 1e-9,
                      "s_and_degrees_match_oracle": bool(gst.s == ost.s and
                                                         gst.degree_list() == list(ost.degrees))}
    cpu = {"value": 1.0 / t_serial, "unit": "steps/s", "cores": 1, "kind": "oracle",
           "sample": (f"{what} with the serial oracle (numpy, 1 thread): {t_serial:.2f} s, "
                      f"s = {ost.s}, degrees {list(ost.degrees)}"),
           "nproc": os.cpu_count()}
    return cpu, errs


def run_batch_vs_plain_loop(args):
    """The comparison the learned, FP32 and batched forms are built for: the
    1024 uneven 2D problems at tol 1e-6, (a) the learned schedule with FP32
    vectors in one persistent launch per pass, against (b) the plain method in
    native FP64, one ei_phi_apply per problem.  Both are timed the same way
    (W warm-up passes, K timed passes between CUDA events); both outputs are
    held against the FP64 oracle at tol 1e-10 on a fixed sample of problems."""
    import torch
    from paper_1309_4616_gb300 import build, ei
    from paper_1309_4616_gb300 import workloads as W
    build.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = ei.Context(0, stream)
    n = args.n if args.n is not None else 1024
    res = {}
    outs = {}
    for key, cls in (("learned_fp32_batched", Batch2dLearnedFp32),
                     ("plain_fp64_loop", Batch2dPlainLoop)):
        wl = cls(torch, ei, W, dev, ctx, n)
        r = timed_steps(wl, ctx, args, torch, dev, stream, None, 0)
        wl.state_reset()
        wl.step(ctx)
        torch.cuda.synchronize()
        outs[key] = wl.out.double().cpu().numpy()
        res[key] = {"value": args.steps / (r["ms"] * 1e-3), "unit": "passes/s",
                    "ms_per_pass": r["ms"] / args.steps, "dtype": wl.dtype,
                    "matvecs_per_pass": r["matvecs"][0], "gpu_launches": r["launches"],
                    "clocks": r["clocks"], "config": wl.config}
        probs, offsets = wl.probs, np.concatenate([[0], np.cumsum([p.v.size for p in wl.probs])])
    # errors against the FP64 oracle at tol 1e-10 on every 16th problem with
    # at most 160^2 points (the oracle finishes those in seconds)
    from oracle import leja as L
    from oracle import newton as Nw
    from oracle import operators as O
    xi = L.leja_points(100)
    sample = [i for i in range(0, len(probs), 16) if probs[i].v.size <= 160 * 160]
    worst = {k: 0.0 for k in outs}
    for i in sample:
        p = probs[i]
        ref, _ = Nw.phi_apply(O.StencilOperator(p.n, p.dx, p.D, p.b, bc=p.bc), 1, p.h,
                              p.v, 1e-10, xi=xi)
        for k, o in outs.items():
            g = o[offsets[i]:offsets[i + 1]].reshape(ref.shape)
            e = float(np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-300))
            worst[k] = max(worst[k], e)
    for k in res:
        res[k]["max_rel_err_vs_oracle_tol_1e-10"] = worst[k]
    a, b = res["learned_fp32_batched"], res["plain_fp64_loop"]
    line = {"metric": "passes/s of 1024 uneven 2D phi_1 problems at tol 1e-6",
            "value": a["value"], "unit": "passes/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": a["ms_per_pass"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": a["dtype"], "data": "synthetic",
            "config": {"workload": "learned_fp32_batched_vs_plain_fp64_loop",
                       "problems": n, "tol": 1e-6,
                       "error_sample": f"{len(sample)} problems (every 16th with <= 160^2 points)"},
            "forms": res, "speedup_vs_plain_fp64": a["value"] / b["value"]}
    print(json.dumps(line))
    ctx.close()


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

    r = timed_steps(wl, ctx, args, torch, dev, stream, dist, local)
    roof = roofline(wl, r, args, npts)
    ms = r["ms"]

    # the headline's float-float form: the same steps in the float-float format,
    # measured the same way on the same context
    forms = None
    headline = type(wl) is Adr3d
    states, stats1 = {}, {}
    phi_leg = type(wl) in (RggCsr, AdvDiff2d)
    if type(wl) in (Adr3d, RggCsr, AdvDiff2d):
        if headline:
            states["f64"], stats1["f64"] = first_step_state(wl, ctx, torch)
        elif phi_leg:
            stats1["f64"] = wl.step(ctx)
            states["f64"] = wl.out.cpu().numpy()
        wl.set_arith(0)
        rf = timed_steps(wl, ctx, args, torch, dev, stream, dist, local)
        if headline:
            states["float_float"], stats1["float_float"] = first_step_state(wl, ctx, torch)
        elif phi_leg:
            stats1["float_float"] = wl.step(ctx)
            states["float_float"] = wl.out.cpu().numpy()
        froof = roofline(wl, rf, args, npts)
        forms = {"float_float": {
            "value": args.steps * world / (rf["ms"] * 1e-3), "unit": "steps/s",
            "ms_per_step": rf["ms"] / args.steps, "dtype": DTYPE_FF,
            "matvecs_per_step": rf["matvecs"], "degrees": rf["degrees"][:3],
            "gpu_launches": rf["launches"], "roofline": froof, "clocks": rf["clocks"]}}
        wl.set_arith(1)

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

    cpu, errs = None, None
    if rank == 0 and world == 1 and not args.no_cpu and headline:
        cpu, errs = cpu_leg(wl.w, states, stats1)
        forms["float_float"]["rel_err"] = errs["float_float"]
    elif rank == 0 and world == 1 and not args.no_cpu and phi_leg:
        cpu, errs = cpu_leg_phi(wl, states, stats1)
        forms["float_float"]["rel_err"] = errs["float_float"]

    if rank == 0:
        steps_total = args.steps * world
        value = steps_total / (ms * 1e-3)
        esz = u_host.element_size()
        config = {"workload": wl.name, **wl.config, "parallelism": f"replicas x{world}",
                  "l2": getattr(wl, "l2_note",
                                "inputs larger than L2 (each vector >= 8 MB and the step's "
                                "working set >= 0.3 GB; 256^3: 134 MB per vector)"),
                  "matvecs_per_step": r["matvecs"], "degrees": r["degrees"][:3]}
        if r["learned_kept"] is not None and getattr(wl, "model", None) is not None:
            config["learned_problems_kept_per_pass"] = r["learned_kept"]
        elif any(r["learned_flags"]):
            config["learned_accepted_steps"] = sum(1 for f in r["learned_flags"] if f == 1)
        line = {
            "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": wl.dtype, "data": "synthetic", "config": config,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": k_e2e * world / e2e_s, "unit": "steps/s",
                    "h2d_bytes_per_step": npts * esz, "d2h_bytes_per_step": npts * esz},
            "gpu_launches": r["launches"],
            "clocks": r["clocks"],
        }
        if errs is not None:
            line["rel_err"] = errs["f64"]
        if forms is not None:
            line["forms"] = forms
        print(json.dumps(line))
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch_vs_plain_loop":
        run_batch_vs_plain_loop(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
