"""Training the schedule network on traces of the plain method, and loading it.

The plain method picks the substep count s by a conservative a priori rule
(Sec. III-C) and ends every substep by the a posteriori estimate.  A trace
records one phi_1 call of the plain method at a given s with no restart
(ei_options fixed_s, no_restart, learned = 2): the twelve features the
library reports for the call, whether every substep met the tolerance within
m_max, and then the largest degree.  For each problem, traces are taken at the
plain rule's s and at s/8, s/4, s/2, 2s and 4s.  The network learns the degree as a
fraction of m_max (output 0; rows that did not converge are masked out) and
the convergence logit (output 1).

Problems are seeded and synthetic, drawn from the four families the method
runs on, at sizes where one call takes about a millisecond:

  adv2d  2D advection-diffusion, N x N' interior grids with N in [24, 256],
         constant or sinusoidally varying D in [0.01, 1], constant b in
         [-1, 1]^2, Dirichlet or per-side mixed boundaries, v a sum of sine
         modes, a smooth cosine field or white noise;
  adr3d  3D advection-diffusion-reaction on N^3, N in [12, 64], with
         D = 1 + 0.5 sin sin sin, a smooth random b (max |b| = 2), Neumann
         boundaries, one exponential Euler or Rosenbrock-Euler step from four
         Gaussian bumps (phi_1 acts on F = A u + u(1-u));
  rgg    -(graph Laplacian) of random geometric graphs in the unit cube,
         2^11 to 2^17 nodes, mean degree 12, weights U[0.5, 2], v ~ N(0, 1).

h is drawn so that h*gamma (gamma a quarter of the Gershgorin interval's
width) is log-uniform over [0.05, 5000] in 2D, [0.05, 2000] in 3D, and h*rho
over [1, 200] for the graphs; tol is 1e-10, 1e-8 or 1e-6.

Everything runs through the library: the traces are its own plain method,
training is its own forward/backward/Adam kernels (ei_mlp_*).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import ei
from . import workloads as W

MODEL_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "schedule_mlp.npz")
M_MAX = 100
LAM, KAPPA = 0.2, 4.0


# ---------------------------------------------------------------------------
# problem families
# ---------------------------------------------------------------------------
def _sine_modes(rng, nx, ny, modes=8):
    x = (np.arange(nx) + 1) / (nx + 1)
    y = (np.arange(ny) + 1) / (ny + 1)
    v = np.zeros((ny, nx))
    for _ in range(modes):
        p, r = rng.integers(1, 17, size=2)
        v += rng.standard_normal() * np.outer(np.sin(r * math.pi * y), np.sin(p * math.pi * x))
    return v


def _cosine_field(rng, nx, ny):
    x = (np.arange(nx) + 1) / (nx + 1)
    y = (np.arange(ny) + 1) / (ny + 1)
    v = np.zeros((ny, nx))
    for _ in range(3):
        kx, ky = rng.integers(1, 6, size=2)
        px, py = rng.uniform(0, 2 * math.pi, size=2)
        v += rng.standard_normal() * np.outer(np.cos(ky * math.pi * y + py),
                                              np.cos(kx * math.pi * x + px))
    return v


class _Op:
    """An operator set on the context plus what a draw needs."""

    def __init__(self, kind, n, make_v, step=None):
        self.kind, self.n, self.make_v, self.step = kind, n, make_v, step


def _adv2d(torch, ctx, rng):
    nx = int(round(math.exp(rng.uniform(math.log(24), math.log(256)))))
    ny = nx if rng.uniform() < 0.5 else int(round(nx * rng.uniform(0.6, 1.4)))
    dx = (1.0 / (nx + 1), 1.0 / (ny + 1))
    D0 = math.exp(rng.uniform(math.log(0.01), math.log(1.0)))
    if rng.uniform() < 0.5:
        D = D0
    else:
        x = (np.arange(nx) + 1) * dx[0]
        y = (np.arange(ny) + 1) * dx[1]
        D = torch.from_numpy(D0 * (1 + 0.5 * np.outer(np.sin(2 * math.pi * y),
                                                      np.sin(2 * math.pi * x)))).cuda()
    b = [float(t) for t in rng.uniform(-1, 1, size=2)]
    bc = [0, 0, 0, 0] if rng.uniform() < 0.4 else [int(t) for t in rng.integers(0, 2, size=4)]
    ctx.set_operator_stencil((nx, ny), dx, D, b, 0.0, bc, ei.PREC_F64)

    def make_v(r):
        u = r.uniform()
        if u < 0.45:
            v = _sine_modes(r, nx, ny)
        elif u < 0.9:
            v = _cosine_field(r, nx, ny)
        else:
            v = r.standard_normal((ny, nx))
        return torch.from_numpy(np.ascontiguousarray(v)).cuda()
    return _Op("stencil", nx * ny, make_v)


def _adr3d(torch, ctx, rng):
    n = int(round(math.exp(rng.uniform(math.log(12), math.log(64)))))
    b = W.smooth_vector_field(rng, n)
    D = W.diffusion_field(n)
    dx = (1.0 / n,) * 3
    ctx.set_operator_stencil((n, n, n), dx, torch.from_numpy(D).cuda(),
                             [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in b], 0.0,
                             [1] * 6, ei.PREC_F64)

    def make_v(r):
        return torch.from_numpy(W.gaussian_bumps(r, n)).cuda()
    method = ei.EXP_ROSENBROCK if rng.uniform() < 0.6 else ei.EXP_EULER
    return _Op("stencil", n ** 3, make_v, step=method)


_GRAPHS = {}


def _rgg(torch, ctx, rng):
    n = int(2 ** rng.integers(11, 18))
    key = (n, int(rng.integers(0, 3)))
    if key not in _GRAPHS:
        _GRAPHS[key] = W.rgg_graph(n=n, seed=1000 + 17 * key[1] + n)
    g = _GRAPHS[key]
    ctx.set_operator_csr(g.n, torch.from_numpy(g.rowptr).cuda(), torch.from_numpy(g.col).cuda(),
                         torch.from_numpy(g.val).cuda(), torch.from_numpy(-g.deg_w).cuda())

    def make_v(r):
        return torch.from_numpy(r.standard_normal(g.n)).cuda()
    return _Op("csr", g.n, make_v)


FAMILIES = (("adv2d", _adv2d, 0.4), ("adr3d", _adr3d, 0.3), ("rgg", _rgg, 0.3))


# ---------------------------------------------------------------------------
# traces
# ---------------------------------------------------------------------------
def _call(ctx, op, h, v, tol, s):
    """One plain-method call at substep count s (0: the a priori rule) with
    no restart.  Returns (converged, stats)."""
    import torch
    opts = {"learned": 2}
    if s:
        opts.update(fixed_s=s, no_restart=1)
    if op.step is None:
        out = torch.empty_like(v)
        rc, st = ctx.phi_apply(1, h, v, out, tol, opts, check=False)
    else:
        u = v.clone()
        rc, st = ctx.step(op.step, h, u, ei.NONLIN_LOGISTIC, tol, opts, check=False)
    # a non-finite iterate (a non-normal operator whose spectrum leaves the
    # real interval) is an outcome of the method like reaching m_max
    if rc not in (ei.OK, ei.ERR_NOT_CONVERGED, ei.ERR_NONFINITE):
        ei._check(rc, "trace call")
    return rc == ei.OK, st


HG_RANGE = {"adv2d": (0.05, 5000.0), "adr3d": (0.05, 2000.0)}


def generate(count, seed, draws_per_op=6, log=None, budget_s=None):
    """At least `count` traces (or as many as `budget_s` seconds give).
    Returns X (rows x 12), Y (rows x 2), mask, the problem id of every row and
    its operator applications."""
    import torch
    rng = np.random.default_rng(seed)
    ctx = ei.Context()
    X, Y, M, P, Cst = [], [], [], [], []
    pid = 0
    next_log = 0
    t0 = time.time()
    names = [f[0] for f in FAMILIES]
    probs = np.array([f[2] for f in FAMILIES])
    while len(X) < count and (budget_s is None or time.time() - t0 < budget_s):
        fam = int(rng.choice(len(FAMILIES), p=probs / probs.sum()))
        op = FAMILIES[fam][1](torch, ctx, rng)
        alpha, beta = ctx.estimate_spectrum()
        gamma = 0.25 * (beta - alpha)
        rho = max(abs(alpha), abs(beta))
        for _ in range(draws_per_op):
            if op.kind == "csr":
                h = math.exp(rng.uniform(math.log(1.0), math.log(200.0))) / rho
            else:
                lo, hi = HG_RANGE[names[fam]]
                h = math.exp(rng.uniform(math.log(lo), math.log(hi))) / gamma
            tol = float(rng.choice([1e-10, 1e-8, 1e-6]))
            v = op.make_v(rng)
            ok, st = _call(ctx, op, h, v, tol, 0)
            if not ok:
                continue
            s_plain = st.s
            rows = [(ok, st)]
            for s in (s_plain // 8, s_plain // 4, s_plain // 2, 2 * s_plain, 4 * s_plain):
                if s >= 1 and s != s_plain:
                    rows.append(_call(ctx, op, h, v, tol, s))
            for ok_s, st_s in rows:
                X.append(st_s.feature_list())
                Y.append([st_s.degree_max / M_MAX if ok_s else 0.0, 1.0 if ok_s else 0.0])
                M.append(1.0 if ok_s else 0.0)
                P.append(pid)
                Cst.append(st_s.matvecs)
            pid += 1
        if log and len(X) >= next_log:
            log(f"traces {len(X)} problems {pid} {time.time() - t0:.0f}s")
            next_log += 10000
    ctx.close()
    return (np.array(X, dtype=np.float64), np.array(Y, dtype=np.float64),
            np.array(M, dtype=np.float64), np.array(P, dtype=np.int64),
            np.array(Cst, dtype=np.float64))


# ---------------------------------------------------------------------------
# training and the decision margins
# ---------------------------------------------------------------------------
def init_params(seed):
    """He-normal weights, zero biases, in the library's flat layout."""
    rng = np.random.default_rng(seed)
    sizes = (ei.MLP_INPUTS, 64, 64, 64, ei.MLP_OUTPUTS)
    parts = []
    for i in range(4):
        fi, fo = sizes[i], sizes[i + 1]
        parts.append(rng.standard_normal(fo * fi) * math.sqrt(2.0 / fi))
        parts.append(np.zeros(fo))
    return np.concatenate(parts).astype(np.float32)


def train(X, Y, mask, epochs=300, batch=4096, lr=2e-3, seed=0, log=None):
    """Adam with a cosine learning-rate decay, on the device, by the
    library's kernels.  Returns (model, final training loss)."""
    import torch
    rng = np.random.default_rng(seed)
    net = ei.Mlp()
    net.set_params(init_params(seed))
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    Yd = torch.from_numpy(Y.astype(np.float32)).cuda()
    Md = torch.from_numpy(mask.astype(np.float32)).cuda()
    n = X.shape[0]
    steps_per_epoch = max(1, n // batch)
    total = epochs * steps_per_epoch
    k = 0
    loss = float("nan")
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(n)).cuda()
        for b in range(steps_per_epoch):
            idx = perm[b * batch:(b + 1) * batch]
            rate = lr * 0.5 * (1 + math.cos(math.pi * k / total))
            last = (b == steps_per_epoch - 1)
            r = net.train_step(Xd[idx].contiguous(), Yd[idx].contiguous(), Md[idx].contiguous(),
                               rate, LAM, KAPPA, want_loss=last)
            if last:
                loss = r
            k += 1
        if log and (ep % 50 == 0 or ep == epochs - 1):
            log(f"epoch {ep} loss {loss:.5f}")
    return net, loss


def predict(net, X):
    import torch
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    out = torch.empty((X.shape[0], 2), dtype=torch.float32, device="cuda")
    net.forward(Xd, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def calibrate(net, X, Y, mask, pid, cost):
    """Margins (z_min, rho_m, delta_m) that minimise the operator applications
    of the held-out problems under the decision rule (the cheapest accepted
    q) in adaptive mode: a proposal at q is accepted when the plain method
    converged at that q and then costs what it cost there; a rejected one
    costs the work it did before reaching m_max plus the plain call.  Only
    the q values that have traces are candidates here."""
    O = predict(net, X)
    groups = {}
    for i, p in enumerate(pid):
        groups.setdefault(int(p), []).append(i)
    best = None
    for z_min in (-1.0, 0.0, 1.0, 2.0):
        for rho_m in (0.0, 0.05, 0.1, 0.2):
            for delta_m in (1.0, 2.0, 4.0, 8.0):
                total = plain = 0.0
                acc = 0
                for rows in groups.values():
                    by_q = {int(round(X[i, 3] * 10)): i for i in rows}
                    plain_cost = cost[rows[0]]  # the first row is the plain call
                    plain += plain_cost
                    chosen = None
                    for q in range(ei.MLP_MAX_Q + 1):
                        if q not in by_q:
                            continue
                        i = by_q[q]
                        need = M_MAX * O[i, 0] * (1 + rho_m) + delta_m
                        if O[i, 1] >= z_min and need <= M_MAX:
                            m = max(1, min(M_MAX, math.ceil(need)))
                            c = 2 ** q * (m + 1) - 1
                            if chosen is None or c < chosen[3]:
                                chosen = (q, i, m, c)
                    if chosen is None:
                        total += plain_cost
                        continue
                    q, i, m, _ = chosen
                    if mask[i] > 0:
                        total += cost[i]
                        acc += 1
                    else:
                        total += cost[i] + plain_cost
                if best is None or total < best[0]:
                    best = (total, z_min, rho_m, delta_m, acc / max(len(groups), 1),
                            total / plain)
    return {"z_min": best[1], "rho_m": best[2], "delta_m": best[3], "val_accept": best[4],
            "val_cost_ratio": best[5]}


def evaluate(net, count, seed, log=None):
    """The trained network against the plain method on fresh problems of the
    same families: for each, the plain call and the learned call on the same
    (h, tol, v).  Returns per-family totals of wall time, operator
    applications, proposals accepted, and the largest relative difference of
    the two results in units of tol."""
    import torch
    rng = np.random.default_rng(seed)
    ctx = ei.Context()
    ctx.set_schedule_model(net)
    names = [f[0] for f in FAMILIES]
    res = {n: {"calls": 0, "plain_s": 0.0, "learned_s": 0.0, "plain_matvecs": 0,
               "learned_matvecs": 0, "accepted": 0, "fallback": 0, "no_proposal": 0,
               "max_diff_over_tol": 0.0} for n in names}
    per_fam = max(1, count // len(FAMILIES))
    for fam, (name, make, _) in enumerate(FAMILIES):
        done = 0
        while done < per_fam:
            op = make(torch, ctx, rng)
            alpha, beta = ctx.estimate_spectrum()
            gamma = 0.25 * (beta - alpha)
            rho = max(abs(alpha), abs(beta))
            for _ in range(3):
                if op.kind == "csr":
                    h = math.exp(rng.uniform(math.log(1.0), math.log(200.0))) / rho
                else:
                    lo, hi = HG_RANGE[name]
                    h = math.exp(rng.uniform(math.log(lo), math.log(hi))) / gamma
                tol = float(rng.choice([1e-10, 1e-8, 1e-6]))
                v = op.make_v(rng)
                outs = {}
                failed = False
                # warm both paths, then time the second pair.  The warm-up calls use
                # h (1 + 2^-40): the context keeps the plain rule's last plan, and a
                # timed call that repeated the warm-up's exact (h, interval) would skip
                # the a-priori search, which a call whose step or interval moves (every
                # Rosenbrock step) cannot
                for i, mode in enumerate((0, 1, 0, 1)):
                    hh = h * (1.0 + 2.0 ** -40) if i < 2 else h
                    torch.cuda.synchronize()
                    t = time.perf_counter()
                    if op.step is None:
                        out = torch.empty_like(v)
                        rc, st = ctx.phi_apply(1, hh, v, out, tol, {"learned": mode}, check=False)
                    else:
                        out = v.clone()
                        rc, st = ctx.step(op.step, hh, out, ei.NONLIN_LOGISTIC, tol,
                                          {"learned": mode}, check=False)
                    dt = time.perf_counter() - t
                    if rc != ei.OK:  # the plain method fails too (non-finite iterates)
                        failed = True
                        break
                    outs[mode] = (out, st, dt)
                if failed:
                    res[name]["skipped"] = res[name].get("skipped", 0) + 1
                    continue
                (yp, sp, tp), (yl, sl, tl) = outs[0], outs[1]
                if op.step is not None:
                    yp, yl = yp - v, yl - v
                r = res[name]
                r["calls"] += 1
                r["plain_s"] += tp
                r["learned_s"] += tl
                r["plain_matvecs"] += sp.matvecs
                r["learned_matvecs"] += sl.matvecs
                r["accepted"] += sl.learned == 1
                r["fallback"] += sl.learned == 2
                r["no_proposal"] += sl.learned == 3
                nrm = float(torch.linalg.vector_norm(yp))
                diff = float(torch.linalg.vector_norm(yl - yp)) / (nrm if nrm > 0 else 1.0)
                r["max_diff_over_tol"] = max(r["max_diff_over_tol"], diff / tol)
                done += 1
        if log:
            log(f"{name}: {res[name]}")
    ctx.close()
    return res


def save(net, decision, meta, path=MODEL_PATH):
    np.savez(path, theta=net.get_params(), z_min=decision["z_min"], rho_m=decision["rho_m"],
             delta_m=decision["delta_m"], q_max=ei.MLP_MAX_Q, meta=json.dumps(meta))


def load(path=MODEL_PATH, device=0):
    """The trained network as an ei.Mlp with its decision margins."""
    z = np.load(path)
    net = ei.Mlp(device)
    net.set_params(z["theta"])
    net.set_decision(float(z["z_min"]), float(z["rho_m"]), float(z["delta_m"]), int(z["q_max"]))
    return net


def main():
    ap = argparse.ArgumentParser(description="generate traces and train the schedule network")
    ap.add_argument("--traces", type=int, default=100000)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=MODEL_PATH)
    ap.add_argument("--save-traces", default=None)
    ap.add_argument("--load-traces", default=None, help="traces saved by an earlier run")
    ap.add_argument("--budget-s", type=float, default=None, help="wall-clock limit of generation")
    ap.add_argument("--evaluate", type=int, default=0, help="held-out problems to compare on")
    args = ap.parse_args()
    from . import build
    build.build()
    log = lambda m: print(m, flush=True)  # noqa: E731
    t0 = time.time()
    if args.load_traces:
        z = np.load(args.load_traces)
        X, Y, M, P, Cst = z["X"], z["Y"], z["M"], z["P"], z["C"]
    else:
        X, Y, M, P, Cst = generate(args.traces, args.seed, log=log, budget_s=args.budget_s)
    t_gen = time.time() - t0
    if args.save_traces:
        np.savez(args.save_traces, X=X, Y=Y, M=M, P=P, C=Cst)
    # held-out problems for the margins
    rng = np.random.default_rng(args.seed + 1)
    probs = np.unique(P)
    val = set(rng.choice(probs, size=max(1, len(probs) // 10), replace=False).tolist())
    is_val = np.array([p in val for p in P])
    t1 = time.time()
    net, loss = train(X[~is_val], Y[~is_val], M[~is_val], epochs=args.epochs, seed=args.seed,
                      log=log)
    t_train = time.time() - t1
    dec = calibrate(net, X[is_val], Y[is_val], M[is_val], P[is_val], Cst[is_val])
    meta = {"traces": int(X.shape[0]), "problems": int(len(probs)),
            "train_rows": int((~is_val).sum()), "val_rows": int(is_val.sum()),
            "train_loss": loss, "gen_s": t_gen, "train_s": t_train, "epochs": args.epochs,
            "seed": args.seed, **dec}
    save(net, dec, meta, args.out)
    print(json.dumps(meta))
    if args.evaluate:
        net.set_decision(dec["z_min"], dec["rho_m"], dec["delta_m"], ei.MLP_MAX_Q)
        print(json.dumps(evaluate(net, args.evaluate, args.seed + 7, log=log)))


if __name__ == "__main__":
    main()
