"""What the trained network gains over the method without it.

On fresh problems of the three training families (a seed the training never
used), the plain a priori schedule and the learned schedule (the committed
network, adaptive mode: its substep count, the per-substep a posteriori
stop) run the same calls.  The learned calls must be accepted almost always,
cost no more operator applications, and take less wall time in total; both
results pass the same a posteriori test, so they differ by a small multiple
of tol."""
import pytest

from gpu_helpers import require_gpu

pytestmark = pytest.mark.gpu


def test_trained_network_gains():
    torch, ei = require_gpu()
    from paper_1309_4616_gb300 import learned
    net = learned.load()
    res = learned.evaluate(net, 45, seed=4242)
    print()
    print(f"{'family':8s} {'calls':>5s} {'plain s':>9s} {'learned s':>9s} {'ratio':>6s} "
          f"{'plain mv':>9s} {'learned mv':>10s} {'accepted':>8s} {'diff/tol':>8s}")
    tp = tl = mp = ml = 0.0
    for name, r in res.items():
        print(f"{name:8s} {r['calls']:5d} {r['plain_s']:9.4f} {r['learned_s']:9.4f} "
              f"{r['learned_s'] / r['plain_s']:6.3f} {r['plain_matvecs']:9d} "
              f"{r['learned_matvecs']:10d} {r['accepted']:8d} {r['max_diff_over_tol']:8.1f}")
        assert r["calls"] >= 15
        assert r["accepted"] >= 0.85 * r["calls"], name
        assert r["max_diff_over_tol"] <= 1e3, name
        tp += r["plain_s"]
        tl += r["learned_s"]
        mp += r["plain_matvecs"]
        ml += r["learned_matvecs"]
    print(f"total: time ratio {tl / tp:.3f}, matvec ratio {ml / mp:.3f}")
    assert ml <= 1.02 * mp
    assert tl < tp
