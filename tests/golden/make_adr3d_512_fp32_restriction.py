"""Writes adr3d_512_fp32_restriction.npz, the expected values of the 512^3
reduced-precision parity test.

The workload: the 3D advection-diffusion-reaction problem on 512^3 cells with
its seeded fields (paper_1309_4616_gb300.workloads.adr_3d_fp32: Neumann faces,
logistic g, h = 5e-5, tol 1e-6), 10 exponential Euler steps (Eq. (2)).  The
FP64 oracle runs on the FP32-rounded D, b and u0, the inputs the FP32 form
receives, with its steps split over the host cores (oracle/slab.py, equal to
the serial oracle up to the norms' summation order).  Stored: the final state
on the 64^3 restriction (every 8th point per axis from offset 4), u0 on the
same points, and per step the substep count and Newton degrees.

Calls only oracle/ and the seeded input generators.  About 30-60 minutes and
25 GB of host memory:  python tests/golden/make_adr3d_512_fp32_restriction.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import leja as L  # noqa: E402
from oracle import slab as S  # noqa: E402
from paper_1309_4616_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "adr3d_512_fp32_restriction.npz")
RESTRICT = (slice(4, None, 8),) * 3


def main():
    w = W.adr_3d_fp32(n=512)
    D = w.D.astype(np.float32).astype(np.float64)
    b = [x.astype(np.float32).astype(np.float64) for x in w.b]
    u = w.u0.astype(np.float32).astype(np.float64)
    u0r = u[RESTRICT].copy()
    xi = L.leja_points(100)
    sop = S.SlabStencil(w.n, w.dx, D, b, bc=w.bc)
    del D, b
    s_list, deg_list = [], []
    t0 = time.perf_counter()
    for k in range(w.steps):
        u, st = S.exp_euler_step(sop, u, w.h, w.tol, xi=xi)
        s_list.append(st.s)
        deg_list.append(list(st.degrees))
        print(f"step {k + 1}/{w.steps}: s = {st.s}, degrees {st.degrees}, "
              f"{time.perf_counter() - t0:.0f} s", flush=True)
    sop.close()
    degs = np.full((w.steps, max(len(d) for d in deg_list)), -1, dtype=np.int64)
    for k, d in enumerate(deg_list):
        degs[k, : len(d)] = d
    np.savez_compressed(OUT, u=u[RESTRICT].copy(), u0=u0r, s=np.array(s_list), degrees=degs,
                        h=w.h, tol=w.tol, steps=w.steps)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
